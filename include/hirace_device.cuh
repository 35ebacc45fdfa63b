/*
 * hirace_device.cuh - device side of the race checker.
 *
 * 1. The shadow value and the FSM step (Sec. IV-B, Algorithm 1
 *    UpdateShadow): unpack <oState, oTid, oBC, oWC>, compareTids -> tRel,
 *    checkSync -> sRel, one flat-table lookup, pack <nState, tid, bc, wc>,
 *    atomicCAS until it sticks.  The library's trace kernels use the same
 *    code through hr_fsm_step().
 * 2. Source-level instrumentation for hand-written kernels (Sec. IV-A: the
 *    paper's wrapper intercepts indexing, atomics and barriers): call
 *    hr_access() next to every monitored
 *    load, store or atomic, and use hr_syncthreads() / hr_syncwarp() in place
 *    of __syncthreads() / __syncwarp() so the thread-private clocks advance
 *    at the barrier (Sec. III-A Scenario 2).
 *
 * Shadow value, 8 bytes per monitored word (Sec. IV-B default):
 *     bits 63..59  FSM state (5 bits; 0 = INIT, 31 = RACE)
 *     bits 58..56  kernel tag (kernel ordinal mod 8; a stale tag reads as INIT)
 *     bits 55..40  bc of the last accessor (16 bits)
 *     bits 39..32  wc of the last accessor (8 bits)
 *     bits 31..0   global tid of the last accessor
 * Only the fields a state needs are kept; the others are zero, so an access
 * that leaves the summarised history unchanged produces the identical value
 * and needs no atomic at all:
 *     thread scope: tid, bc, wc      warp scope: warp's first tid, bc, wc
 *     block scope:  block's first tid, bc      grid scope and RACE: nothing
 *
 * Compact shadow value, 4 bytes per word (the shadow size is configurable,
 * Sec. IV-B), for regions whose thread ids fit T = tid_bits bits:
 *     bits 31..27  FSM state        bits 26..24  kernel tag
 *     bits 23..T+W bc (B = 24 - T - W bits)
 *     bits T+W-1..T wc (W = (24 - T) / 2 bits)     bits T-1..0  tid
 * e.g. T = 16: bc and wc 4 bits each; T = 18: 3 bits each.  The state
 * machine runs on the 8-byte layout; the compact word is only its storage
 * form (hr_expand32 / hr_compress64), so both sizes take the same
 * transitions.  A tid, bc or wc beyond its width is HR_ERR_CLOCK_OVERFLOW.
 */
#ifndef HIRACE_DEVICE_CUH
#define HIRACE_DEVICE_CUH

#include <stdint.h>

#include "hirace.h"

#define HR_SH_STATE_SHIFT 59
#define HR_SH_KTAG_SHIFT 56
#define HR_SH_BC_SHIFT 40
#define HR_SH_WC_SHIFT 32
#define HR_WC_MAX 255u
#define HR_BC_MAX 65535u
#define HR_STATE_INIT 0u
#define HR_STATE_RACE 31u
#define HR_CAS_RETRY_CAP 4096

/* scope level of a state (bits 5..7 of a table entry) */
#define HR_LVL_INIT 0u
#define HR_LVL_THREAD 1u
#define HR_LVL_WARP 2u
#define HR_LVL_BLOCK 3u
#define HR_LVL_GRID 4u
#define HR_LVL_RACE 5u

/* thread relation (compareTids) and sync status (checkSync) labels */
#define HR_TREL_SAME 0u
#define HR_TREL_WARP 1u
#define HR_TREL_BLOCK 2u
#define HR_TREL_GRID 3u
#define HR_SREL_UNSYNC 0u
#define HR_SREL_WARP 1u
#define HR_SREL_BLOCK 2u

/* Thread geometry of a region: divisions by block_dim and warp_size use a
 * precomputed 64-bit reciprocal (Lemire, Kaser & Kurz 2019, "Faster remainder
 * by direct computation": q = hi64(n * (floor((2^64-1)/d) + 1)) is exact for
 * every 32-bit n); magic 0 stands for d == 1. */
typedef struct hr_geom {
    uint32_t block_dim;
    uint32_t warp_size;
    uint64_t bd_magic;
    uint64_t ws_magic;
    uint32_t bd_shift;     /* log2(block_dim) when block_dim and warp_size are both powers of two, else ~0u */
    uint32_t ws_shift;     /* log2(warp_size) in that case */
    uint32_t shadow_bytes; /* shadow bytes per word: 8, 4 (compact packing) or 24 (every-epoch mode) */
    uint32_t tid_bits;     /* compact packing: width of the tid field (4..22) */
    uint32_t report_mode;  /* HR_REPORT_FIRST or HR_REPORT_EVERY_EPOCH */
    uint32_t pad;
} hr_geom;

/* Everything an instrumented kernel needs for one region; pass by value. */
typedef struct hr_view {
    unsigned long long* shadow;     /* n_words shadow values */
    hr_race* ring;                  /* ring_cap race records */
    unsigned long long* n_races;    /* race counter (may exceed ring_cap) */
    unsigned int* error;            /* sticky error word (first error wins) */
    unsigned int* flags;            /* HR_FLAG_* bits */
    const unsigned char* table;     /* 2048-byte FSM table */
    unsigned long long n_words;
    unsigned long long ring_cap;
    hr_geom geom;
    unsigned int kernel;            /* kernel ordinal of the launch being checked */
    unsigned int region;
    hr_filter filter;               /* monitored words, blocks and lanes (hr_set_filter) */
} hr_view;

/* Thread-private clocks of an instrumented thread. */
typedef struct hr_clock {
    uint32_t tid;
    uint32_t bc;
    uint32_t wc;
} hr_clock;

#ifdef __CUDACC__

static __device__ __forceinline__ uint32_t hr_fastdiv(uint32_t n, uint64_t magic)
{
    return magic ? (uint32_t)__umul64hi(magic, (uint64_t)n) : n;
}

/* Thread relation of `tid` to the stored last accessor `otid` (compareTids). */
static __device__ __forceinline__ uint32_t hr_thread_rel(uint32_t tid, uint32_t otid, const hr_geom& g)
{
    if (otid == tid) return HR_TREL_SAME;
    if (g.bd_shift != ~0u) {
        const uint32_t x = tid ^ otid;
        if (x >> g.bd_shift) return HR_TREL_GRID;
        const uint32_t m = g.block_dim - 1u;
        return ((tid & m) >> g.ws_shift) == ((otid & m) >> g.ws_shift) ? HR_TREL_WARP : HR_TREL_BLOCK;
    }
    const uint32_t blk = hr_fastdiv(tid, g.bd_magic);
    const uint32_t oblk = hr_fastdiv(otid, g.bd_magic);
    if (oblk != blk) return HR_TREL_GRID;
    const uint32_t warp = hr_fastdiv(tid - blk * g.block_dim, g.ws_magic);
    const uint32_t owarp = hr_fastdiv(otid - oblk * g.block_dim, g.ws_magic);
    return owarp == warp ? HR_TREL_WARP : HR_TREL_BLOCK;
}

/* First tid of the warp / block of `tid` (canonical identities of WARP and
 * BLOCK states). */
static __device__ __forceinline__ void hr_scope_heads(uint32_t tid, const hr_geom& g, uint32_t* warp_head,
                                                      uint32_t* block_head)
{
    if (g.bd_shift != ~0u) {
        const uint32_t loc = tid & (g.block_dim - 1u);
        *block_head = tid - loc;
        *warp_head = tid - (loc & (g.warp_size - 1u));
        return;
    }
    const uint32_t blk = hr_fastdiv(tid, g.bd_magic);
    const uint32_t loc = tid - blk * g.block_dim;
    const uint32_t warp = hr_fastdiv(loc, g.ws_magic);
    *block_head = tid - loc;
    *warp_head = tid - (loc - warp * g.warp_size);
}

/* One FSM transition: fold access (tid, op, bc, wc) of kernel tag `ktag` into
 * the raw shadow value `o`.  `table` is the 2048-entry flat table (shared or
 * global memory).  Returns the new packed value; *raced is set to 1 + the old
 * state when this access moves the word into RACE, else left alone. */
static __device__ __forceinline__ uint64_t hr_fsm_step(uint64_t o, uint32_t tid, uint32_t op, uint32_t bc,
                                                       uint32_t wc, uint32_t ktag, const hr_geom& g,
                                                       const unsigned char* table, uint32_t* raced)
{
    uint32_t os = (uint32_t)(o >> HR_SH_STATE_SHIFT);
    if (os != HR_STATE_INIT && (uint32_t)((o >> HR_SH_KTAG_SHIFT) & 7u) != ktag) os = HR_STATE_INIT;
    const uint32_t trel = hr_thread_rel(tid, (uint32_t)o, g);
    const uint32_t obc = (uint32_t)(o >> HR_SH_BC_SHIFT) & 0xFFFFu;
    const uint32_t owc = (uint32_t)(o >> HR_SH_WC_SHIFT) & 0xFFu;
    const uint32_t srel = bc != obc ? HR_SREL_BLOCK : (wc != owc ? HR_SREL_WARP : HR_SREL_UNSYNC);
    const uint32_t e = table[(os << 6) | (op << 4) | (trel << 2) | srel];
    const uint32_t ns = e & 31u;
    const uint32_t lvl = e >> 5;
    uint64_t n = ((uint64_t)ns << HR_SH_STATE_SHIFT) | ((uint64_t)ktag << HR_SH_KTAG_SHIFT);
    if (lvl >= HR_LVL_THREAD && lvl <= HR_LVL_BLOCK) {
        uint32_t wh, bh;
        hr_scope_heads(tid, g, &wh, &bh);
        const uint32_t who = lvl == HR_LVL_THREAD ? tid : (lvl == HR_LVL_WARP ? wh : bh);
        const uint64_t clk = lvl == HR_LVL_BLOCK ? ((uint64_t)bc << HR_SH_BC_SHIFT)
                                                 : (((uint64_t)bc << HR_SH_BC_SHIFT) | ((uint64_t)wc << HR_SH_WC_SHIFT));
        n |= clk | who;
    }
    if (ns == HR_STATE_RACE && os != HR_STATE_RACE) *raced = 1u + os;
    return n;
}

/* hr_fsm_step for a power-of-two geometry (g.bd_shift != ~0u; bd_shift and
 * ws_shift are g.bd_shift and g.ws_shift): the same transition, with
 * compareTids and the scope heads reduced to bit operations on the two tids
 * and the new value assembled from its two 32-bit halves.  Two tids in one
 * block (their xor below 2^bd_shift) share a warp when the xor is also below
 * 2^ws_shift; a warp's first tid clears the low min(ws_shift, bd_shift) bits,
 * a block's the low bd_shift bits. */
static __device__ __forceinline__ uint64_t hr_fsm_step_pow2(uint64_t o, uint32_t tid, uint32_t op, uint32_t bc,
                                                            uint32_t wc, uint32_t ktag, uint32_t bd_shift,
                                                            uint32_t ws_shift, const unsigned char* table,
                                                            uint32_t* raced)
{
    const uint32_t ohi = (uint32_t)(o >> 32);
    uint32_t os = ohi >> (HR_SH_STATE_SHIFT - 32);
    if (os != HR_STATE_INIT && ((ohi >> (HR_SH_KTAG_SHIFT - 32)) & 7u) != ktag) os = HR_STATE_INIT;
    const uint32_t x = tid ^ (uint32_t)o;
    const uint32_t trel = x == 0u ? HR_TREL_SAME
                        : (x >> bd_shift) ? HR_TREL_GRID
                        : (x >> ws_shift) ? HR_TREL_BLOCK : HR_TREL_WARP;
    const uint32_t obc = (ohi >> (HR_SH_BC_SHIFT - 32)) & 0xFFFFu;
    const uint32_t owc = (ohi >> (HR_SH_WC_SHIFT - 32)) & 0xFFu;
    const uint32_t srel = bc != obc ? HR_SREL_BLOCK : (wc != owc ? HR_SREL_WARP : HR_SREL_UNSYNC);
    const uint32_t e = table[(os << 6) | (op << 4) | (trel << 2) | srel];
    const uint32_t ns = e & 31u;
    const uint32_t lvl = e >> 5;
    uint32_t hi = (ns << (HR_SH_STATE_SHIFT - 32)) | (ktag << (HR_SH_KTAG_SHIFT - 32));
    uint32_t lo = 0u;
    if (lvl >= HR_LVL_THREAD && lvl <= HR_LVL_BLOCK) {
        const uint32_t low = lvl == HR_LVL_THREAD ? 0u : (lvl == HR_LVL_WARP ? min(ws_shift, bd_shift) : bd_shift);
        lo = tid & ~((1u << low) - 1u);
        hi |= (bc << (HR_SH_BC_SHIFT - 32)) | (lvl == HR_LVL_BLOCK ? 0u : (wc << (HR_SH_WC_SHIFT - 32)));
    }
    if (ns == HR_STATE_RACE && os != HR_STATE_RACE) *raced = 1u + os;
    return ((uint64_t)hi << 32) | lo;
}

static __device__ __forceinline__ uint64_t hr_ld_relaxed(const unsigned long long* p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

static __device__ __forceinline__ uint32_t hr_ld_relaxed32(const unsigned int* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

/* widths of the compact packing's clock fields */
static __device__ __forceinline__ uint32_t hr_wc_bits(const hr_geom& g) { return (24u - g.tid_bits) >> 1; }
static __device__ __forceinline__ uint32_t hr_bc_bits(const hr_geom& g) { return 24u - g.tid_bits - hr_wc_bits(g); }

/* Whether a filter selects only part of the accesses (or folds a symmetric group). */
static __device__ __forceinline__ bool hr_filter_active(const hr_filter& f)
{
    return f.word_hi != 0 || f.block_hi != 0 || f.lane_mask != 0xFFFFFFFFu || f.sym_hi != 0;
}

/* Whether thread *tid's access to `word` is monitored under filter f; *idx gets
 * the shadow index of the word (word - word_lo inside a window).  A member of
 * the filter's symmetric group is first folded onto the group's
 * representative block: *tid and the word become the representative's. */
static __device__ __forceinline__ bool hr_monitored(const hr_filter& f, const hr_geom& g, uint32_t* tid_io,
                                                    unsigned long long word, unsigned long long* idx)
{
    uint32_t tid = *tid_io;
    if (f.sym_hi != 0) {
        const uint32_t b = g.bd_shift != ~0u ? tid >> g.bd_shift : hr_fastdiv(tid, g.bd_magic);
        if (b > f.sym_lo && b < f.sym_hi) {
            const uint32_t m = b - f.sym_lo;
            const unsigned long long shift = (unsigned long long)m * f.sym_stride;
            if (word < shift) return false;
            word -= shift;
            tid -= m * g.block_dim;
            *tid_io = tid;
        }
    }
    *idx = word;
    if (f.word_hi != 0) {
        if (word < f.word_lo || word >= f.word_hi) return false;
        *idx = word - f.word_lo;
    }
    if (f.block_hi != 0 || f.lane_mask != 0xFFFFFFFFu) {
        uint32_t blk, loc;
        if (g.bd_shift != ~0u) {
            blk = tid >> g.bd_shift;
            loc = tid & (g.block_dim - 1u);
        } else {
            blk = hr_fastdiv(tid, g.bd_magic);
            loc = tid - blk * g.block_dim;
        }
        const uint32_t lane = g.ws_shift != ~0u ? (loc & (g.warp_size - 1u))
                                                : loc - hr_fastdiv(loc, g.ws_magic) * g.warp_size;
        if (f.block_hi != 0 && (blk < f.block_lo || blk >= f.block_hi)) return false;
        if (((f.lane_mask >> lane) & 1u) == 0) return false;
    }
    return true;
}

/* Whether an access's identity and clocks fit the region's packing. */
static __device__ __forceinline__ bool hr_fits(uint32_t tid, uint32_t bc, uint32_t wc, const hr_geom& g)
{
    if (g.shadow_bytes != 4) return bc <= HR_BC_MAX && wc <= HR_WC_MAX;
    return (tid >> g.tid_bits) == 0 && (wc >> hr_wc_bits(g)) == 0 && (bc >> hr_bc_bits(g)) == 0;
}

/* compact storage form -> the 8-byte layout */
static __device__ __forceinline__ uint64_t hr_expand32(uint32_t x, const hr_geom& g)
{
    const uint32_t t = g.tid_bits, w = hr_wc_bits(g);
    const uint32_t tid = x & ((1u << t) - 1u);
    const uint32_t wc = (x >> t) & ((1u << w) - 1u);
    const uint32_t bc = (x & 0x00FFFFFFu) >> (t + w);
    return ((uint64_t)(x >> 24) << HR_SH_KTAG_SHIFT) | ((uint64_t)bc << HR_SH_BC_SHIFT) |
           ((uint64_t)wc << HR_SH_WC_SHIFT) | tid;
}

/* 8-byte layout -> compact storage form (fields must fit, see hr_fits) */
static __device__ __forceinline__ uint32_t hr_compress64(uint64_t v, const hr_geom& g)
{
    const uint32_t t = g.tid_bits, w = hr_wc_bits(g);
    const uint32_t wc = (uint32_t)(v >> HR_SH_WC_SHIFT) & 0xFFu;
    const uint32_t bc = (uint32_t)(v >> HR_SH_BC_SHIFT) & 0xFFFFu;
    return ((uint32_t)(v >> HR_SH_KTAG_SHIFT) << 24) | (bc << (t + w)) | (wc << t) | (uint32_t)v;
}

/* Shadow word `word` of a region, in the 8-byte layout whatever its storage size. */
static __device__ __forceinline__ uint64_t hr_shadow_load(unsigned long long* shadow, unsigned long long word,
                                                          const hr_geom& g)
{
    if (g.shadow_bytes == 4) return hr_expand32(hr_ld_relaxed32((unsigned int*)shadow + word), g);
    return hr_ld_relaxed(shadow + word);
}

/* CAS of shadow word `word` from o to n (8-byte layout); returns the value seen. */
static __device__ __forceinline__ uint64_t hr_shadow_cas(unsigned long long* shadow, unsigned long long word,
                                                         uint64_t o, uint64_t n, const hr_geom& g)
{
    if (g.shadow_bytes == 4)
        return hr_expand32(atomicCAS((unsigned int*)shadow + word, hr_compress64(o, g), hr_compress64(n, g)), g);
    return atomicCAS(shadow + word, (unsigned long long)o, (unsigned long long)n);
}

static __device__ __forceinline__ void hr_set_error(unsigned int* err, unsigned int code)
{
    atomicCAS(err, 0u, code);
}

/* Append one race record; the counter keeps counting past the capacity. */
static __device__ __forceinline__ void hr_append_race(hr_race* ring, unsigned long long ring_cap,
                                                      unsigned long long* n_races, unsigned int* flags,
                                                      uint32_t word, uint32_t tid, uint32_t kernel,
                                                      uint32_t epoch, uint32_t region, uint32_t op,
                                                      uint32_t prior)
{
    const unsigned long long slot = atomicAdd(n_races, 1ull);
    if (slot < ring_cap) {
        hr_race r;
        r.word = word;
        r.tid = tid;
        r.kernel = (uint16_t)kernel;
        r.epoch = (uint16_t)epoch;
        r.region = (uint16_t)region;
        r.op = (uint8_t)op;
        r.prior = (uint8_t)prior;
        ring[slot] = r;
    } else {
        atomicOr(flags, HR_FLAG_TRUNCATED);
    }
}

/* ---------------------------------------------------------------------------
 * Every-epoch reporting (report mode HR_REPORT_EVERY_EPOCH)
 *
 * The first-race FSM stops at RACE; this mode keeps checking and reports each
 * (word, kernel, epoch) in which some access completes a racy pair.  Deciding
 * that exactly for every later access needs, for each of the two conflict
 * kinds (bit 0: reads and writes; bit 1: atomics and writes), where the
 * accesses holding it sit: a later access conflicts with bit b's holders when
 * one of them is in another block, or in its block and epoch but another
 * warp, or in its warp and sub-epoch but another thread (Sec. II-B).  So each
 * bit gets its own 8-byte summary, the narrowest scope holding all its
 * accessors of the latest epoch plus that epoch's clocks:
 *     bits 63..59 level (0 none, 1 thread, 2 warp, 3 block, 4 grid)
 *     bits 58..56 kernel tag, 55..40 bc, 39..32 wc,
 *     bits 31..0  the thread, the warp's first thread or the block's first thread
 * A word's shadow is three 8-byte values in three arrays of n_words values
 * (24 bytes per word): the bit-0 summary, the bit-1 summary, and 1 + (kernel
 * << 16 | epoch) of the last epoch reported.  An access updates the summaries
 * of the bits it holds (CAS), then - after a sequentially consistent fence,
 * so that of two concurrent conflicting accesses at least one sees the other
 * - reads the summaries of the bits it conflicts with.
 * ------------------------------------------------------------------------- */
#define HR_EP_NONE 0u
#define HR_EP_THREAD 1u
#define HR_EP_WARP 2u
#define HR_EP_BLOCK 3u
#define HR_EP_GRID 4u

static __device__ __forceinline__ uint64_t hr_ep_pack(uint32_t lvl, uint32_t ktag, uint32_t bc, uint32_t wc,
                                                      uint32_t who)
{
    return ((uint64_t)lvl << HR_SH_STATE_SHIFT) | ((uint64_t)ktag << HR_SH_KTAG_SHIFT) |
           ((uint64_t)bc << HR_SH_BC_SHIFT) | ((uint64_t)wc << HR_SH_WC_SHIFT) | who;
}

static __device__ __forceinline__ uint32_t hr_ep_level(uint64_t s, uint32_t ktag)
{
    const uint32_t lvl = (uint32_t)(s >> HR_SH_STATE_SHIFT);
    return (lvl != HR_EP_NONE && (uint32_t)((s >> HR_SH_KTAG_SHIFT) & 7u) != ktag) ? HR_EP_NONE : lvl;
}

/* Summary of one conflict bit after adding an access of thread tid at (bc, wc). */
static __device__ __forceinline__ uint64_t hr_ep_update(uint64_t s, uint32_t tid, uint32_t bc, uint32_t wc,
                                                        uint32_t ktag, const hr_geom& g)
{
    const uint32_t lvl = hr_ep_level(s, ktag);
    if (lvl == HR_EP_NONE) return hr_ep_pack(HR_EP_THREAD, ktag, bc, wc, tid);
    if (lvl == HR_EP_GRID) return s;
    const uint32_t rel = hr_thread_rel(tid, (uint32_t)s, g);
    if (rel == HR_TREL_GRID) return hr_ep_pack(HR_EP_GRID, ktag, 0, 0, 0);
    const uint32_t obc = (uint32_t)(s >> HR_SH_BC_SHIFT) & 0xFFFFu;
    if (obc != bc) return hr_ep_pack(HR_EP_THREAD, ktag, bc, wc, tid);  // a later epoch of the block
    if (lvl == HR_EP_BLOCK) return s;
    uint32_t wh, bh;
    hr_scope_heads(tid, g, &wh, &bh);
    if (rel == HR_TREL_BLOCK) return hr_ep_pack(HR_EP_BLOCK, ktag, bc, 0, bh);
    const uint32_t owc = (uint32_t)(s >> HR_SH_WC_SHIFT) & 0xFFu;
    if (owc != wc) return hr_ep_pack(HR_EP_THREAD, ktag, bc, wc, tid);  // a later sub-epoch of the warp
    if (lvl == HR_EP_WARP || rel == HR_TREL_SAME) return s;
    return hr_ep_pack(HR_EP_WARP, ktag, bc, wc, wh);
}

/* Whether a conflict bit's holders (summary s) include an access unordered with
 * an access of thread tid at (bc, wc) from another thread. */
static __device__ __forceinline__ bool hr_ep_pred(uint64_t s, uint32_t tid, uint32_t bc, uint32_t wc, uint32_t ktag,
                                                  const hr_geom& g)
{
    const uint32_t lvl = hr_ep_level(s, ktag);
    if (lvl == HR_EP_NONE) return false;
    if (lvl == HR_EP_GRID) return true;
    const uint32_t rel = hr_thread_rel(tid, (uint32_t)s, g);
    if (rel == HR_TREL_GRID) return true;
    if (((uint32_t)(s >> HR_SH_BC_SHIFT) & 0xFFFFu) != bc) return false;  // earlier epochs of its block
    if (lvl == HR_EP_BLOCK || rel == HR_TREL_BLOCK) return true;
    if (((uint32_t)(s >> HR_SH_WC_SHIFT) & 0xFFu) != wc) return false;    // earlier sub-epochs of its warp
    return lvl == HR_EP_WARP || rel != HR_TREL_SAME;
}

/* Apply one access in every-epoch mode to shadow index idx of a region whose
 * three arrays start at `shadow` (stride n_words).  Reports the race under
 * `report_word`, once per (word, kernel, epoch).  Returns 0 or
 * HR_ERR_CONTENTION when a CAS loop reached `cap` retries. */
static __device__ __forceinline__ uint32_t hr_ep_apply(unsigned long long* shadow, unsigned long long n_words,
                                                       unsigned long long idx, uint32_t report_word, uint32_t tid,
                                                       uint32_t op, uint32_t bc, uint32_t wc, uint32_t kernel,
                                                       const hr_geom& g, hr_race* ring, unsigned long long ring_cap,
                                                       unsigned long long* n_races, unsigned int* flags,
                                                       uint32_t region, uint32_t cap)
{
    const uint32_t ktag = kernel & 7u;
    const uint32_t holds = op == HR_R ? 1u : (op == HR_A ? 2u : 3u);
    const uint32_t against = op == HR_R ? 2u : (op == HR_A ? 1u : 3u);
    for (uint32_t b = 0; b < 2; ++b) {
        if (((holds >> b) & 1u) == 0) continue;
        unsigned long long* p = shadow + b * n_words + idx;
        uint64_t o = hr_ld_relaxed(p);
        for (uint32_t tries = 0;; ++tries) {
            const uint64_t n = hr_ep_update(o, tid, bc, wc, ktag, g);
            if (n == o) break;
            const uint64_t seen = atomicCAS(p, (unsigned long long)o, (unsigned long long)n);
            if (seen == o) break;
            if (tries + 1 >= cap) return HR_ERR_CONTENTION;
            o = seen;
        }
    }
    asm volatile("fence.sc.gpu;" ::: "memory");
    uint32_t prior = 0;
    for (uint32_t b = 0; b < 2 && !prior; ++b) {
        if (((against >> b) & 1u) == 0) continue;
        const uint64_t s = hr_ld_relaxed(shadow + b * n_words + idx);
        if (hr_ep_pred(s, tid, bc, wc, ktag, g)) prior = hr_ep_level(s, ktag);
    }
    if (!prior) return 0;
    unsigned long long* st = shadow + 2 * n_words + idx;
    const unsigned long long mine = ((((unsigned long long)kernel) << 16) | bc) + 1ull;
    unsigned long long cur = hr_ld_relaxed(st);
    for (uint32_t tries = 0; cur < mine && tries < cap; ++tries) {
        const unsigned long long seen = atomicCAS(st, cur, mine);
        if (seen == cur) {
            hr_append_race(ring, ring_cap, n_races, flags, report_word, tid, kernel, bc, region, op, prior);
            return 0;
        }
        cur = seen;
    }
    return cur < mine ? HR_ERR_CONTENTION : 0u;
}

/* ---------------------------------------------------------------------------
 * Hand instrumentation
 * ------------------------------------------------------------------------- */

/* Clocks of the calling thread at kernel start (1-D or flattened launch). */
static __device__ __forceinline__ hr_clock hr_clock_init(void)
{
    hr_clock c;
    const uint32_t tpb = blockDim.x * blockDim.y * blockDim.z;
    const uint32_t b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const uint32_t t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    c.tid = b * tpb + t;
    c.bc = 0;
    c.wc = 0;
    return c;
}

/* __syncthreads() plus the block-clock advance (bc++, wc = 0). */
static __device__ __forceinline__ void hr_syncthreads(hr_clock& c)
{
    __syncthreads();
    c.bc += 1;
    c.wc = 0;
}

/* full-mask __syncwarp() plus the warp-clock advance (wc++). */
static __device__ __forceinline__ void hr_syncwarp(hr_clock& c)
{
    __syncwarp();
    c.wc += 1;
}

/* Record one access (op = HR_R, HR_W or HR_A) to monitored word `word`.
 * Call it right next to the real access; the two need not be atomic together
 * (Sec. III-A).  Errors go to the view's sticky error word; the first one
 * wins and hr_report returns it. */
static __device__ __forceinline__ void hr_access(const hr_view& v, unsigned long long word, uint32_t op,
                                                 const hr_clock& c)
{
    hr_clock cf = c;  // the representative's thread when a symmetric group folds this one
    if (hr_filter_active(v.filter) && !hr_monitored(v.filter, v.geom, &cf.tid, word, &word)) return;
    // the word races are reported on (absolute, the representative's under a symmetric group)
    const unsigned long long abs_word = word + (v.filter.word_hi != 0 ? v.filter.word_lo : 0ull);
    if (word >= v.n_words || op > HR_A) {
        hr_set_error(v.error, word >= v.n_words ? HR_ERR_RANGE : HR_ERR_UNSUPPORTED);
        return;
    }
    if (!hr_fits(cf.tid, cf.bc, cf.wc, v.geom)) {
        hr_set_error(v.error, HR_ERR_CLOCK_OVERFLOW);
        return;
    }
    if (v.geom.report_mode == HR_REPORT_EVERY_EPOCH) {
        const uint32_t st = hr_ep_apply(v.shadow, v.n_words, word, (uint32_t)abs_word, cf.tid, op, cf.bc, cf.wc,
                                        v.kernel, v.geom, v.ring, v.ring_cap, v.n_races, v.flags, v.region,
                                        HR_CAS_RETRY_CAP);
        if (st) hr_set_error(v.error, st);
        return;
    }
    const uint32_t ktag = v.kernel & 7u;
    uint64_t o = hr_shadow_load(v.shadow, word, v.geom);
    for (int it = 0; it < HR_CAS_RETRY_CAP; ++it) {
        uint32_t raced = 0;
        const uint64_t n = hr_fsm_step(o, cf.tid, op, cf.bc, cf.wc, ktag, v.geom, v.table, &raced);
        if (n == o) return;
        const uint64_t prev = hr_shadow_cas(v.shadow, word, o, n, v.geom);
        if (prev == o) {
            if (raced)
                hr_append_race(v.ring, v.ring_cap, v.n_races, v.flags, (uint32_t)abs_word, cf.tid, v.kernel, cf.bc,
                               v.region, op, raced - 1u);
            return;
        }
        o = prev;
    }
    hr_set_error(v.error, HR_ERR_CONTENTION);
}

/* ---------------------------------------------------------------------------
 * Shadow in shared memory for a block's __shared__ array
 *
 * A __shared__ array belongs to one block, so only that block's threads can
 * touch it and its shadow can live beside it in shared memory: the FSM step is
 * the same (thread relations never reach "other block"), the CAS is a
 * shared-memory atomic, and the shadow is fresh in every launch.  Races go to
 * the region's report ring with word = block index * n_words + word, the
 * numbering a trace of the same kernel uses for per-block arrays.
 * ------------------------------------------------------------------------- */
typedef struct hr_smem_view {
    unsigned long long* shadow; /* n_words shadow values in this block's shared memory */
    uint32_t n_words;           /* monitored words of the block's array */
    uint32_t word_base;         /* this block's first word in race reports */
} hr_smem_view;

/* Every thread of the block calls this before its first monitored access:
 * zeroes the shadow `buf` (n_words values in shared memory) and waits for the
 * whole block (a barrier that precedes all monitored accesses, so it orders
 * nothing the checker sees). */
static __device__ __forceinline__ hr_smem_view hr_smem_begin(unsigned long long* buf, uint32_t n_words)
{
    const uint32_t nt = blockDim.x * blockDim.y * blockDim.z;
    const uint32_t t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    for (uint32_t i = t; i < n_words; i += nt) buf[i] = 0ull;
    __syncthreads();
    hr_smem_view sv;
    sv.shadow = buf;
    sv.n_words = n_words;
    sv.word_base = (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)) * n_words;
    return sv;
}

/* hr_access for word `word` of the block's shared array; `v` supplies the
 * table, geometry, kernel ordinal, report ring and error word. */
static __device__ __forceinline__ void hr_access_shared(const hr_view& v, const hr_smem_view& sv, uint32_t word,
                                                        uint32_t op, const hr_clock& c)
{
    if (word >= sv.n_words || op > HR_A) {
        hr_set_error(v.error, word >= sv.n_words ? HR_ERR_RANGE : HR_ERR_UNSUPPORTED);
        return;
    }
    if (c.bc > HR_BC_MAX || c.wc > HR_WC_MAX) {
        hr_set_error(v.error, HR_ERR_CLOCK_OVERFLOW);
        return;
    }
    unsigned long long* p = sv.shadow + word;
    const uint32_t ktag = v.kernel & 7u;
    uint64_t o = *(volatile unsigned long long*)p;
    for (int it = 0; it < HR_CAS_RETRY_CAP; ++it) {
        uint32_t raced = 0;
        const uint64_t n = hr_fsm_step(o, c.tid, op, c.bc, c.wc, ktag, v.geom, v.table, &raced);
        if (n == o) return;
        const uint64_t prev = atomicCAS(p, (unsigned long long)o, (unsigned long long)n);
        if (prev == o) {
            if (raced)
                hr_append_race(v.ring, v.ring_cap, v.n_races, v.flags, sv.word_base + word, c.tid, v.kernel, c.bc,
                               v.region, op, raced - 1u);
            return;
        }
        o = prev;
    }
    hr_set_error(v.error, HR_ERR_CONTENTION);
}

#endif /* __CUDACC__ */

#ifdef __cplusplus
extern "C" {
#endif
/* Host: a by-value view of one region for instrumented kernels.  The view is
 * valid while the context lives; its kernel ordinal is the region's current
 * one (advanced by hr_sync).  Returns HR_ERR_INVALID for a bad region. */
hr_status hr_device_view(hr_ctx* ctx, uint32_t region, hr_view* out);
#ifdef __cplusplus
}
#endif

#endif /* HIRACE_DEVICE_CUH */

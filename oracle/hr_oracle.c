/*
 * CPU oracle for the HiRace race check.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant with the CUDA
 * checker; the only thing the two have in common is the documented 16-byte
 * trace record layout (word, tid, wc, bc, kernel, op, flags).
 *
 * Three independent pieces, each slow and plain on purpose:
 *
 *  hro_validate     Recomputes every thread's block clock (bc) and warp clock
 *                   (wc) from its own __syncthreads / __syncwarp records and
 *                   checks they equal the clocks the producer wrote
 *                   (Sec. III-A, Scenario 2: each thread's private block
 *                   clock advances when it passes a block barrier; warp
 *                   barriers add a warp clock, Sec. III-B).
 *
 *  hro_bruteforce   The race definition itself (Sec. II-A): two accesses to
 *                   the same word race when they come from different threads,
 *                   at least one modifies the word, they are not both atomic,
 *                   and no happens-before order separates them.  The GPU
 *                   happens-before model is Sec. II-B: __syncthreads orders a
 *                   block, __syncwarp orders a warp, nothing orders two
 *                   blocks of one kernel, and kernel end orders everything.
 *                   Every pair of accesses on a word is tested (the
 *                   two-thread theorem of Sec. II-B: a race always shows up
 *                   between two threads).  Words with very many accesses use
 *                   the same definition written as pair *counts* per scope.
 *
 *  hro_serial_fsm   A serial restatement of the paper's parallel FSM
 *                   (Sec. III, Algorithm 1): per word it keeps a constant-size
 *                   summary of the history, read -> compare thread ids ->
 *                   compare clocks -> decide the transition -> write back,
 *                   one record at a time in trace order.  The summary is
 *                   written with explicit fields (how many blocks / warps /
 *                   threads share the current scope and the exact set of
 *                   operation kinds seen in it), not with a transition table.
 *
 * Race key: (kernel, word, epoch).  The epoch of a racy word is
 *   e* = min over racy pairs (a, b) of max(bc_a, bc_b),
 * i.e. the block clock of the first wave, in wave order, that completes a racy
 * pair.  The wave of an access is (kernel, bc, wc); a trace is sorted by wave.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t word;
    uint32_t tid;
    uint16_t wc;
    uint16_t bc;
    uint16_t kernel;
    uint8_t op;
    uint8_t flags;
} hro_rec;

typedef struct {
    uint32_t word;
    uint16_t kernel;
    uint16_t epoch;
    uint8_t ops_mask;   /* ops (bit 1<<op) of accesses that can complete the first racy pair */
    uint8_t kinds_mask; /* racy pair kinds at e*: bit0 R-W, bit1 W-W, bit2 A-W, bit3 A-R; 0xFF unknown */
    uint8_t method;     /* 0 pairwise, 1 pair counts */
    uint8_t pad;
    uint32_t pad2;
} hro_race;

typedef struct {
    uint32_t word;
    uint32_t tid;
    uint16_t kernel;
    uint16_t epoch;
    uint8_t op;
    uint8_t pad[3];
} hro_report;

enum { OR_ = 0, OW_ = 1, OA_ = 2, OST_ = 3, OSW_ = 4 };
enum { PARTIAL_MASK_FLAG = 2 };

/* ---------------------------------------------------------------- helpers */

static int is_access(uint8_t op) { return op <= OA_; }
static int modifies(uint8_t op) { return op == OW_ || op == OA_; }

/* Sec. II-A: at least one write; atomics count as modifying accesses but two
 * atomics never race with each other (they are a separate class of action,
 * Sec. III-B). */
static int conflicting(uint8_t a, uint8_t b)
{
    return (modifies(a) || modifies(b)) && !(a == OA_ && b == OA_);
}

static uint64_t wave_of(const hro_rec* r)
{
    return ((uint64_t)r->kernel << 32) | ((uint64_t)r->bc << 16) | (uint64_t)r->wc;
}

/* Sec. II-B: blocks are unordered inside a kernel; __syncthreads orders the
 * threads of a block (different bc); different warps of a block are unordered
 * between two __syncthreads; __syncwarp orders the lanes of a warp. */
static int concurrent(const hro_rec* a, const hro_rec* b, uint32_t bd, uint32_t ws)
{
    uint32_t block_a = a->tid / bd, block_b = b->tid / bd;
    if (block_a != block_b) return 1;
    if (a->bc != b->bc) return 0;
    uint32_t warp_a = (a->tid % bd) / ws, warp_b = (b->tid % bd) / ws;
    if (warp_a != warp_b) return 1;
    return a->wc == b->wc;
}

static uint8_t pair_kind_bit(uint8_t a, uint8_t b)
{
    int has_r = (a == OR_) || (b == OR_);
    int has_w = (a == OW_) || (b == OW_);
    int has_a = (a == OA_) || (b == OA_);
    if (has_w && !has_r && !has_a) return 1u << 1;  /* W-W */
    if (has_w && has_r) return 1u << 0;             /* R-W */
    if (has_w && has_a) return 1u << 2;             /* A-W */
    return 1u << 3;                                 /* A-R */
}

/* ------------------------------------------------------- clock validation */

/* Returns 0 when the trace is well formed; else 1 unsorted, 2 clock mismatch,
 * 3 partial-mask __syncwarp, 4 unknown op.  *bad gets the record index. */
int hro_validate(const hro_rec* r, uint64_t n, uint64_t* bad)
{
    uint32_t max_tid = 0;
    for (uint64_t i = 0; i < n; i++)
        if (r[i].tid > max_tid) max_tid = r[i].tid;
    uint64_t nt = (uint64_t)max_tid + 1;
    uint16_t* kern = (uint16_t*)malloc(nt * sizeof(uint16_t));
    uint16_t* bc = (uint16_t*)malloc(nt * sizeof(uint16_t));
    uint16_t* wc = (uint16_t*)malloc(nt * sizeof(uint16_t));
    uint8_t* seen = (uint8_t*)calloc(nt, 1);
    int rc = 0;
    for (uint64_t i = 0; i < n && rc == 0; i++) {
        const hro_rec* x = &r[i];
        if (i > 0 && wave_of(x) < wave_of(&r[i - 1])) { rc = 1; *bad = i; break; }
        if (x->op > OSW_) { rc = 4; *bad = i; break; }
        uint32_t t = x->tid;
        if (!seen[t] || x->kernel != kern[t]) {  /* a new launch: clocks restart */
            seen[t] = 1;
            kern[t] = x->kernel;
            bc[t] = 0;
            wc[t] = 0;
        }
        if (x->op == OST_) {
            bc[t] = (uint16_t)(bc[t] + 1);
            wc[t] = 0;
        } else if (x->op == OSW_) {
            if (x->flags & PARTIAL_MASK_FLAG) { rc = 3; *bad = i; break; }
            wc[t] = (uint16_t)(wc[t] + 1);
        }
        if (x->bc != bc[t] || x->wc != wc[t]) { rc = 2; *bad = i; break; }
    }
    free(kern); free(bc); free(wc); free(seen);
    return rc;
}

/* ------------------------------------------------ brute force (definition) */

/* stable LSD radix sort of (key, idx) pairs on the low `bits` bits of key */
static void radix_sort(uint64_t* key, uint64_t* idx, uint64_t m, int bits)
{
    uint64_t* k2 = (uint64_t*)malloc(m * sizeof(uint64_t));
    uint64_t* i2 = (uint64_t*)malloc(m * sizeof(uint64_t));
    uint64_t* cnt = (uint64_t*)malloc(65536 * sizeof(uint64_t));
    for (int shift = 0; shift < bits; shift += 16) {
        memset(cnt, 0, 65536 * sizeof(uint64_t));
        for (uint64_t i = 0; i < m; i++) cnt[(key[i] >> shift) & 0xFFFF]++;
        uint64_t s = 0;
        for (int d = 0; d < 65536; d++) { uint64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (uint64_t i = 0; i < m; i++) {
            uint64_t d = (key[i] >> shift) & 0xFFFF;
            k2[cnt[d]] = key[i];
            i2[cnt[d]] = idx[i];
            cnt[d]++;
        }
        memcpy(key, k2, m * sizeof(uint64_t));
        memcpy(idx, i2, m * sizeof(uint64_t));
    }
    free(k2); free(i2); free(cnt);
}

/* pairwise: every pair of accesses of one (kernel, word) group */
static int group_pairwise(const hro_rec* r, const uint64_t* g, uint64_t m, uint32_t bd, uint32_t ws,
                          hro_race* out)
{
    uint64_t best_wave = UINT64_MAX;
    for (uint64_t i = 0; i < m; i++)
        for (uint64_t j = i + 1; j < m; j++) {
            const hro_rec* a = &r[g[i]];
            const hro_rec* b = &r[g[j]];
            if (a->tid == b->tid || !conflicting(a->op, b->op) || !concurrent(a, b, bd, ws)) continue;
            uint64_t later = wave_of(b);  /* g is in trace (= wave) order, so b is not earlier */
            if (later < best_wave) best_wave = later;
        }
    if (best_wave == UINT64_MAX) return 0;
    uint16_t estar = (uint16_t)((best_wave >> 16) & 0xFFFF);
    uint8_t ops = 0, kinds = 0;
    for (uint64_t i = 0; i < m; i++)
        for (uint64_t j = i + 1; j < m; j++) {
            const hro_rec* a = &r[g[i]];
            const hro_rec* b = &r[g[j]];
            if (a->tid == b->tid || !conflicting(a->op, b->op) || !concurrent(a, b, bd, ws)) continue;
            uint16_t e = a->bc > b->bc ? a->bc : b->bc;
            if (e == estar) kinds |= pair_kind_bit(a->op, b->op);
            if (wave_of(b) == best_wave) {
                ops |= (uint8_t)(1u << b->op);
                if (wave_of(a) == best_wave) ops |= (uint8_t)(1u << a->op);
            }
        }
    out->word = r[g[0]].word;
    out->kernel = r[g[0]].kernel;
    out->epoch = estar;
    out->ops_mask = ops;
    out->kinds_mask = kinds;
    out->method = 0;
    return 1;
}

/* open-addressing map: 64-bit key -> three counters (one per op kind) */
typedef struct {
    uint64_t* keys;
    int32_t* cnt;
    uint64_t cap;
} hmap;

static void hm_init(hmap* h, uint64_t n)
{
    uint64_t cap = 16;
    while (cap < 2 * n + 16) cap <<= 1;
    h->cap = cap;
    h->keys = (uint64_t*)malloc(cap * sizeof(uint64_t));
    memset(h->keys, 0xFF, cap * sizeof(uint64_t));
    h->cnt = (int32_t*)calloc(cap * 3, sizeof(int32_t));
}

static void hm_free(hmap* h) { free(h->keys); free(h->cnt); }

static int32_t* hm_get(hmap* h, uint64_t key)
{
    uint64_t x = key * 0x9E3779B97F4A7C15ull;
    uint64_t i = (x ^ (x >> 29)) & (h->cap - 1);
    while (h->keys[i] != key && h->keys[i] != UINT64_MAX) i = (i + 1) & (h->cap - 1);
    h->keys[i] = key;
    return &h->cnt[3 * i];
}

/* The same definition as group_pairwise, counted instead of enumerated.
 * Accesses enter the counts one whole wave at a time; after a wave has been
 * added, an access x of that wave has a racy partner in an earlier-or-same
 * wave iff, for some op c conflicting with op_x, one of these counts of
 * c-accesses is positive:
 *   other blocks                         total[c]           - block[b_x][c]
 *   same block, same bc, other warp      blockbc[b_x,bc][c] - warpbc[w_x,bc][c]
 *   same warp, same bc and wc, other tid warpwave[w_x,bc,wc][c] - tidwave[t_x,bc,wc][c]
 */
static int group_counts(const hro_rec* r, const uint64_t* g, uint64_t m, uint32_t bd, uint32_t ws,
                        hro_race* out)
{
    hmap mb, mbbc, mwbc, mww, mtw;
    hm_init(&mb, m); hm_init(&mbbc, m); hm_init(&mwbc, m); hm_init(&mww, m); hm_init(&mtw, m);
    int32_t total[3] = {0, 0, 0};
    uint32_t wpb = (bd + ws - 1) / ws;
    int found = 0;
    uint64_t s = 0;
    while (s < m && !found) {
        uint64_t e = s;
        uint64_t wv = wave_of(&r[g[s]]);
        while (e < m && wave_of(&r[g[e]]) == wv) e++;
        for (uint64_t q = s; q < e; q++) {
            const hro_rec* x = &r[g[q]];
            uint64_t blk = x->tid / bd;
            uint64_t gw = blk * wpb + (x->tid % bd) / ws;
            total[x->op]++;
            hm_get(&mb, blk)[x->op]++;
            hm_get(&mbbc, (blk << 16) | x->bc)[x->op]++;
            hm_get(&mwbc, (gw << 16) | x->bc)[x->op]++;
            hm_get(&mww, (gw << 32) | ((uint64_t)x->bc << 16) | x->wc)[x->op]++;
            hm_get(&mtw, ((uint64_t)x->tid << 32) | ((uint64_t)x->bc << 16) | x->wc)[x->op]++;
        }
        uint8_t ops = 0;
        for (uint64_t q = s; q < e; q++) {
            const hro_rec* x = &r[g[q]];
            uint64_t blk = x->tid / bd;
            uint64_t gw = blk * wpb + (x->tid % bd) / ws;
            int32_t* cb = hm_get(&mb, blk);
            int32_t* cbbc = hm_get(&mbbc, (blk << 16) | x->bc);
            int32_t* cwbc = hm_get(&mwbc, (gw << 16) | x->bc);
            int32_t* cww = hm_get(&mww, (gw << 32) | ((uint64_t)x->bc << 16) | x->wc);
            int32_t* ctw = hm_get(&mtw, ((uint64_t)x->tid << 32) | ((uint64_t)x->bc << 16) | x->wc);
            for (uint8_t c = 0; c < 3; c++) {
                if (!conflicting(c, x->op)) continue;
                if (total[c] - cb[c] > 0 || cbbc[c] - cwbc[c] > 0 || cww[c] - ctw[c] > 0) {
                    ops |= (uint8_t)(1u << x->op);
                    break;
                }
            }
        }
        if (ops) {
            out->word = r[g[s]].word;
            out->kernel = r[g[s]].kernel;
            out->epoch = (uint16_t)((wv >> 16) & 0xFFFF);
            out->ops_mask = ops;
            out->kinds_mask = 0xFF;
            out->method = 1;
            found = 1;
        }
        s = e;
    }
    hm_free(&mb); hm_free(&mbbc); hm_free(&mwbc); hm_free(&mww); hm_free(&mtw);
    return found;
}

/* All racy (kernel, word) groups of a validated trace, sorted by (kernel, word).
 * Groups larger than pair_limit use the count form.  Returns the number of
 * racy groups (may exceed cap; only cap are written). */
int64_t hro_bruteforce(const hro_rec* r, uint64_t n, uint32_t block_dim, uint32_t warp_size,
                       uint64_t pair_limit, hro_race* out, uint64_t cap)
{
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; i++) m += is_access(r[i].op);
    uint64_t* key = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    uint64_t* idx = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    uint64_t j = 0;
    for (uint64_t i = 0; i < n; i++)
        if (is_access(r[i].op)) {
            key[j] = ((uint64_t)r[i].kernel << 32) | r[i].word;
            idx[j] = i;
            j++;
        }
    radix_sort(key, idx, m, 48);
    int64_t nr = 0;
    uint64_t s = 0;
    while (s < m) {
        uint64_t e = s + 1;
        while (e < m && key[e] == key[s]) e++;
        hro_race rr;
        memset(&rr, 0, sizeof rr);
        int racy = (e - s <= pair_limit) ? group_pairwise(r, idx + s, e - s, block_dim, warp_size, &rr)
                                         : group_counts(r, idx + s, e - s, block_dim, warp_size, &rr);
        if (racy) {
            if ((uint64_t)nr < cap) out[nr] = rr;
            nr++;
        }
        s = e;
    }
    free(key); free(idx);
    return nr;
}

/* The brute force restricted to words in [lo, hi): the same groups and forms,
 * so the union over disjoint ranges is hro_bruteforce's result (used to run the
 * definition on several host cores, one range per thread). */
int64_t hro_bruteforce_range(const hro_rec* r, uint64_t n, uint32_t block_dim, uint32_t warp_size,
                             uint64_t pair_limit, uint64_t lo, uint64_t hi, hro_race* out, uint64_t cap)
{
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; i++) m += is_access(r[i].op) && r[i].word >= lo && r[i].word < hi;
    uint64_t* key = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    uint64_t* idx = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    uint64_t j = 0;
    for (uint64_t i = 0; i < n; i++)
        if (is_access(r[i].op) && r[i].word >= lo && r[i].word < hi) {
            key[j] = ((uint64_t)r[i].kernel << 32) | r[i].word;
            idx[j] = i;
            j++;
        }
    radix_sort(key, idx, m, 48);
    int64_t nr = 0;
    uint64_t s = 0;
    while (s < m) {
        uint64_t e = s + 1;
        while (e < m && key[e] == key[s]) e++;
        hro_race rr;
        memset(&rr, 0, sizeof rr);
        int racy = (e - s <= pair_limit) ? group_pairwise(r, idx + s, e - s, block_dim, warp_size, &rr)
                                         : group_counts(r, idx + s, e - s, block_dim, warp_size, &rr);
        if (racy) {
            if ((uint64_t)nr < cap) out[nr] = rr;
            nr++;
        }
        s = e;
    }
    free(key); free(idx);
    return nr;
}

/* --------------------------------------- every racy epoch (report mode 1) */

/* Rows for one (kernel, word) group: one per distinct epoch e = max(bc_a, bc_b)
 * over its racy pairs (a, b).  ops_mask of a row: the ops of the accesses that
 * complete such a pair (the later one of the pair in wave order, and both when
 * they share a wave).  `ops` is a zeroed scratch of 65536 entries, zeroed again
 * on return. */
static int64_t emit_epochs(const hro_rec* r0, uint8_t* ops, uint8_t* form_of, uint8_t form, hro_race* out,
                           uint64_t cap, int64_t nr)
{
    for (uint32_t e = 0; e < 65536; e++) {
        if (!ops[e]) continue;
        if ((uint64_t)nr < cap) {
            hro_race* o = &out[nr];
            memset(o, 0, sizeof *o);
            o->word = r0->word;
            o->kernel = r0->kernel;
            o->epoch = (uint16_t)e;
            o->ops_mask = ops[e];
            o->kinds_mask = 0xFF;
            o->method = form;
        }
        nr++;
        ops[e] = 0;
    }
    (void)form_of;
    return nr;
}

static void epochs_pairwise(const hro_rec* r, const uint64_t* g, uint64_t m, uint32_t bd, uint32_t ws,
                            uint8_t* ops)
{
    for (uint64_t i = 0; i < m; i++)
        for (uint64_t j = i + 1; j < m; j++) {
            const hro_rec* a = &r[g[i]];
            const hro_rec* b = &r[g[j]];  /* g is in wave order: b is not earlier than a */
            if (a->tid == b->tid || !conflicting(a->op, b->op) || !concurrent(a, b, bd, ws)) continue;
            uint16_t e = a->bc > b->bc ? a->bc : b->bc;
            ops[e] |= (uint8_t)(1u << b->op);
            if (wave_of(a) == wave_of(b)) ops[e] |= (uint8_t)(1u << a->op);
        }
}

/* The count form of epochs_pairwise: every wave, not only up to the first racy one. */
static void epochs_counts(const hro_rec* r, const uint64_t* g, uint64_t m, uint32_t bd, uint32_t ws,
                          uint8_t* ops)
{
    hmap mb, mbbc, mwbc, mww, mtw;
    hm_init(&mb, m); hm_init(&mbbc, m); hm_init(&mwbc, m); hm_init(&mww, m); hm_init(&mtw, m);
    int32_t total[3] = {0, 0, 0};
    uint32_t wpb = (bd + ws - 1) / ws;
    uint64_t s = 0;
    while (s < m) {
        uint64_t e = s;
        uint64_t wv = wave_of(&r[g[s]]);
        while (e < m && wave_of(&r[g[e]]) == wv) e++;
        for (uint64_t q = s; q < e; q++) {
            const hro_rec* x = &r[g[q]];
            uint64_t blk = x->tid / bd;
            uint64_t gw = blk * wpb + (x->tid % bd) / ws;
            total[x->op]++;
            hm_get(&mb, blk)[x->op]++;
            hm_get(&mbbc, (blk << 16) | x->bc)[x->op]++;
            hm_get(&mwbc, (gw << 16) | x->bc)[x->op]++;
            hm_get(&mww, (gw << 32) | ((uint64_t)x->bc << 16) | x->wc)[x->op]++;
            hm_get(&mtw, ((uint64_t)x->tid << 32) | ((uint64_t)x->bc << 16) | x->wc)[x->op]++;
        }
        for (uint64_t q = s; q < e; q++) {
            const hro_rec* x = &r[g[q]];
            uint64_t blk = x->tid / bd;
            uint64_t gw = blk * wpb + (x->tid % bd) / ws;
            int32_t* cb = hm_get(&mb, blk);
            int32_t* cbbc = hm_get(&mbbc, (blk << 16) | x->bc);
            int32_t* cwbc = hm_get(&mwbc, (gw << 16) | x->bc);
            int32_t* cww = hm_get(&mww, (gw << 32) | ((uint64_t)x->bc << 16) | x->wc);
            int32_t* ctw = hm_get(&mtw, ((uint64_t)x->tid << 32) | ((uint64_t)x->bc << 16) | x->wc);
            for (uint8_t c = 0; c < 3; c++) {
                if (!conflicting(c, x->op)) continue;
                if (total[c] - cb[c] > 0 || cbbc[c] - cwbc[c] > 0 || cww[c] - ctw[c] > 0) {
                    ops[x->bc] |= (uint8_t)(1u << x->op);
                    break;
                }
            }
        }
        s = e;
    }
    hm_free(&mb); hm_free(&mbbc); hm_free(&mwbc); hm_free(&mww); hm_free(&mtw);
}

/* Every racy (kernel, word, epoch) of a validated trace, sorted by (kernel,
 * word, epoch): the report set when RACE is not absorbing.  Groups larger
 * than pair_limit use the count form.  Returns the row count (may exceed
 * cap; only cap rows are written). */
int64_t hro_bruteforce_epochs(const hro_rec* r, uint64_t n, uint32_t block_dim, uint32_t warp_size,
                              uint64_t pair_limit, hro_race* out, uint64_t cap)
{
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; i++) m += is_access(r[i].op);
    uint64_t* key = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    uint64_t* idx = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    uint8_t* ops = (uint8_t*)calloc(65536, 1);
    uint64_t j = 0;
    for (uint64_t i = 0; i < n; i++)
        if (is_access(r[i].op)) {
            key[j] = ((uint64_t)r[i].kernel << 32) | r[i].word;
            idx[j] = i;
            j++;
        }
    radix_sort(key, idx, m, 48);
    int64_t nr = 0;
    uint64_t s = 0;
    while (s < m) {
        uint64_t e = s + 1;
        while (e < m && key[e] == key[s]) e++;
        const int counts = e - s > pair_limit;
        if (counts)
            epochs_counts(r, idx + s, e - s, block_dim, warp_size, ops);
        else
            epochs_pairwise(r, idx + s, e - s, block_dim, warp_size, ops);
        nr = emit_epochs(&r[idx[s]], ops, NULL, (uint8_t)counts, out, cap, nr);
        s = e;
    }
    free(key); free(idx); free(ops);
    return nr;
}

/* Force one group through a chosen form (for cross-checking the two forms). */
int hro_group_check(const hro_rec* r, const uint64_t* g, uint64_t m, uint32_t block_dim,
                    uint32_t warp_size, int use_counts, hro_race* out)
{
    memset(out, 0, sizeof *out);
    return use_counts ? group_counts(r, g, m, block_dim, warp_size, out)
                      : group_pairwise(r, g, m, block_dim, warp_size, out);
}

/* ------------------------------------------------------------- serial FSM */

/* Constant-size summary of the accesses a word has seen in the current kernel. */
typedef struct {
    uint32_t block;      /* the only block that accessed the word (nblocks == 1) */
    uint32_t gwarp;      /* the only warp in the current block epoch (nwarps == 1) */
    uint32_t tid;        /* the only thread in the current warp sub-epoch (nthreads == 1) */
    uint16_t kernel;
    uint16_t epoch;      /* E: block clock of the latest access of that block */
    uint16_t sub;        /* F: warp clock of the latest access of that warp */
    uint8_t valid;       /* 0: no access yet in `kernel` (INIT) */
    uint8_t raced;       /* RACE reached: absorbing for the rest of the kernel */
    uint8_t nblocks, nwarps, nthreads;  /* 1, or 2 meaning "two or more" */
    uint8_t k_all;       /* op kinds over the whole kernel   (bit 1<<op) */
    uint8_t k_epoch;     /* op kinds in epoch E              (bit 1<<op) */
    uint8_t k_sub;       /* op kinds in sub-epoch (E, F)     (bit 1<<op) */
} hro_word;

/* does a new access of kind `op` conflict with some access whose kind is in `set`? */
static int conflicts_with(uint8_t set, uint8_t op)
{
    for (uint8_t c = 0; c < 3; c++)
        if ((set >> c) & 1u)
            if (conflicting(c, op)) return 1;
    return 0;
}

enum {
    NM_INIT = 0, NM_READ, NM_WRITE, NM_ATOMIC, NM_WREAD, NM_WATOMIC, NM_BREAD, NM_BATOMIC,
    NM_GREAD, NM_GATOMIC, NM_RACE
};

static uint8_t name_of(const hro_word* s)
{
    const uint8_t R = 1u << OR_, A = 1u << OA_;
    if (!s->valid) return NM_INIT;
    if (s->raced) return NM_RACE;
    if (s->nblocks >= 2) return s->k_all == R ? NM_GREAD : NM_GATOMIC;
    if (s->nwarps >= 2) return s->k_epoch == R ? NM_BREAD : NM_BATOMIC;
    if (s->nthreads >= 2) return s->k_sub == R ? NM_WREAD : NM_WATOMIC;
    if (s->k_sub == R) return NM_READ;
    if (s->k_sub == A) return NM_ATOMIC;
    return NM_WRITE;
}

/* Apply one access to a word summary (Algorithm 1: read the shadow, compare
 * thread ids, compare clocks, take the transition, write back).  Returns 1 when
 * this access moves the word into RACE. */
static int fsm_apply(hro_word* s, const hro_rec* x, uint32_t bd, uint32_t ws)
{
    if (s->valid && s->kernel != x->kernel) s->valid = 0;   /* kernel end ordered everything */
    if (!s->valid) {
        memset(s, 0, sizeof *s);
        s->kernel = x->kernel;
    }
    if (s->raced) return 0;
    uint32_t wpb = (bd + ws - 1) / ws;
    uint32_t blk = x->tid / bd;
    uint32_t gw = blk * wpb + (x->tid % bd) / ws;
    uint8_t bit = (uint8_t)(1u << x->op);

    /* does x race with the summarised history? */
    int race;
    if (!s->valid) race = 0;                                     /* first access */
    else if (s->nblocks >= 2 || blk != s->block) race = conflicts_with(s->k_all, x->op);
    else if (x->bc != s->epoch) race = 0;                        /* a barrier separates */
    else if (s->nwarps >= 2 || gw != s->gwarp) race = conflicts_with(s->k_epoch, x->op);
    else if (x->wc != s->sub) race = 0;                          /* a warp barrier separates */
    else if (s->nthreads >= 2 || x->tid != s->tid) race = conflicts_with(s->k_sub, x->op);
    else race = 0;                                               /* same thread */
    if (race) {
        s->raced = 1;
        return 1;
    }

    /* fold x into the summary */
    if (!s->valid) {
        s->valid = 1;
        s->nblocks = 1; s->block = blk;
        s->nwarps = 1; s->gwarp = gw; s->epoch = x->bc;
        s->nthreads = 1; s->tid = x->tid; s->sub = x->wc;
        s->k_all = s->k_epoch = s->k_sub = bit;
    } else if (s->nblocks >= 2 || blk != s->block) {
        s->nblocks = 2;
        s->k_all |= bit;
    } else if (x->bc != s->epoch) {
        s->epoch = x->bc;
        s->nwarps = 1; s->gwarp = gw;
        s->nthreads = 1; s->tid = x->tid; s->sub = x->wc;
        s->k_epoch = s->k_sub = bit;
        s->k_all |= bit;
    } else if (s->nwarps >= 2 || gw != s->gwarp) {
        s->nwarps = 2;
        s->k_epoch |= bit;
        s->k_all |= bit;
    } else if (x->wc != s->sub) {
        s->sub = x->wc;
        s->nthreads = 1; s->tid = x->tid;
        s->k_sub = bit;
        s->k_epoch |= bit;
        s->k_all |= bit;
    } else {
        if (x->tid != s->tid) s->nthreads = 2;
        s->k_sub |= bit;
        s->k_epoch |= bit;
        s->k_all |= bit;
    }
    return 0;
}

/* Serial FSM over a validated trace, in trace order.  Reports are written in
 * the order the words enter RACE.  Returns the report count (may exceed cap),
 * or -1 when a word index is out of range.  If names != NULL, names[i] gets
 * the named state of record i's word after record i (0 for sync records). */
int64_t hro_serial_fsm(const hro_rec* r, uint64_t n, uint32_t block_dim, uint32_t warp_size,
                       uint64_t n_words, hro_report* out, uint64_t cap, uint8_t* names)
{
    hro_word* sh = (hro_word*)calloc(n_words ? n_words : 1, sizeof(hro_word));
    if (!sh) return -2;
    int64_t nr = 0;
    for (uint64_t i = 0; i < n; i++) {
        const hro_rec* x = &r[i];
        if (!is_access(x->op)) {
            if (names) names[i] = 0;
            continue;
        }
        if (x->word >= n_words) { free(sh); return -1; }
        hro_word* s = &sh[x->word];
        if (fsm_apply(s, x, block_dim, warp_size)) {
            if ((uint64_t)nr < cap) {
                out[nr].word = x->word;
                out[nr].tid = x->tid;
                out[nr].kernel = x->kernel;
                out[nr].epoch = x->bc;
                out[nr].op = x->op;
            }
            nr++;
        }
        if (names) names[i] = name_of(s);
    }
    free(sh);
    return nr;
}

/* The serial FSM restricted to the words in [lo, hi): the same per-word
 * processing in trace order, so the union of the reports of disjoint ranges
 * is the report set of hro_serial_fsm (used to run the oracle on several
 * host cores, one range per thread).  Returns the report count or -1/-2. */
uint64_t hro_word_bytes(void) { return sizeof(hro_word); }

/* `sh` is the caller's zeroed array of hi - lo word summaries (so that one
 * allocation, faulted in once, serves every range). */
int64_t hro_serial_fsm_range(const hro_rec* r, uint64_t n, uint32_t block_dim, uint32_t warp_size,
                             uint64_t lo, uint64_t hi, uint64_t n_words, hro_word* sh, hro_report* out,
                             uint64_t cap)
{
    if (hi > n_words) hi = n_words;
    if (lo > hi) lo = hi;
    if (!sh) return -2;
    int64_t nr = 0;
    for (uint64_t i = 0; i < n; i++) {
        const hro_rec* x = &r[i];
        if (!is_access(x->op)) continue;
        if (x->word >= n_words) return -1;
        if (x->word < lo || x->word >= hi) continue;
        if (fsm_apply(&sh[x->word - lo], x, block_dim, warp_size)) {
            if ((uint64_t)nr < cap) {
                out[nr].word = x->word;
                out[nr].tid = x->tid;
                out[nr].kernel = x->kernel;
                out[nr].epoch = x->bc;
                out[nr].op = x->op;
            }
            nr++;
        }
    }
    return nr;
}

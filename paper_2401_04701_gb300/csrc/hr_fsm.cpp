// hr_fsm.cpp - builds the flat FSM transition table (host side).
//
// Sec. III: instead of the set of threads that touched a word, the FSM keeps
// the narrowest level of the thread hierarchy (thread, warp, block, grid) that
// contains all of the word's accessors, plus the last accessor; Sec. IV-B: the FSM is a flat array indexed by the old state and
// the transition labels (access, thread relation, sync status).  The paper's
// own 25-state machine is not published (its Figs. 1 and 4 are absent), so
// the states are derived here from what the race definition (Sec. II-A) and
// the GPU happens-before model (Sec. II-B) need to remember about a word's
// race-free history so far, given that accesses arrive in an order consistent
// with happens-before:
//
//   INIT            no access in this kernel
//   GRID(c)         two or more blocks; every access has kind c
//   BLOCK(a, c)     one block; its latest block epoch (bc) spans >= 2 warps,
//                   all of kind c; a = kinds over the whole kernel
//   WARP(a, e, c)   one block, one warp in the latest epoch (kinds e), its
//                   latest warp sub-epoch (wc) spans >= 2 threads of kind c
//   THREAD(a, e, s) one block, one warp in the latest epoch (kinds e), one
//                   thread in the latest sub-epoch (kinds s)
//   RACE            a racy pair was seen (absorbing until the kernel ends)
//
// A kind set is kept only as far as conflicts can tell it apart: bit 0 "holds
// a read or a write" (conflicts with a later atomic), bit 1 "holds an atomic
// or a write" (conflicts with a later read); a write sets both bits, and so
// does a read next to an atomic.  The last accessor's tid, bc and wc (stored
// beside the state) name the block, warp, thread, epoch and sub-epoch above.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hirace.h"
#include "../../include/hirace_device.cuh"

namespace {

enum Level { L_INIT = 0, L_THREAD = 1, L_WARP = 2, L_BLOCK = 3, L_GRID = 4, L_RACE = 5 };
enum Op { OP_R = 0, OP_W = 1, OP_A = 2 };
enum TRel { T_SAME = 0, T_WARP = 1, T_BLOCK = 2, T_GRID = 3 };
enum SRel { S_UNSYNC = 0, S_WARP = 1, S_BLOCK = 2 };

struct Abs {
    int level, all, epoch, last;  // last: sub-epoch kinds (THREAD) / pure kind (WARP, BLOCK, GRID)
    bool operator<(const Abs& o) const
    {
        return std::tie(level, all, epoch, last) < std::tie(o.level, o.all, o.epoch, o.last);
    }
    bool operator==(const Abs& o) const
    {
        return level == o.level && all == o.all && epoch == o.epoch && last == o.last;
    }
};

static_assert(L_THREAD == HR_LVL_THREAD && L_WARP == HR_LVL_WARP && L_BLOCK == HR_LVL_BLOCK &&
                  L_GRID == HR_LVL_GRID && L_RACE == HR_LVL_RACE,
              "level codes must match the device header");
static_assert(T_GRID == HR_TREL_GRID && T_BLOCK == HR_TREL_BLOCK && S_BLOCK == HR_SREL_BLOCK &&
                  S_WARP == HR_SREL_WARP,
              "label codes must match the device header");
const int HR_STATE_RACE_ID = (int)HR_STATE_RACE;

const Abs kInit{L_INIT, 0, 0, 0};
const Abs kRace{L_RACE, 0, 0, 0};

int kind_bits(int op) { return op == OP_R ? 1 : op == OP_A ? 2 : 3; }
// a later access `op` races with an unordered earlier one whose kinds are `k`
bool conflicts(int k, int op) { return (k & (op == OP_R ? 2 : op == OP_A ? 1 : 3)) != 0; }

Abs transition(const Abs& s, int op, int trel, int srel)
{
    const int k = kind_bits(op);
    if (s.level == L_INIT) return Abs{L_THREAD, k, k, k};
    if (s.level == L_RACE) return s;
    if (s.level == L_GRID) return conflicts(s.last, op) ? kRace : s;
    // one block so far
    if (trel == T_GRID)  // blocks are never ordered inside a kernel
        return conflicts(s.all, op) ? kRace : Abs{L_GRID, 0, 0, k};
    if (srel == S_BLOCK)  // a __syncthreads separates x from the whole history
        return Abs{L_THREAD, s.all | k, k, k};
    if (s.level == L_BLOCK)  // >= 2 warps in x's epoch: one of them is another warp
        return conflicts(s.last, op) ? kRace : s;
    if (trel == T_BLOCK)  // another warp of the block, same epoch
        return conflicts(s.epoch, op) ? kRace : Abs{L_BLOCK, s.all, 0, k};
    if (srel == S_WARP)  // same warp, a __syncwarp separates x from the epoch's history
        return Abs{L_THREAD, s.all | k, s.epoch | k, k};
    if (s.level == L_WARP)  // >= 2 threads in x's sub-epoch: one of them is another thread
        return conflicts(s.last, op) ? kRace : s;
    // THREAD level, same sub-epoch
    if (trel == T_SAME) return Abs{L_THREAD, s.all | k, s.epoch | k, s.last | k};
    return conflicts(s.last, op) ? kRace : Abs{L_WARP, s.all, s.epoch, k};
}

struct Machine {
    std::vector<Abs> states;  // index = state id
    std::vector<uint8_t> table;
};

const char* kind_name(int k) { return k == 1 ? "R" : k == 2 ? "A" : k == 3 ? "M" : "-"; }

std::string name_of(const Abs& s)
{
    char buf[48];
    switch (s.level) {
    case L_INIT: return "INIT";
    case L_RACE: return "RACE";
    case L_GRID: return s.last == 1 ? "GREAD" : "GATOMIC";
    case L_BLOCK: snprintf(buf, sizeof buf, "BLOCK[%s|%s]", kind_name(s.all), kind_name(s.last)); return buf;
    case L_WARP:
        snprintf(buf, sizeof buf, "WARP[%s|%s|%s]", kind_name(s.all), kind_name(s.epoch), kind_name(s.last));
        return buf;
    default:
        snprintf(buf, sizeof buf, "THREAD[%s|%s|%s]", kind_name(s.all), kind_name(s.epoch), kind_name(s.last));
        return buf;
    }
}

Machine build()
{
    Machine m;
    std::map<Abs, int> id;
    id[kInit] = 0;
    m.states.push_back(kInit);
    // breadth-first over every label; RACE is pinned to id 31
    for (size_t q = 0; q < m.states.size(); ++q) {
        const Abs s = m.states[q];
        for (int op = 0; op < 3; ++op)
            for (int trel = 0; trel < 4; ++trel)
                for (int srel = 0; srel < 3; ++srel) {
                    Abs t = transition(s, op, trel, srel);
                    if (t == kRace || id.count(t)) continue;
                    id[t] = (int)m.states.size();
                    m.states.push_back(t);
                }
    }
    const int n_live = (int)m.states.size();
    m.states.resize(32, kInit);
    m.states[HR_STATE_RACE_ID] = kRace;
    id[kRace] = HR_STATE_RACE_ID;
    m.table.assign(2048, 0xFF);
    for (int s = 0; s < 32; ++s) {
        if (s >= n_live && s != HR_STATE_RACE_ID) continue;
        for (int op = 0; op < 3; ++op)
            for (int trel = 0; trel < 4; ++trel)
                for (int srel = 0; srel < 3; ++srel) {
                    const Abs t = transition(m.states[s], op, trel, srel);
                    const int tid = id.at(t);
                    m.table[(s << 6) | (op << 4) | (trel << 2) | srel] = (uint8_t)(tid | (t.level << 5));
                }
    }
    m.states.resize(n_live);
    m.states.push_back(kRace);
    return m;
}

const Machine& machine()
{
    static const Machine m = build();
    return m;
}

}  // namespace

extern "C" hr_status hr_fsm_table(uint8_t* out, uint32_t* n_states)
{
    if (!out) return HR_ERR_INVALID;
    const Machine& m = machine();
    memcpy(out, m.table.data(), 2048);
    if (n_states) *n_states = (uint32_t)m.states.size();
    return HR_OK;
}

extern "C" const char* hr_fsm_state_name(uint32_t state)
{
    static std::vector<std::string> names;
    static bool ready = false;
    if (!ready) {
        const Machine& m = machine();
        names.assign(32, "?");
        for (size_t i = 0; i + 1 < m.states.size(); ++i) names[i] = name_of(m.states[i]);
        names[HR_STATE_RACE_ID] = "RACE";
        ready = true;
    }
    return state < 32 ? names[state].c_str() : "?";
}

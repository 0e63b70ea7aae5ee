// Shared device-side definitions for librpd (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "prim.cuh"
#include "rpd.h"

#define RPD_MAXC 32          // candidate spheres per tet (one warp of lanes)
#define RPD_MAXK 32          // power neighbours per mesh vertex
#define RPD_GATHER 48        // candidate gather capacity before filtering
#define RPD_COORD_MAX ((1 << 21) - 1)

// Device status block: first error code plus counters.
enum {
    CNT_DEGENERATE = 0,   // exact predicate == 0
    CNT_OVERFLOW,         // candidate capacity exceeded
    CNT_LINK_MISSING,     // component link target absent (inconsistency)
    CNT_UF_LIMIT,         // union-find loop hit its iteration bound
    CNT_CAPACITY,         // polytope vertex capacity exceeded (cannot happen by bound)
    CNT_INVALID,          // invalid input value
    CNT_NONMANIFOLD,      // face shared by > 2 tets
    CNT_PRED_FAST,        // predicates decided by the cached filter
    CNT_PRED_FP64,        // decided by the FP64 re-evaluation
    CNT_PRED_EXACT,       // decided by exact integers
    CNT_CAND_FALLBACK,    // tets resolved by the grid-search fallback
    CNT_WHOLE,            // whole-tet pieces
    CNT_NEWVERT1,         // polytope vertices constructed by clipping, by the number
    CNT_NEWVERT2,         //   of radical planes through them (1, 2, 3)
    CNT_NEWVERT3,
    CNT_NUM
};

struct DevState {
    int err;                        // first rpd_status != OK raised on the device
    int pad;
    unsigned long long cnt[CNT_NUM];
};

__device__ __forceinline__ void dev_fail(DevState* st, int code, int counter) {
    atomicCAS(&st->err, 0, code);
    atomicAdd(&st->cnt[counter], 1ull);
}

// Warp-aggregated counter increment (any subset of lanes may call).
__device__ __forceinline__ void dev_count(DevState* st, int counter, unsigned v) {
    unsigned mask = __activemask();
    unsigned tot = __reduce_add_sync(mask, v);
    if ((int)(threadIdx.x & 31) == __ffs(mask) - 1 && tot) atomicAdd(&st->cnt[counter], (unsigned long long)tot);
}

// Exact power distance pd(x, m) = |x - c|^2 - w on the integer grid.
// |x|,|c| <= 2^21 so |x-c|^2 <= 3*2^44 and w <= 2^44: |pd| < 2^46.
__device__ __forceinline__ long long pd_exact(int3 x, int3 c, long long w) {
    int dx = x.x - c.x, dy = x.y - c.y, dz = x.z - c.z;   // |d| <= 2^22: 32-bit exact
    return (long long)dx * dx + (long long)dy * dy + (long long)dz * dz - w;
}

__device__ __forceinline__ int3 ld_int3(const int32_t* p, long long i) {
    return make_int3(p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}

// Local tet edge index of vertices (a, b): (0,1)(0,2)(0,3)(1,2)(1,3)(2,3).
__device__ __forceinline__ int tet_edge_index(int a, int b) {
    int lo = min(a, b), hi = max(a, b);
    return lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5);
}

static inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------ open-addressing hash sets
// 64-bit keys (~0 marks an empty slot and is never a valid key), linear
// probing, capacity a power of two with mask = capacity - 1 and shift = 64 -
// log2(capacity).  Keys are only ever inserted, so a slot once set never
// changes; a stale empty read is settled by the compare-and-swap.
constexpr uint64_t HEMPTY = ~0ull;

__device__ __forceinline__ unsigned long long hslot(uint64_t key, int shift) {
    return (key * 0x9E3779B97F4A7C15ull) >> shift;
}

// Slot holding `key` (inserted if absent), or -1 if the table is full.
__device__ __forceinline__ long long table_insert(uint64_t* tk, unsigned long long mask, int shift, uint64_t key) {
    unsigned long long h = hslot(key, shift);
    for (unsigned long long it = 0; it <= mask; it++) {
        const uint64_t k = tk[h];
        if (k == key) return (long long)h;
        if (k == HEMPTY) {
            const uint64_t old = atomicCAS((unsigned long long*)&tk[h], HEMPTY, key);
            if (old == HEMPTY || old == key) return (long long)h;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// Slot holding `key`, or -1.
__device__ __forceinline__ long long table_find(const uint64_t* tk, unsigned long long mask, int shift, uint64_t key) {
    unsigned long long h = hslot(key, shift);
    for (unsigned long long it = 0; it <= mask; it++) {
        const uint64_t k = tk[h];
        if (k == key) return (long long)h;
        if (k == HEMPTY) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

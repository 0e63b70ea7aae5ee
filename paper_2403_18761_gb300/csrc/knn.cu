// A1-A2: grid-bucketed k-nearest power neighbours and per-tet candidates.
//
// Sec. 4.1.2 clips each (tet, sphere) piece by the radical half-spaces of the
// sphere's power neighbours; Sec. 5.2 leaves the tet-sphere relation and the
// neighbour search to supplementary material.  This file implements them:
//
//  * For every mesh vertex x: the K spheres of smallest power distance
//    pd(x, m) = |x - c|^2 - r^2 (exact 64-bit integers on the grid), found by
//    a ring search over a uniform grid of sphere centres, and D+(x), a lower
//    bound on pd(x, m) for every sphere m NOT in the list.  The ring search
//    stops once (distance to the next ring)^2 - max r^2 exceeds the K-th
//    distance; that bound is the completeness ("security") test.
//
//  * For a tet t with corners X_a: if sphere i owns part of t, then for every
//    sphere j some corner has pd(X_a, i) <= pd(X_a, j) (pd(.,i) - pd(.,j) is
//    affine, so its minimum over t is at a corner).  With j = o_b, the owner
//    of corner b, every such i lies in {m in list(X_a) : pd(X_a, m) <=
//    pd(X_a, o_b)} for some a, provided each list is complete up to that
//    threshold (D+(X_a) > pd(X_a, o_b)).  The gathered set is then filtered
//    exactly with the same corner test against every other gathered sphere.
//    When no corner b gives complete lists, a grid search collects the same
//    set directly (fallback).
#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "internal.cuh"
#include "prim.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }
size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

__device__ __forceinline__ int floordiv(long long a, int b) {
    long long q = a / b;
    if ((a % b) != 0 && ((a < 0) != (b < 0))) q--;
    return (int)q;
}

__device__ __forceinline__ int3 cell_of(int3 x, const GridParams& g) {
    int cx = floordiv((long long)x.x - g.org.x, g.cell);
    int cy = floordiv((long long)x.y - g.org.y, g.cell);
    int cz = floordiv((long long)x.z - g.org.z, g.cell);
    return make_int3(min(max(cx, 0), g.dim.x - 1), min(max(cy, 0), g.dim.y - 1), min(max(cz, 0), g.dim.z - 1));
}

__device__ __forceinline__ long long axis_gap(int x, int org, int q, int cell) {
    long long lo = (long long)org + (long long)q * cell;
    long long hi = lo + cell - 1;
    if (x < lo) return lo - x;
    if (x > hi) return x - hi;
    return 0;
}

__device__ __forceinline__ long long box_dist2(int3 x, const GridParams& g, int qx, int qy, int qz) {
    long long dx = axis_gap(x.x, g.org.x, qx, g.cell);
    long long dy = axis_gap(x.y, g.org.y, qy, g.cell);
    long long dz = axis_gap(x.z, g.org.z, qz, g.cell);
    return dx * dx + dy * dy + dz * dz;
}

// Grid over the sphere centres' bounding box with about four spheres per cell
// and at most ncap cells.
__device__ GridParams grid_params(const int* mn, const int* mx, long long wm, long long ns, long long ncap) {
    long long ext[3];
    for (int a = 0; a < 3; a++) ext[a] = (long long)mx[a] - mn[a] + 1;
    double vol = (double)ext[0] * (double)ext[1] * (double)ext[2];
    // about four spheres per cell: the neighbour walk's cost is in its rows and
    // runs, so fewer, fuller cells pay (one, two, four, eight and sixteen per
    // cell measured on the organic blob: the search took 3.43, 3.12, 3.0,
    // 3.26 and 3.63 ms)
    double target = (double)(ns < 8 ? 1 : ns / 4);
    long long cell = (long long)ceil(cbrt(vol / target));
    if (cell < 1) cell = 1;
    long long d[3];
    for (int it = 0; it < 200; it++) {
        for (int a = 0; a < 3; a++) d[a] = (ext[a] - 1) / cell + 1;
        if (d[0] * d[1] * d[2] <= ncap) break;
        cell = cell + cell / 4 + 1;
    }
    GridParams g;
    g.org = make_int3(mn[0], mn[1], mn[2]);
    g.cell = (int)cell;
    g.dim = make_int3((int)d[0], (int)d[1], (int)d[2]);
    g.ncell = (int)(d[0] * d[1] * d[2]);
    g.wmax = wm;
    g.cbase = 0;
    g.sbase = 0;
    return g;
}

// Shape of vertex v in a batch: the s with voff[s] <= v < voff[s + 1]
// (0 without a batch).
__device__ __forceinline__ int shape_of(const long long* __restrict__ voff, int nshapes, long long v) {
    if (!voff || nshapes <= 1) return 0;
    int lo = 0, hi = nshapes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (voff[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Bounding box of the sphere centres and the largest weight, reduced over
// the block; thread 0 returns the grid parameters in *out (shared memory).
__device__ void block_grid_params(const int32_t* __restrict__ Ci, const long long* __restrict__ W, long long ns,
                                  long long ncap, GridParams* out, long long cut = LLONG_MAX) {
    __shared__ int smin[3][32], smax[3][32];
    __shared__ long long swm[32];
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    long long wm = 0;
    for (long long i = threadIdx.x; i < ns; i += blockDim.x) {
        if (W[i] > cut) continue;   // a heavy sphere: kept out of the grid
        for (int a = 0; a < 3; a++) {
            int v = Ci[3 * i + a];
            mn[a] = min(mn[a], v);
            mx[a] = max(mx[a], v);
        }
        wm = max(wm, W[i]);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int a = 0; a < 3; a++) {
        mn[a] = __reduce_min_sync(0xffffffffu, mn[a]);
        mx[a] = __reduce_max_sync(0xffffffffu, mx[a]);
    }
    for (int off = 16; off; off >>= 1) wm = max(wm, __shfl_xor_sync(0xffffffffu, wm, off));
    if (lane == 0) {
        for (int a = 0; a < 3; a++) { smin[a][w] = mn[a]; smax[a][w] = mx[a]; }
        swm[w] = wm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        for (int q = 1; q < nw; q++) {
            for (int a = 0; a < 3; a++) { mn[a] = min(mn[a], smin[a][q]); mx[a] = max(mx[a], smax[a][q]); }
            wm = max(wm, swm[q]);
        }
        *out = grid_params(mn, mx, wm, ns, ncap);
    }
}

__global__ void k_bbox(const int32_t* __restrict__ Ci, const long long* __restrict__ W, long long ns, long long ncap,
                       GridParams* gp, const long long* __restrict__ wcut) {
    __shared__ GridParams sg;
    block_grid_params(Ci, W, ns, ncap, &sg, wcut ? *wcut : LLONG_MAX);
    if (threadIdx.x == 0) *gp = sg;
}

// The whole sphere grid in one block, for up to GRID_SMALL_CAP cells: the
// grid parameters, per-cell counts in shared memory, their exclusive scan
// (cell_start) and the fill, with no launches in between.
constexpr int GRID_SMALL_CAP = 11264;   // counts within 44 KB of shared memory
constexpr int HEAVY_MAX = 128;          // heavy spheres kept out of the grid at most

__device__ __forceinline__ int block_excl_scan(int v, int* total) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;   // inclusive prefix of the warp totals
    }
    __syncthreads();
    *total = wsum[nw - 1];
    return incl - v + (w > 0 ? wsum[w - 1] : 0);
}

__global__ void __launch_bounds__(1024) k_grid_small(const int32_t* __restrict__ Ci, const long long* __restrict__ W,
                                                     long long ns, long long ncap, GridParams* gp,
                                                     int64_t* __restrict__ start, int32_t* __restrict__ ids,
                                                     int4* __restrict__ sph, long long* __restrict__ sw,
                                                     long long* __restrict__ cwmax, long long* __restrict__ rwmax,
                                                     const long long* __restrict__ wcut) {
    extern __shared__ int scount[];
    __shared__ GridParams sg;
    const long long cut = wcut ? *wcut : LLONG_MAX;
    block_grid_params(Ci, W, ns, ncap, &sg, cut);
    for (long long q = threadIdx.x; q < ncap; q += blockDim.x) {
        scount[q] = 0;
        cwmax[q] = 0;
        rwmax[q] = 0;
    }
    __syncthreads();
    const GridParams g = sg;
    if (threadIdx.x == 0) *gp = g;
    for (long long i = threadIdx.x; i < ns; i += blockDim.x) {
        if (W[i] > cut) continue;
        const int3 c = cell_of(ld_int3(Ci, i), g);
        const int q = (c.z * g.dim.y + c.y) * g.dim.x + c.x;
        atomicAdd(&scount[q], 1);
        atomicMax((unsigned long long*)&cwmax[q], (unsigned long long)W[i]);
        atomicMax((unsigned long long*)&rwmax[c.z * g.dim.y + c.y], (unsigned long long)W[i]);
    }
    __syncthreads();
    const int per = (int)((ncap + blockDim.x - 1) / blockDim.x);
    const int lo = min((long long)threadIdx.x * per, ncap), hi = min((long long)lo + per, ncap);
    int sum = 0;
    for (int q = lo; q < hi; q++) sum += scount[q];
    int total;
    int run = block_excl_scan(sum, &total);
    for (int q = lo; q < hi; q++) {
        const int n = scount[q];
        start[q] = run;
        scount[q] = run;   // becomes the fill cursor
        run += n;
    }
    if (threadIdx.x == 0) start[ncap] = total;
    __syncthreads();
    for (long long i = threadIdx.x; i < ns; i += blockDim.x) {
        if (W[i] > cut) continue;
        const int3 ci = ld_int3(Ci, i);
        const int3 c = cell_of(ci, g);
        const int q = (c.z * g.dim.y + c.y) * g.dim.x + c.x;
        const int pos = atomicAdd(&scount[q], 1);
        ids[pos] = (int32_t)i;
        sph[pos] = make_int4(ci.x, ci.y, ci.z, (int)i);
        sw[pos] = W[i];
    }
}

// Heavy spheres: the up to H largest power weights.  The neighbour walk stops
// once the next shell's distance minus the largest weight of the grid exceeds
// the K-th distance, so a few heavy spheres would keep every vertex walking;
// they are kept out of the grid and every vertex evaluates them first.  One
// block: the (H + 1)-th largest weight t by an 8-bit radix select from the
// top byte down (weights are >= 0), then the spheres with W > t (at most H)
// in id order by a chunked block scan.
__global__ void __launch_bounds__(1024) k_heavy_select(const int32_t* __restrict__ Ci,
                                                       const long long* __restrict__ W, long long ns, int H,
                                                       long long* __restrict__ wcut, int4* __restrict__ hsph,
                                                       long long* __restrict__ hw, int* __restrict__ nheavy) {
    __shared__ int hist[256];
    __shared__ unsigned long long sprefix;
    __shared__ long long sneed;
    if (threadIdx.x == 0) {
        sprefix = 0;
        sneed = H + 1;
    }
    for (int pos = 7; pos >= 0; pos--) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const unsigned long long prefix = sprefix;
        const unsigned long long hmask = pos == 7 ? 0ull : (~0ull << (8 * (pos + 1)));
        for (long long i = threadIdx.x; i < ns; i += blockDim.x) {
            const unsigned long long v = (unsigned long long)W[i];
            if ((v & hmask) == prefix) atomicAdd(&hist[(v >> (8 * pos)) & 0xff], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long need = sneed, cum = 0;
            int b = 255;
            for (; b > 0; b--) {
                if (cum + hist[b] >= need) break;
                cum += hist[b];
            }
            sneed = need - cum;
            sprefix = prefix | ((unsigned long long)b << (8 * pos));
        }
        __syncthreads();
    }
    const long long t = (long long)sprefix;
    int base = 0;
    for (long long c0 = 0; c0 < ns; c0 += blockDim.x) {
        const long long i = c0 + threadIdx.x;
        const int f = i < ns && W[i] > t;
        int total;
        const int at = base + block_excl_scan(f, &total);
        if (f && at < H) {
            hsph[at] = make_int4(Ci[3 * i], Ci[3 * i + 1], Ci[3 * i + 2], (int)i);
            hw[at] = W[i];
        }
        base += total;
        __syncthreads();   // block_excl_scan's shared words are reused
    }
    if (threadIdx.x == 0) {
        *wcut = t;
        *nheavy = min(base, H);
    }
}

// One grid per shape of a batch, a block per shape: as k_grid_small on the
// shape's spheres, with cell offsets relative to the shape's cell base and
// sorted slots at the shape's sphere offset.
__global__ void __launch_bounds__(1024) k_grid_batch(const int32_t* __restrict__ Ci, const long long* __restrict__ W,
                                                     const long long* __restrict__ soff, long long ncap_total,
                                                     GridParams* gp, int64_t* __restrict__ start_all,
                                                     int32_t* __restrict__ ids, int4* __restrict__ sph,
                                                     long long* __restrict__ sw, long long* __restrict__ cwmax_all) {
    extern __shared__ int scount[];
    __shared__ GridParams sg;
    const int sh = blockIdx.x;
    const long long s0 = soff[sh], ns = soff[sh + 1] - s0;
    const long long ncap = 2 * ns + 64, cbase = 2 * s0 + 65ll * sh;
    int64_t* start = start_all + cbase;
    long long* cwmax = cwmax_all + cbase;
    long long* rwmax = cwmax_all + ncap_total + cbase;
    block_grid_params(Ci + 3 * s0, W + s0, ns, ncap, &sg);
    for (long long q = threadIdx.x; q < ncap; q += blockDim.x) {
        scount[q] = 0;
        cwmax[q] = 0;
        rwmax[q] = 0;
    }
    __syncthreads();
    GridParams g = sg;
    g.cbase = cbase;
    g.sbase = s0;
    if (threadIdx.x == 0) gp[sh] = g;
    for (long long i = threadIdx.x; i < ns; i += blockDim.x) {
        const int3 c = cell_of(ld_int3(Ci, s0 + i), g);
        const int q = (c.z * g.dim.y + c.y) * g.dim.x + c.x;
        atomicAdd(&scount[q], 1);
        atomicMax((unsigned long long*)&cwmax[q], (unsigned long long)W[s0 + i]);
        atomicMax((unsigned long long*)&rwmax[c.z * g.dim.y + c.y], (unsigned long long)W[s0 + i]);
    }
    __syncthreads();
    const int per = (int)((ncap + blockDim.x - 1) / blockDim.x);
    const int lo = min((long long)threadIdx.x * per, ncap), hi = min((long long)lo + per, ncap);
    int sum = 0;
    for (int q = lo; q < hi; q++) sum += scount[q];
    int total;
    int run = block_excl_scan(sum, &total);
    for (int q = lo; q < hi; q++) {
        const int n = scount[q];
        start[q] = s0 + run;
        scount[q] = run;
        run += n;
    }
    if (threadIdx.x == 0) start[ncap] = s0 + total;
    __syncthreads();
    for (long long i = threadIdx.x; i < ns; i += blockDim.x) {
        const long long gi = s0 + i;
        const int3 ci = ld_int3(Ci, gi);
        const int3 c = cell_of(ci, g);
        const int q = (c.z * g.dim.y + c.y) * g.dim.x + c.x;
        const long long pos = s0 + atomicAdd(&scount[q], 1);
        ids[pos] = (int32_t)gi;
        sph[pos] = make_int4(ci.x, ci.y, ci.z, (int)i);   // shape-local id: 17 bits of the kNN key suffice
        sw[pos] = W[gi];
    }
}

__global__ void k_cell_count(const int32_t* __restrict__ Ci, const long long* __restrict__ W, long long ns,
                             const GridParams* __restrict__ gp, int32_t* __restrict__ count,
                             long long* __restrict__ cwmax, long long* __restrict__ rwmax,
                             const long long* __restrict__ wcut) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns || (wcut && W[i] > *wcut)) return;
    GridParams g = *gp;
    int3 c = cell_of(ld_int3(Ci, i), g);
    int q = (c.z * g.dim.y + c.y) * g.dim.x + c.x;
    atomicAdd(&count[q], 1);
    atomicMax((unsigned long long*)&cwmax[q], (unsigned long long)W[i]);
    atomicMax((unsigned long long*)&rwmax[c.z * g.dim.y + c.y], (unsigned long long)W[i]);
}

// Cell-sorted copy of the spheres: ids, (centre, id) and weight per slot.
__global__ void k_cell_fill(const int32_t* __restrict__ Ci, const long long* __restrict__ W, long long ns,
                            const GridParams* __restrict__ gp, const int64_t* __restrict__ start,
                            int32_t* __restrict__ fill, int32_t* __restrict__ ids, int4* __restrict__ sph,
                            long long* __restrict__ sw, const long long* __restrict__ wcut) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns || (wcut && W[i] > *wcut)) return;
    GridParams g = *gp;
    int3 c = ld_int3(Ci, i);
    int3 cc = cell_of(c, g);
    int q = (cc.z * g.dim.y + cc.y) * g.dim.x + cc.x;
    int slot = atomicAdd(&fill[q], 1);
    long long pos = start[q] + slot;
    ids[pos] = (int32_t)i;
    sph[pos] = make_int4(c.x, c.y, c.z, (int)i);
    sw[pos] = W[i];
}

// ---------------------------------------------------------------- kNN
// Tiled form (any number of spheres; with up to 2^17 the warp form below is
// used unless a test asks for this one): eight mesh vertices per warp, four lanes per vertex.  Vertices
// are processed in the order of their sphere-grid cell (a stable sort by cell
// index), so the vertices of a warp lie in a few neighbouring cells.  The
// warp walks box shells around the bounding box of its vertices' cells; each
// row run of the cell-sorted spheres is loaded 32 at a time (coalesced), and
// sphere j of a chunk goes to lane j mod 4 of every vertex group, so each
// lane sees a quarter of the stream.  Each lane keeps the K best (distance,
// id) pairs of its quarter in a binary max-heap in shared memory.  A sphere
// farther than the root of a full heap of its group cannot be among the K
// best and is rejected.  Per chunk, every lane first marks the spheres that
// survive this test; the marked spheres are then inserted in rounds in which
// all lanes that still hold one insert together (one heap update each, log2 K
// levels).  Once a lane's or its group's bound proves that no unexplored
// sphere can enter, the group is done; at the end the four heaps of a vertex
// are sorted and merged.  Everything rejected, evicted, left out of the
// merge or left unexplored lowers D+.  The walk stops once the distance to
// the next shell minus max r^2 exceeds the group's K-th distance bound.

__device__ __forceinline__ bool pair_less(long long d1, int i1, long long d2, int i2) {
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

// Lower bound of |x - y|^2 over cells outside the box [lo, hi] (cell
// indices); LLONG_MAX when the box covers the whole grid.
__device__ __forceinline__ long long outside_box_lb2(int3 x, const GridParams& g, int3 lo, int3 hi) {
    long long best = LLONG_MAX;
    const int xs[3] = {x.x, x.y, x.z}, ls[3] = {lo.x, lo.y, lo.z}, hs[3] = {hi.x, hi.y, hi.z},
              ds[3] = {g.dim.x, g.dim.y, g.dim.z}, os[3] = {g.org.x, g.org.y, g.org.z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (hs[a] + 1 <= ds[a] - 1) {
            long long start = (long long)os[a] + (long long)(hs[a] + 1) * g.cell;
            best = min(best, max(0LL, start - xs[a]));
        }
        if (ls[a] - 1 >= 0) {
            long long end = (long long)os[a] + (long long)ls[a] * g.cell - 1;
            best = min(best, max(0LL, (long long)xs[a] - end));
        }
    }
    return best == LLONG_MAX ? LLONG_MAX : best * best;
}

// Heap entries, ordered by (power distance, sphere id), the distance and the
// id kept apart (any number of spheres).
struct PairEntry {
    struct E {
        long long d;
        int i;
    };
    static __device__ __forceinline__ E make(long long d, int id) { return {d, id}; }
    static __device__ __forceinline__ long long dist(E e) { return e.d; }
    static __device__ __forceinline__ int sid(E e) { return e.i; }
    static __device__ __forceinline__ bool less(E a, E b) { return pair_less(a.d, a.i, b.d, b.i); }
    static __device__ __forceinline__ E empty() { return {LLONG_MAX, INT_MAX}; }
    template <int KMAX>
    struct Storage {
        long long d[4][KMAX][32];
        int i[4][KMAX][32];
    };
    template <int KMAX>
    struct Heap {
        long long (*d)[32];
        int (*i)[32];
        __device__ __forceinline__ Heap(Storage<KMAX>& s, int warp) : d(s.d[warp]), i(s.i[warp]) {}
        __device__ __forceinline__ E get(int p, int l) const { return {d[p][l], i[p][l]}; }
        __device__ __forceinline__ void set(int p, int l, E e) const {
            d[p][l] = e.d;
            i[p][l] = e.i;
        }
    };
};

// Sift e down from the root of a max-heap of size m held in column `lane`.
template <typename P, typename H>
__device__ __forceinline__ void heap_sift_down(const H& h, int lane, int m, typename P::E e) {
    int p = 0;
    while (true) {
        int ch = 2 * p + 1;
        if (ch >= m) break;
        typename P::E c = h.get(ch, lane);
        if (ch + 1 < m) {
            const typename P::E c2 = h.get(ch + 1, lane);
            if (P::less(c, c2)) {
                ch++;
                c = c2;
            }
        }
        if (!P::less(e, c)) break;
        h.set(p, lane, c);
        p = ch;
    }
    h.set(p, lane, e);
}

template <int KMAX, typename P>
__global__ void __launch_bounds__(128) k_knn_group(const int32_t* __restrict__ Xi, const uint32_t* __restrict__ vorder,
                                                    long long nv, const GridParams* __restrict__ gp,
                                                    const int64_t* __restrict__ start, const int4* __restrict__ sph,
                                                    const long long* __restrict__ sw, int K,
                                                    int32_t* __restrict__ knn, long long* __restrict__ dplus,
                                                    const int* __restrict__ err) {
    typedef typename P::E E;
    // the vertex order comes from a sort whose bounded wait may have run out
    // and left entries unwritten: then compute nothing (the build fails)
    if (*(volatile const int*)err != 0) return;
    const unsigned FULL = 0xffffffffu;
    __shared__ typename P::template Storage<KMAX> store;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane & 3;   // quarter of the stream this lane sees
    const typename P::template Heap<KMAX> heap(store, warp);
    const long long wbase = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 8;
    if (wbase >= nv) return;   // warp-uniform
    const long long idx = wbase + (lane >> 2);
    const bool valid = idx < nv;
    const long long v = vorder[valid ? idx : wbase];
    const GridParams g = *gp;
    const int3 x = ld_int3(Xi, v);
    const int3 c = cell_of(x, g);
    int3 lo, hi3;
    lo.x = __reduce_min_sync(FULL, c.x);
    lo.y = __reduce_min_sync(FULL, c.y);
    lo.z = __reduce_min_sync(FULL, c.z);
    hi3.x = __reduce_max_sync(FULL, c.x);
    hi3.y = __reduce_max_sync(FULL, c.y);
    hi3.z = __reduce_max_sync(FULL, c.z);
    int cnt = 0;                 // size of this lane's heap
    E kr = P::empty();           // its root once full
    long long gmin = LLONG_MAX;  // smallest full-heap root distance in the group
    long long dp = LLONG_MAX;
    bool done = !valid;
    int3 plo = make_int3(1, 1, 1), phi = make_int3(0, 0, 0);   // processed box (empty)
    for (int r = 0; r < (1 << 22); r++) {
        const int3 blo = make_int3(max(lo.x - r, 0), max(lo.y - r, 0), max(lo.z - r, 0));
        const int3 bhi =
            make_int3(min(hi3.x + r, g.dim.x - 1), min(hi3.y + r, g.dim.y - 1), min(hi3.z + r, g.dim.z - 1));
        // rows (y, z) of the new shell, one per lane: the whole row outside
        // the processed box's (y, z) range, else the parts left and right of
        // it; their spheres are concatenated and processed 32 at a time
        const int ny = bhi.y - blo.y + 1, nrow = ny * (bhi.z - blo.z + 1);
        for (int rb = 0; rb < nrow; rb += 32) {
            long long a0 = 0, b0 = 0;
            int na = 0, nbb = 0;
            if (rb + lane < nrow) {
                const int yy = blo.y + (rb + lane) % ny, zz = blo.z + (rb + lane) / ny;
                const int qrow = (zz * g.dim.y + yy) * g.dim.x;
                const bool inner = zz >= plo.z && zz <= phi.z && yy >= plo.y && yy <= phi.y;
                if (inner) {
                    a0 = start[qrow + blo.x];
                    na = (int)(start[qrow + plo.x] - a0);
                    b0 = start[qrow + phi.x + 1];
                    nbb = (int)(start[qrow + bhi.x + 1] - b0);
                } else {
                    a0 = start[qrow + blo.x];
                    na = (int)(start[qrow + bhi.x + 1] - a0);
                }
            }
            const int m = na + nbb;
            int incl = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const int ntot = __shfl_sync(FULL, incl, 31);
            for (int pb = 0; pb < ntot; pb += 32) {
                const int item = pb + lane;
                int j = 0;   // first lane whose inclusive count exceeds item
#pragma unroll
                for (int step = 16; step; step >>= 1) {
                    const int probe = __shfl_sync(FULL, incl, j + step - 1);
                    if (probe <= item) j += step;
                }
                j = min(j, 31);
                const int oj = item - __shfl_sync(FULL, incl - m, j);
                const int naj = __shfl_sync(FULL, na, j);
                const long long a0j = __shfl_sync(FULL, a0, j), b0j = __shfl_sync(FULL, b0, j);
                int4 cs = make_int4(0, 0, 0, 0);
                long long ws = 0;
                if (item < ntot) {
                    const long long e = oj < naj ? a0j + oj : b0j + (oj - naj);
                    cs = sph[e];
                    ws = sw[e];
                }
                const int nb = min(32, ntot - pb);
                // pass 1: spheres sub, sub + 4, ... of the chunk that may enter
                unsigned mark = 0;
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    const int jj = 4 * t + sub;
                    const int3 cj = make_int3(__shfl_sync(FULL, cs.x, jj), __shfl_sync(FULL, cs.y, jj),
                                              __shfl_sync(FULL, cs.z, jj));
                    const int idj = __shfl_sync(FULL, cs.w, jj);
                    const long long wj = __shfl_sync(FULL, ws, jj);
                    if (done || jj >= nb) continue;
                    const long long d = pd_exact(x, cj, wj);
                    if (d <= gmin && (cnt < K || P::less(P::make(d, idj), kr))) mark |= 1u << t;
                    else dp = min(dp, d);
                }
                // pass 2: insert the marked spheres, one per lane per round
                while (__any_sync(FULL, mark != 0)) {
                    const bool has = mark != 0;
                    const int jj = has ? 4 * (__ffs(mark) - 1) + sub : 0;
                    mark &= mark - 1;
                    const int3 cj = make_int3(__shfl_sync(FULL, cs.x, jj), __shfl_sync(FULL, cs.y, jj),
                                              __shfl_sync(FULL, cs.z, jj));
                    const int id = __shfl_sync(FULL, cs.w, jj);
                    const long long wj = __shfl_sync(FULL, ws, jj);
                    if (!has) continue;
                    const long long d = pd_exact(x, cj, wj);
                    const E e = P::make(d, id);
                    if (cnt < K) {   // push and sift up
                        int p = cnt++;
                        while (p > 0) {
                            const int q = (p - 1) >> 1;
                            const E qe = heap.get(q, lane);
                            if (!P::less(qe, e)) break;
                            heap.set(p, lane, qe);
                            p = q;
                        }
                        heap.set(p, lane, e);
                        if (cnt == K) kr = heap.get(0, lane);
                    } else if (P::less(e, kr)) {   // replace the root
                        dp = min(dp, P::dist(kr));
                        heap_sift_down<P>(heap, lane, K, e);
                        kr = heap.get(0, lane);
                    } else {
                        dp = min(dp, d);
                    }
                }
                // group bound: smallest root among the group's full heaps
                long long gr = cnt == K ? P::dist(kr) : LLONG_MAX;
                gr = min(gr, __shfl_xor_sync(FULL, gr, 1));
                gr = min(gr, __shfl_xor_sync(FULL, gr, 2));
                gmin = min(gmin, gr);
            }
        }
        plo = blo;
        phi = bhi;
        const long long lb2 = outside_box_lb2(x, g, blo, bhi);
        if (!done) {   // uniform over the group: same x and gmin
            if (lb2 == LLONG_MAX) {
                done = true;
            } else if (gmin != LLONG_MAX && lb2 - g.wmax > gmin) {
                dp = min(dp, lb2 - g.wmax);
                done = true;
            }
        }
        if (__all_sync(FULL, done)) break;
    }
    if (valid) {   // whatever was not explored is bounded by the last box
        const long long lbu = outside_box_lb2(x, g, plo, phi);
        if (lbu != LLONG_MAX) dp = min(dp, lbu - g.wmax);
    }
    // heap sort each lane's column into ascending order
    for (int n = cnt; n > 1; n--) {
        const E r = heap.get(0, lane);
        heap_sift_down<P>(heap, lane, n - 1, heap.get(n - 1, lane));
        heap.set(n - 1, lane, r);
    }
    __syncwarp();
    // merge the four sorted columns of each vertex: the K smallest go to the
    // list, the smallest left out bounds D+
    const int n0 = __shfl_sync(FULL, cnt, lane & ~3), n1 = __shfl_sync(FULL, cnt, (lane & ~3) + 1),
              n2 = __shfl_sync(FULL, cnt, (lane & ~3) + 2), n3 = __shfl_sync(FULL, cnt, (lane & ~3) + 3);
    long long dmin = dp;
    if (valid && sub == 0) {
        int p0 = 0, p1 = 0, p2 = 0, p3 = 0;
        const int l0 = lane;
        for (int j = 0; j < K; j++) {
            E be = P::empty();
            int bc = -1;
            if (p0 < n0 && P::less(heap.get(p0, l0), be)) { be = heap.get(p0, l0); bc = 0; }
            if (p1 < n1 && P::less(heap.get(p1, l0 + 1), be)) { be = heap.get(p1, l0 + 1); bc = 1; }
            if (p2 < n2 && P::less(heap.get(p2, l0 + 2), be)) { be = heap.get(p2, l0 + 2); bc = 2; }
            if (p3 < n3 && P::less(heap.get(p3, l0 + 3), be)) { be = heap.get(p3, l0 + 3); bc = 3; }
            knn[v * K + j] = bc < 0 ? -1 : P::sid(be);
            p0 += bc == 0;
            p1 += bc == 1;
            p2 += bc == 2;
            p3 += bc == 3;
        }
        if (p0 < n0) dmin = min(dmin, P::dist(heap.get(p0, l0)));
        if (p1 < n1) dmin = min(dmin, P::dist(heap.get(p1, l0 + 1)));
        if (p2 < n2) dmin = min(dmin, P::dist(heap.get(p2, l0 + 2)));
        if (p3 < n3) dmin = min(dmin, P::dist(heap.get(p3, l0 + 3)));
    }
    dmin = min(dmin, __shfl_xor_sync(FULL, dmin, 1));
    dmin = min(dmin, __shfl_xor_sync(FULL, dmin, 2));
    if (valid && sub == 0) dplus[v] = dmin;
}

// Warp form, for up to 2^17 spheres: one mesh vertex per warp.  A list
// entry is one 64-bit key, (pd + 2^46) << 17 | id (|pd| < 2^46), whose
// integer order is the (power distance, id) order.  The warp keeps the K
// smallest keys seen so far sorted across its lanes (lane j holds the j-th,
// lanes >= K hold nothing), walks box shells around the vertex's grid cell
// and evaluates the spheres of each shell 32 at a time, one per lane.  A
// chunk key enters only if it is below the K-th key; when a few enter they
// are inserted one by one (a ballot finds the position, a shuffle shifts the
// tail), when many enter the chunk is sorted by a bitonic network and merged
// with the list (the elementwise minimum of the list and the reversed chunk
// holds the 32 smallest of both as a bitonic sequence).  Everything rejected,
// pushed out or left unexplored lowers D+.  The walk stops as in the tiled
// form: once the distance to the next shell minus max r^2 exceeds the K-th
// distance.
__device__ __forceinline__ unsigned long long knn_key(long long d, int id) {
    return ((unsigned long long)(d + (1ll << 46)) << 17) | (unsigned)id;
}
__device__ __forceinline__ long long knn_key_dist(unsigned long long e) { return (long long)(e >> 17) - (1ll << 46); }

// One chunk of 32 keys (one per lane, EMPTY for none) into the warp's sorted
// list of the K smallest keys L (lane j holds the j-th): keys below the K-th
// enter one by one (ballot + shuffle) when few, else by a bitonic sort of the
// chunk merged with the list; every key rejected or pushed out lowers dp.
__device__ __forceinline__ void knn_insert(unsigned long long key, unsigned long long& L, long long& dp, int K,
                                           int lane) {
    typedef unsigned long long U;
    const unsigned FULL = 0xffffffffu;
    const U EMPTY = ~0ull;
    const U tau = __shfl_sync(FULL, L, K - 1);
    const bool pass = key < tau;
    if (!pass && key != EMPTY) dp = min(dp, knn_key_dist(key));
    unsigned bal = __ballot_sync(FULL, pass);
    if (__popc(bal) <= 6) {
        while (bal) {   // one by one
            const int src = __ffs(bal) - 1;
            bal &= bal - 1;
            const U k = __shfl_sync(FULL, key, src);
            const int pos = __popc(__ballot_sync(FULL, L < k));
            if (pos >= K) {   // an earlier insertion raised the bar
                dp = min(dp, knn_key_dist(k));
                continue;
            }
            const U ev = __shfl_sync(FULL, L, K - 1);
            if (ev != EMPTY) dp = min(dp, knn_key_dist(ev));
            const U up = __shfl_up_sync(FULL, L, 1);
            if (lane > pos) L = up;
            if (lane == pos) L = k;
            if (lane >= K) L = EMPTY;
        }
    } else {   // bitonic sort of the entering keys, then merge
        U s = pass ? key : EMPTY;
#pragma unroll
        for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                const U o = __shfl_xor_sync(FULL, s, jj);
                const bool lower = (lane & jj) == 0, up = (lane & kk) == 0;
                s = (lower == up) ? min(s, o) : max(s, o);
            }
        }
        const U rv = __shfl_sync(FULL, s, 31 - lane);
        U lo = min(L, rv);
        const U hi = max(L, rv);
        if (hi != EMPTY) dp = min(dp, knn_key_dist(hi));
#pragma unroll
        for (int jj = 16; jj > 0; jj >>= 1) {
            const U o = __shfl_xor_sync(FULL, lo, jj);
            lo = (lane & jj) ? max(lo, o) : min(lo, o);
        }
        L = lo;
        if (lane >= K) {
            if (L != EMPTY) dp = min(dp, knn_key_dist(L));
            L = EMPTY;
        }
    }
}

template <bool HEAVY>
__global__ void __launch_bounds__(256, 4) k_knn_warp(const int32_t* __restrict__ Xi, const uint32_t* __restrict__ vorder,
                                                  long long nv, const GridParams* __restrict__ gp,
                                                  const int64_t* __restrict__ start_all, const int4* __restrict__ sph,
                                                  const long long* __restrict__ sw,
                                                  const long long* __restrict__ rwmax_all, int K,
                                                  int32_t* __restrict__ knn, long long* __restrict__ dplus,
                                                  const long long* __restrict__ voff, int nshapes,
                                                  const int4* __restrict__ hsph, const long long* __restrict__ hw,
                                                  const int* __restrict__ nheavy) {
    typedef unsigned long long U;
    const unsigned FULL = 0xffffffffu;
    const U EMPTY = ~0ull;
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nv) return;   // warp-uniform
    const long long v = vorder ? (long long)vorder[w] : w;
    const GridParams g = gp[shape_of(voff, nshapes, v)];   // the vertex's own shape's grid
    const int64_t* __restrict__ start = start_all + g.cbase;
    const long long* __restrict__ rwmax = rwmax_all + g.cbase;
    const int3 x = ld_int3(Xi, v);
    const int3 c = cell_of(x, g);
    U L = EMPTY;               // lane j: the j-th smallest key so far
    long long dp = LLONG_MAX;  // smallest distance known to be outside the list
    int3 plo = make_int3(1, 1, 1), phi = make_int3(0, 0, 0);   // processed box (empty)
    long long lb2 = LLONG_MAX;
    // the heavy spheres, kept out of the grid, first
    const int nh = HEAVY ? *nheavy : 0;
    for (int hb = 0; hb < nh; hb += 32) {
        U key = EMPTY;
        if (hb + lane < nh) {
            const int4 cs = hsph[hb + lane];
            key = knn_key(pd_exact(x, make_int3(cs.x, cs.y, cs.z), hw[hb + lane]), cs.w);
        }
        knn_insert(key, L, dp, K, lane);
    }
    for (int r = 0; r < (1 << 22); r++) {
        const int3 blo = make_int3(max(c.x - r, 0), max(c.y - r, 0), max(c.z - r, 0));
        const int3 bhi = make_int3(min(c.x + r, g.dim.x - 1), min(c.y + r, g.dim.y - 1), min(c.z + r, g.dim.z - 1));
        // rows (y, z) of the new shell, one per lane: the whole row outside
        // the processed box's (y, z) range, else the parts left and right of
        // it; their spheres are concatenated and evaluated 32 at a time
        const int ny = bhi.y - blo.y + 1, nrow = ny * (bhi.z - blo.z + 1);
        for (int rb = 0; rb < nrow; rb += 32) {
            long long a0 = 0, b0 = 0;
            int na = 0, nbb = 0;
            // a run whose lower bound |x - box|^2 - (max r^2 of its row)
            // exceeds the K-th distance cannot enter; the bound goes to D+
            const U tau = __shfl_sync(FULL, L, K - 1);
            const long long td = tau == EMPTY ? LLONG_MAX : knn_key_dist(tau);
            if (rb + lane < nrow) {
                const int yy = blo.y + (rb + lane) % ny, zz = blo.z + (rb + lane) / ny;
                const int qrow = (zz * g.dim.y + yy) * g.dim.x;
                const long long gy = axis_gap(x.y, g.org.y, yy, g.cell), gz = axis_gap(x.z, g.org.z, zz, g.cell);
                const long long base = gy * gy + gz * gz - rwmax[zz * g.dim.y + yy];
                // spheres of cells q0..q1 of the row, or 0 when the run is culled
                auto run = [&](int q0, int q1, long long first) -> int {
                    const int n = (int)(start[qrow + q1 + 1] - first);
                    if (n == 0) return 0;
                    const long long lo = (long long)g.org.x + (long long)q0 * g.cell;
                    const long long hi = (long long)g.org.x + (long long)(q1 + 1) * g.cell - 1;
                    const long long gx = x.x < lo ? lo - x.x : (x.x > hi ? x.x - hi : 0);
                    const long long lb = base + gx * gx;
                    if (lb <= td) return n;
                    dp = min(dp, lb);
                    return 0;
                };
                a0 = start[qrow + blo.x];
                if (zz >= plo.z && zz <= phi.z && yy >= plo.y && yy <= phi.y) {
                    if (blo.x < plo.x) na = run(blo.x, plo.x - 1, a0);
                    b0 = start[qrow + phi.x + 1];
                    if (phi.x < bhi.x) nbb = run(phi.x + 1, bhi.x, b0);
                } else {
                    na = run(blo.x, bhi.x, a0);
                }
            }
            const int m = na + nbb;
            int incl = m;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const int ntot = __shfl_sync(FULL, incl, 31);
            for (int pb = 0; pb < ntot; pb += 32) {
                const int item = pb + lane;
                int j = 0;   // first lane whose inclusive count exceeds item
#pragma unroll
                for (int step = 16; step; step >>= 1) {
                    const int probe = __shfl_sync(FULL, incl, j + step - 1);
                    if (probe <= item) j += step;
                }
                j = min(j, 31);
                const int oj = item - __shfl_sync(FULL, incl - m, j);
                const int naj = __shfl_sync(FULL, na, j);
                const long long a0j = __shfl_sync(FULL, a0, j), b0j = __shfl_sync(FULL, b0, j);
                U key = EMPTY;
                if (item < ntot) {
                    const long long e = oj < naj ? a0j + oj : b0j + (oj - naj);
                    const int4 cs = sph[e];
                    key = knn_key(pd_exact(x, make_int3(cs.x, cs.y, cs.z), sw[e]), cs.w);
                }
                knn_insert(key, L, dp, K, lane);
            }
        }
        plo = blo;
        phi = bhi;
        lb2 = outside_box_lb2(x, g, blo, bhi);   // uniform over the warp
        const U tau = __shfl_sync(FULL, L, K - 1);
        if (lb2 == LLONG_MAX || (tau != EMPTY && lb2 - g.wmax > knn_key_dist(tau))) break;
    }
    if (lb2 != LLONG_MAX) dp = min(dp, lb2 - g.wmax);   // whatever was not explored
#pragma unroll
    for (int o = 16; o; o >>= 1) dp = min(dp, __shfl_xor_sync(FULL, dp, o));
    if (lane < K) knn[v * K + lane] = L == EMPTY ? -1 : (int)(L & 0x1ffffu) + (int)g.sbase;
    if (lane == 0) dplus[v] = dp;
}

// Sort key of a vertex: the index of its sphere-grid cell.
__global__ void k_vertex_cells(const int32_t* __restrict__ Xi, long long nv, const GridParams* __restrict__ gp,
                               uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const GridParams g = *gp;
    const int3 c = cell_of(ld_int3(Xi, v), g);
    key[v] = (uint64_t)((c.z * g.dim.y + c.y) * g.dim.x + c.x);
    val[v] = (uint32_t)v;
}

// ---------------------------------------------------------- candidates
__device__ __forceinline__ bool load_tet(const int32_t* __restrict__ T, long long t, long long nv,
                                         const int32_t* __restrict__ Xi, int* v, int3* X) {
    for (int a = 0; a < 4; a++) {
        v[a] = T[4 * t + a];
        if (v[a] < 0 || v[a] >= nv) return false;
        X[a] = ld_int3(Xi, v[a]);
    }
    return true;
}

// One warp per tet: the gathered spheres live one per lane.
__global__ void __launch_bounds__(256, 5) k_candidates_warp(
    const int32_t* __restrict__ T, long long nt, long long nv, const int32_t* __restrict__ Xi,
    const int32_t* __restrict__ Ci, const long long* __restrict__ W, const int32_t* __restrict__ knn,
    const long long* __restrict__ dplus, int K, int32_t* __restrict__ cand_cnt, int32_t* __restrict__ cand,
    uint8_t* __restrict__ cand_ord, int32_t* __restrict__ fb_list, int32_t* __restrict__ fb_count, DevState* st) {
    const int lane = threadIdx.x & 31;
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= nt) return;   // warp-uniform
    int v[4];
    int3 X[4];
    // an earlier stage that raised an error (e.g. a neighbour-list sort whose
    // bounded wait ran out) may have left the lists unwritten: no candidates,
    // so nothing downstream reads them; the build reports the error
    if (*(volatile const int*)&st->err != 0 || !load_tet(T, t, nv, Xi, v, X)) {
        if (lane == 0) cand_cnt[t] = 0;
        return;
    }
    // Entries 0..7 of every corner's list (lanes 8a..8a+7), with their
    // centres and weights, are loaded first: entry 0 is the corner's owner,
    // so everything up to the gather needs only these and shuffles.
    const unsigned FULL = 0xffffffffu;
    const int a8 = lane >> 3, j8 = lane & 7;
    const int va = a8 == 0 ? v[0] : (a8 == 1 ? v[1] : (a8 == 2 ? v[2] : v[3]));
    const int3 xa8 = a8 == 0 ? X[0] : (a8 == 1 ? X[1] : (a8 == 2 ? X[2] : X[3]));
    const int s8 = j8 < K ? knn[(long long)va * K + j8] : -1;
    int3 c8 = make_int3(0, 0, 0);
    long long w8 = 0;
    if (s8 >= 0) {
        c8 = ld_int3(Ci, s8);
        w8 = W[s8];
    }
    const long long pd8 = s8 >= 0 ? pd_exact(xa8, c8, w8) : LLONG_MAX;
    long long dp[4];
#pragma unroll
    for (int a = 0; a < 4; a++) dp[a] = dplus[v[a]];
    // M(a, b) = pd(X_a, owner of corner b), one entry per lane 0..15.  Lane
    // (a, b) also holds whether corner a's list is complete up to M(a, b) and
    // M(a, b) - M(a, a); the lanes of one b then combine over a.
    long long Ml = 0;
    bool comp = true;
    long long score = 0;
    {
        const int a = (lane >> 2) & 3, b = lane & 3;
        const int3 cb = make_int3(__shfl_sync(FULL, c8.x, 8 * b), __shfl_sync(FULL, c8.y, 8 * b),
                                  __shfl_sync(FULL, c8.z, 8 * b));
        const long long wb = __shfl_sync(FULL, w8, 8 * b);
        const int3 xa = a == 0 ? X[0] : (a == 1 ? X[1] : (a == 2 ? X[2] : X[3]));
        const long long dpa = a == 0 ? dp[0] : (a == 1 ? dp[1] : (a == 2 ? dp[2] : dp[3]));
        if (lane < 16) Ml = pd_exact(xa, cb, wb);
        const long long maa = __shfl_sync(FULL, Ml, a * 5);
        comp = dpa > Ml;
        score = Ml - maa;
    }
    score = max(score, __shfl_xor_sync(FULL, score, 4));
    score = max(score, __shfl_xor_sync(FULL, score, 8));
    const unsigned cbits = __ballot_sync(FULL, comp);
    int bstar = -1;
    long long best = LLONG_MAX;
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const long long sb = __shfl_sync(FULL, score, b);
        if (((cbits >> b) & 0x1111u) == 0x1111u && sb < best) {
            best = sb;
            bstar = b;
        }
    }
    if (bstar < 0) {
        if (lane == 0) {
            fb_list[atomicAdd(fb_count, 1)] = (int32_t)t;
            cand_cnt[t] = 0;
        }
        return;
    }
    // Gather.  The lists ascend in power distance, so the entries within a
    // corner's threshold are a prefix: lanes 8a..8a+7 test entries 0..7 of
    // corner a's list at once; a corner whose 8th entry still passes goes on
    // through the rest of its list below.  Each sphere is kept once, with its
    // centre and weight.
    int sid = -1, nheld = 0;
    int3 hc = make_int3(0, 0, 0);
    long long hw = 0;
    unsigned more;
    {
        const long long thr = __shfl_sync(FULL, Ml, a8 * 4 + bstar);
        const bool in = s8 >= 0 && pd8 <= thr;
        const unsigned peers = __match_any_sync(FULL, in ? s8 : -1 - lane);
        const bool first = in && (__ffs(peers) - 1 == lane);
        const unsigned fm = __ballot_sync(FULL, first);
        nheld = __popc(fm);
        const int src = lane < nheld ? __fns(fm, 0, lane + 1) : 0;
        const int sn = __shfl_sync(FULL, s8, src);
        const int3 cn = make_int3(__shfl_sync(FULL, c8.x, src), __shfl_sync(FULL, c8.y, src),
                                  __shfl_sync(FULL, c8.z, src));
        const long long wn = __shfl_sync(FULL, w8, src);
        if (lane < nheld) {
            sid = sn;
            hc = cn;
            hw = wn;
        }
        more = __ballot_sync(FULL, in && j8 == 7);
    }
    for (; more; more &= more - 1) {
        const int a = (__ffs(more) - 1) >> 3;
        const long long thr = __shfl_sync(FULL, Ml, a * 4 + bstar);
        const int vb = a == 0 ? v[0] : (a == 1 ? v[1] : (a == 2 ? v[2] : v[3]));
        const int3 xa = a == 0 ? X[0] : (a == 1 ? X[1] : (a == 2 ? X[2] : X[3]));
        for (int base = 8; base < K; base += 32) {
            const int e = base + lane;
            const int s = e < K ? knn[(long long)vb * K + e] : -1;
            bool in = false;
            int3 cs = make_int3(0, 0, 0);
            long long ws = 0;
            if (s >= 0) {
                cs = ld_int3(Ci, s);
                ws = W[s];
                in = pd_exact(xa, cs, ws) <= thr;
            }
            for (int h = 0; h < nheld; h++)
                if (__shfl_sync(FULL, sid, h) == s) in = false;
            const unsigned mask = __ballot_sync(FULL, in);
            const int cnt = __popc(mask);
            if (nheld + cnt > 32) {
                if (lane == 0) {
                    fb_list[atomicAdd(fb_count, 1)] = (int32_t)t;
                    cand_cnt[t] = 0;
                }
                return;
            }
            const bool take = lane >= nheld && lane < nheld + cnt;
            const int src = take ? __fns(mask, 0, lane - nheld + 1) : 0;
            const int sn = __shfl_sync(FULL, s, src);
            const int3 cn = make_int3(__shfl_sync(FULL, cs.x, src), __shfl_sync(FULL, cs.y, src),
                                      __shfl_sync(FULL, cs.z, src));
            const long long wn = __shfl_sync(FULL, ws, src);
            if (take) {
                sid = sn;
                hc = cn;
                hw = wn;
            }
            nheld += cnt;
        }
    }
    const bool held = lane < nheld;
    long long D[4] = {0, 0, 0, 0};
    if (held) {
#pragma unroll
        for (int c = 0; c < 4; c++) D[c] = pd_exact(X[c], hc, hw);
    }
    // exact corner filter against every other gathered sphere; the corner
    // distances of the warp's spheres are read back from shared memory
    // (broadcast loads)
    struct alignas(32) D4 {
        long long x, y, z, w;
    };
    __shared__ D4 sD[8][32];
    __shared__ long long sKey[8][32];
    __shared__ int sSid[8][32];
    const int wib = threadIdx.x >> 5;
    const long long key = D[0] + D[1] + D[2] + D[3];
    sD[wib][lane] = D4{D[0], D[1], D[2], D[3]};
    sKey[wib][lane] = key;
    sSid[wib][lane] = sid;
    __syncwarp();
    bool ok = held;
    for (int j = 0; j < nheld; j++) {
        const D4 dj = sD[wib][j];
        const bool some = D[0] <= dj.x || D[1] <= dj.y || D[2] <= dj.z || D[3] <= dj.w;
        if (j != lane) ok = ok && some;
    }
    const unsigned kmask = __ballot_sync(0xffffffffu, ok);
    int rank = 0, rank2 = 0;
    for (unsigned m = kmask; m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        const int sj = sSid[wib][j];
        const long long kj = sKey[wib][j];
        rank += sj < sid;
        rank2 += (kj < key) || (kj == key && sj < sid);
    }
    if (ok) {
        cand[t * RPD_MAXC + rank] = sid;
        cand_ord[t * RPD_MAXC + rank2] = (uint8_t)rank;
    }
    if (lane == 0) cand_cnt[t] = __popc(kmask);
}

// Fallback for a tet whose corner lists are not complete enough: one block
// per tet collects every sphere m with pd(X_a, m) <= pd(X_a, o_b*) for some
// corner a (b* as in the warp form), then applies the same exact corner
// filter and orders.  The threads split all grid cells (each cell and each
// sphere seen once, so the list needs no duplicate check; cells pruned by
// their largest weight) and append through a shared counter.  A bounded scan
// replaces a ring search, whose stop test with the largest weight of all
// spheres can keep it going over most of the grid.
constexpr int FB_GATHER = 128;   // spheres gathered per tet at most
constexpr int FB_THREADS = 256;

__global__ void __launch_bounds__(FB_THREADS) k_candidates_fallback(
    const int32_t* __restrict__ T, long long nv, const int32_t* __restrict__ Xi, const int32_t* __restrict__ Ci,
    const long long* __restrict__ W, const int32_t* __restrict__ knn, int K, const GridParams* __restrict__ gp,
    const int64_t* __restrict__ start_all, const int32_t* __restrict__ ids, const long long* __restrict__ cwmax_all,
    const int32_t* __restrict__ fb_list, const int32_t* __restrict__ fb_count, int32_t* __restrict__ cand_cnt,
    int32_t* __restrict__ cand, uint8_t* __restrict__ cand_ord, DevState* st, const long long* __restrict__ voff,
    int nshapes, const int4* __restrict__ hsph, const long long* __restrict__ hw, const int* __restrict__ nheavy) {
    const unsigned FULL = 0xffffffffu;
    __shared__ int sid[FB_GATHER];
    __shared__ long long sD[FB_GATHER][4];
    __shared__ uint8_t skeep[FB_GATHER];
    __shared__ int sn;
    const int tid = threadIdx.x, lane = tid & 31;
    const long long nfb = *fb_count;
    const int nh = nheavy ? *nheavy : 0;
    for (long long q = blockIdx.x; q < nfb; q += gridDim.x) {
        const long long t = fb_list[q];   // uniform over the block
        int v[4];
        int3 X[4];
        if (!load_tet(T, t, nv, Xi, v, X)) {
            if (tid == 0) cand_cnt[t] = 0;
            continue;
        }
        // the grid of the tet's shape (its first corner's)
        const GridParams g = gp[shape_of(voff, nshapes, v[0])];
        const int64_t* __restrict__ start = start_all + g.cbase;
        const long long* __restrict__ cwmax = cwmax_all + g.cbase;

        int o[4];
        for (int a = 0; a < 4; a++) o[a] = knn[(long long)v[a] * K];
        long long M[4][4];
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 4; a++) M[a][b] = pd_exact(X[a], ld_int3(Ci, o[b]), W[o[b]]);
        int bstar = 0;
        long long best = LLONG_MAX;
        for (int b = 0; b < 4; b++) {
            long long score = 0;
            for (int a = 0; a < 4; a++) score = max(score, M[a][b] - M[a][a]);
            if (score < best) {
                best = score;
                bstar = b;
            }
        }
        long long thr[4];
        for (int a = 0; a < 4; a++) thr[a] = M[a][bstar];
        if (tid == 0) sn = 0;
        __syncthreads();
        // A sphere with pd(X_a) <= thr_a has its centre within
        // sqrt(thr_a + wmax) of X_a, so only the cells of the box around the
        // four corners' balls can hold one; each of those cells is opened
        // when some corner a may have a sphere of it within thr_a
        // (|X_a - cell|^2 - max r^2 of the cell <= thr_a).
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        for (int a = 0; a < 4; a++) {
            const long long r2 = thr[a] + g.wmax;
            const long long rad = r2 > 0 ? (long long)sqrt((double)r2) + 2 : 1;
            const long long xa[3] = {X[a].x, X[a].y, X[a].z};
            const int org[3] = {g.org.x, g.org.y, g.org.z}, dim[3] = {g.dim.x, g.dim.y, g.dim.z};
            for (int k = 0; k < 3; k++) {
                const long long c0 = (xa[k] - rad - org[k]) / g.cell - 1, c1 = (xa[k] + rad - org[k]) / g.cell + 1;
                lo[k] = min(lo[k], (int)max(0LL, min(c0, (long long)dim[k] - 1)));
                hi[k] = max(hi[k], (int)max(0LL, min(c1, (long long)dim[k] - 1)));
            }
        }
        const int bx = hi[0] - lo[0] + 1, by = hi[1] - lo[1] + 1, bxy = bx * by;
        const int nbox = bxy * (hi[2] - lo[2] + 1);
        for (int bi = tid; bi < nbox; bi += FB_THREADS) {
            const int bz = bi / bxy, rxy = bi - bz * bxy, byy = rxy / bx, bxx = rxy - byy * bx;
            const int qx = lo[0] + bxx, qy = lo[1] + byy, qz = lo[2] + bz;
            const int ci = (qz * g.dim.y + qy) * g.dim.x + qx;
            const long long cw = cwmax[ci];
            bool open = false;
            for (int a = 0; a < 4; a++) open |= box_dist2(X[a], g, qx, qy, qz) - cw <= thr[a];
            if (!open) continue;
            for (long long e = start[ci]; e < start[ci + 1]; e++) {
                const int sph = ids[e];
                const int3 cs = ld_int3(Ci, sph);
                const long long ws = W[sph];
                bool in = false;
                for (int a = 0; a < 4; a++) in |= pd_exact(X[a], cs, ws) <= thr[a];
                if (!in) continue;
                const int pos = atomicAdd(&sn, 1);
                if (pos < FB_GATHER) sid[pos] = sph;
            }
        }
        // and the heavy spheres, which the grid leaves out
        for (int h = tid; h < nh; h += FB_THREADS) {
            const int4 cs = hsph[h];
            bool in = false;
            for (int a = 0; a < 4; a++) in |= pd_exact(X[a], make_int3(cs.x, cs.y, cs.z), hw[h]) <= thr[a];
            if (!in) continue;
            const int pos = atomicAdd(&sn, 1);
            if (pos < FB_GATHER) sid[pos] = cs.w;
        }
        __syncthreads();
        const int n = sn;
        if (n > FB_GATHER) {
            if (tid == 0) {
                dev_fail(st, RPD_E_OVERFLOW, CNT_OVERFLOW);
                cand_cnt[t] = 0;
            }
            __syncthreads();
            continue;
        }
        // corner distances of the gathered spheres, then the exact corner
        // filter: keep i when, against every other j, some corner is at least
        // as close to i as to j
        if (tid < n) {
            const int3 cs = ld_int3(Ci, sid[tid]);
            const long long ws = W[sid[tid]];
            for (int cc = 0; cc < 4; cc++) sD[tid][cc] = pd_exact(X[cc], cs, ws);
        }
        __syncthreads();
        if (tid < n) {
            const long long d0 = sD[tid][0], d1 = sD[tid][1], d2 = sD[tid][2], d3 = sD[tid][3];
            bool ok = true;
            for (int j = 0; j < n && ok; j++)
                if (j != tid) ok = d0 <= sD[j][0] || d1 <= sD[j][1] || d2 <= sD[j][2] || d3 <= sD[j][3];
            skeep[tid] = ok;
        }
        __syncthreads();
        if (tid < 32) {   // the kept spheres, one per lane: rank by id and by (sum of corner distances, id)
            unsigned keep[FB_GATHER / 32];
            int nk = 0;
            for (int k = 0; k < FB_GATHER / 32; k++) {
                const int i = 32 * k + lane;
                keep[k] = __ballot_sync(FULL, i < n && skeep[i]);
                nk += __popc(keep[k]);
            }
            if (nk > RPD_MAXC) {
                if (lane == 0) {
                    dev_fail(st, RPD_E_OVERFLOW, CNT_OVERFLOW);
                    cand_cnt[t] = 0;
                }
            } else {
                int mine = -1, k0 = 0;
                for (int k = 0; k < FB_GATHER / 32; k++) {
                    const unsigned m = keep[k];
                    const int c = __popc(m);
                    if (lane >= k0 && lane < k0 + c) mine = 32 * k + (int)__fns(m, 0, lane - k0 + 1);
                    k0 += c;
                }
                int my = -1;
                long long key = 0;
                if (mine >= 0) {
                    my = sid[mine];
                    key = sD[mine][0] + sD[mine][1] + sD[mine][2] + sD[mine][3];
                }
                int rank = 0, rank2 = 0;
                for (int j = 0; j < nk; j++) {
                    const int sj = __shfl_sync(FULL, my, j);
                    const long long kj = __shfl_sync(FULL, key, j);
                    rank += sj < my;
                    rank2 += (kj < key) || (kj == key && sj < my);
                }
                if (mine >= 0) {
                    cand[t * RPD_MAXC + rank] = my;
                    cand_ord[t * RPD_MAXC + rank2] = (uint8_t)rank;
                }
                if (lane == 0) {
                    cand_cnt[t] = nk;
                    atomicAdd(&st->cnt[CNT_CAND_FALLBACK], 1ull);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t grid_tmp_bytes(long long ns, long long ncap) {
    return al(sizeof(int32_t) * (ncap + 1)) * 2 + al(scan_tmp_bytes(ncap));
}

int heavy_count(long long ns) { return (int)std::min<long long>(HEAVY_MAX, ns / 128); }

void launch_heavy_select(const int32_t* Ci, const long long* W, long long ns, long long* wcut, int4* hsph,
                         long long* hw, int* nheavy, cudaStream_t s) {
    const int H = heavy_count(ns);
    if (H < 1) {
        const long long big = LLONG_MAX;
        const int zero = 0;
        cudaMemcpyAsync(wcut, &big, sizeof(big), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(nheavy, &zero, sizeof(zero), cudaMemcpyHostToDevice, s);
        return;
    }
    k_heavy_select<<<1, 1024, 0, s>>>(Ci, W, ns, H, wcut, hsph, hw, nheavy);
    note_launch();
}

void launch_sphere_grid(const int32_t* Ci, const long long* W, long long ns, long long ncap, GridParams* gp,
                        int64_t* cell_start, int32_t* cell_ids, int4* cell_sph, long long* cell_w,
                        long long* cell_wmax, void* tmp, cudaStream_t s, const long long* wcut) {
    if (ncap <= GRID_SMALL_CAP) {
        k_grid_small<<<1, 1024, sizeof(int) * ncap, s>>>(Ci, W, ns, ncap, gp, cell_start, cell_ids, cell_sph, cell_w,
                                                         cell_wmax, cell_wmax + ncap, wcut);
        note_launch();
        return;
    }
    char* p = (char*)tmp;
    int32_t* count = (int32_t*)p; p += al(sizeof(int32_t) * (ncap + 1));
    int32_t* fill = (int32_t*)p; p += al(sizeof(int32_t) * (ncap + 1));
    void* stmp = p;
    k_bbox<<<1, 1024, 0, s>>>(Ci, W, ns, ncap, gp, wcut);
    note_launch();
    cudaMemsetAsync(count, 0, sizeof(int32_t) * ncap, s);
    cudaMemsetAsync(fill, 0, sizeof(int32_t) * ncap, s);
    cudaMemsetAsync(cell_wmax, 0, sizeof(long long) * 2 * ncap, s);
    k_cell_count<<<nblk(ns, 256), 256, 0, s>>>(Ci, W, ns, gp, count, cell_wmax, cell_wmax + ncap, wcut);
    note_launch();
    scan_excl(count, cell_start, ncap, stmp, s);
    k_cell_fill<<<nblk(ns, 256), 256, 0, s>>>(Ci, W, ns, gp, cell_start, fill, cell_ids, cell_sph, cell_w, wcut);
    note_launch();
}

size_t knn_tmp_bytes(long long nv) {
    return 2 * al(sizeof(uint64_t) * nv) + 2 * al(sizeof(uint32_t) * nv) + radix_tmp_bytes(nv);
}

long long batch_grid_cap() { return GRID_SMALL_CAP; }

void launch_sphere_grid_batch(const int32_t* Ci, const long long* W, const long long* soff, int nshapes,
                              long long ncap_total, GridParams* gp, int64_t* cell_start, int32_t* cell_ids,
                              int4* cell_sph, long long* cell_w, long long* cell_wmax, long long max_shape_ncap,
                              cudaStream_t s) {
    if (nshapes <= 0) return;
    k_grid_batch<<<(unsigned)nshapes, 1024, sizeof(int) * max_shape_ncap, s>>>(Ci, W, soff, ncap_total, gp, cell_start,
                                                                                cell_ids, cell_sph, cell_w, cell_wmax);
    note_launch();
}

void launch_knn(const int32_t* Xi, long long nv, long long ns, const GridParams* gp, const int64_t* cell_start,
                const int4* cell_sph, const long long* cell_w, const long long* cell_wmax, long long ncap, int K,
                int32_t* knn, long long* dplus, void* tmp, int* d_err, bool two_word, cudaStream_t s,
                const long long* voff, int nshapes, const int4* hsph, const long long* hw, const int* nheavy) {
    if (nv == 0) return;
    char* p = (char*)tmp;
    uint64_t* k0 = (uint64_t*)p; p += al(sizeof(uint64_t) * nv);
    uint64_t* k1 = (uint64_t*)p; p += al(sizeof(uint64_t) * nv);
    uint32_t* v0 = (uint32_t*)p; p += al(sizeof(uint32_t) * nv);
    uint32_t* v1 = (uint32_t*)p; p += al(sizeof(uint32_t) * nv);
    int bits = 1;
    while ((1ll << bits) < ncap) bits++;
    if ((ns <= (1 << 17) || nshapes > 1) && !two_word) {   // batches: shape-local ids in the key
        // one vertex per warp in input order: the sphere grid stays in cache
        if (nheavy)
            k_knn_warp<true><<<nblk(32 * nv, 256), 256, 0, s>>>(Xi, nullptr, nv, gp, cell_start, cell_sph, cell_w,
                                                                 cell_wmax + ncap, K, knn, dplus, voff, nshapes, hsph,
                                                                 hw, nheavy);
        else
            k_knn_warp<false><<<nblk(32 * nv, 256), 256, 0, s>>>(Xi, nullptr, nv, gp, cell_start, cell_sph, cell_w,
                                                                  cell_wmax + ncap, K, knn, dplus, voff, nshapes,
                                                                  nullptr, nullptr, nullptr);
    } else {
        k_vertex_cells<<<nblk(nv, 256), 256, 0, s>>>(Xi, nv, gp, k0, v0);
        note_launch();
        radix_sort_pairs(k0, v0, k1, v1, nv, bits, p, d_err, s);
        k_knn_group<RPD_MAXK, PairEntry><<<nblk(nv, 32), 128, 0, s>>>(Xi, v1, nv, gp, cell_start, cell_sph, cell_w, K,
                                                                       knn, dplus, d_err);
    }
    note_launch();
}

void launch_candidates(const int32_t* d_tets, long long nt, long long nv, const int32_t* Xi, const int32_t* Ci,
                       const long long* W, const int32_t* knn, const long long* dplus, int K, const GridParams* gp,
                       const int64_t* cell_start, const int32_t* cell_ids, const long long* cell_wmax,
                       int32_t* cand_cnt, int32_t* cand, uint8_t* cand_ord, int32_t* fb_list, int32_t* fb_count,
                       DevState* st, cudaStream_t s, const long long* voff, int nshapes, const int4* hsph,
                       const long long* hw, const int* nheavy) {
    if (nt == 0) return;
    cudaMemsetAsync(fb_count, 0, sizeof(int32_t), s);
    k_candidates_warp<<<nblk(32 * nt, 256), 256, 0, s>>>(d_tets, nt, nv, Xi, Ci, W, knn, dplus, K, cand_cnt, cand,
                                                          cand_ord,
                                               fb_list, fb_count, st);
    note_launch();
    k_candidates_fallback<<<152 * 4, FB_THREADS, 0, s>>>(d_tets, nv, Xi, Ci, W, knn, K, gp, cell_start, cell_ids,
                                                         cell_wmax, fb_list, fb_count, cand_cnt, cand, cand_ord, st,
                                                         voff, nshapes, hsph, hw, nheavy);
    note_launch();
}

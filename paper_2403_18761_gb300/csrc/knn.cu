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

// Lower bound of |x - y|^2 over points y in grid cells at Chebyshev index
// distance >= r from cell c (LLONG_MAX when there is no such cell).
__device__ __forceinline__ long long ring_lb2(int3 x, const GridParams& g, int3 c, int r) {
    long long best = LLONG_MAX;
    const int xs[3] = {x.x, x.y, x.z}, cs[3] = {c.x, c.y, c.z}, ds[3] = {g.dim.x, g.dim.y, g.dim.z},
              os[3] = {g.org.x, g.org.y, g.org.z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (cs[a] + r <= ds[a] - 1) {
            long long start = (long long)os[a] + (long long)(cs[a] + r) * g.cell;
            best = min(best, max(0LL, start - xs[a]));
        }
        if (cs[a] - r >= 0) {
            long long end = (long long)os[a] + (long long)(cs[a] - r + 1) * g.cell - 1;
            best = min(best, max(0LL, (long long)xs[a] - end));
        }
    }
    return best == LLONG_MAX ? LLONG_MAX : best * best;
}

// Visit the cells of the Chebyshev shell of radius r around c.
template <typename F>
__device__ __forceinline__ void for_shell(const GridParams& g, int3 c, int r, F&& f) {
    const int z0 = max(-r, -c.z), z1 = min(r, g.dim.z - 1 - c.z);
    const int y0 = max(-r, -c.y), y1 = min(r, g.dim.y - 1 - c.y);
    for (int dz = z0; dz <= z1; dz++) {
        for (int dy = y0; dy <= y1; dy++) {
            bool full = (dz == -r || dz == r || dy == -r || dy == r);
            if (full) {
                const int x0 = max(-r, -c.x), x1 = min(r, g.dim.x - 1 - c.x);
                for (int dx = x0; dx <= x1; dx++) f(c.x + dx, c.y + dy, c.z + dz);
            } else {
                if (c.x - r >= 0) f(c.x - r, c.y + dy, c.z + dz);
                if (r > 0 && c.x + r <= g.dim.x - 1) f(c.x + r, c.y + dy, c.z + dz);
            }
        }
    }
}

__global__ void k_bbox(const int32_t* __restrict__ Ci, const long long* __restrict__ W, long long ns, long long ncap,
                       GridParams* gp) {
    __shared__ int smin[3][32], smax[3][32];
    __shared__ long long swm[32];
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    long long wm = 0;
    for (long long i = threadIdx.x; i < ns; i += blockDim.x) {
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
        long long ext[3];
        for (int a = 0; a < 3; a++) ext[a] = (long long)mx[a] - mn[a] + 1;
        double vol = (double)ext[0] * (double)ext[1] * (double)ext[2];
        double target = (double)(ns < 1 ? 1 : ns);
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
        *gp = g;
    }
}

__global__ void k_cell_count(const int32_t* __restrict__ Ci, const long long* __restrict__ W, long long ns,
                             const GridParams* __restrict__ gp, int32_t* __restrict__ count,
                             long long* __restrict__ cwmax) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    GridParams g = *gp;
    int3 c = cell_of(ld_int3(Ci, i), g);
    int q = (c.z * g.dim.y + c.y) * g.dim.x + c.x;
    atomicAdd(&count[q], 1);
    atomicMax((unsigned long long*)&cwmax[q], (unsigned long long)W[i]);
}

__global__ void k_cell_fill(const int32_t* __restrict__ Ci, long long ns, const GridParams* __restrict__ gp,
                            const int64_t* __restrict__ start, int32_t* __restrict__ fill, int32_t* __restrict__ ids) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    GridParams g = *gp;
    int3 c = cell_of(ld_int3(Ci, i), g);
    int q = (c.z * g.dim.y + c.y) * g.dim.x + c.x;
    int slot = atomicAdd(&fill[q], 1);
    ids[start[q] + slot] = (int32_t)i;
}

// ---------------------------------------------------------------- kNN
__global__ void __launch_bounds__(128) k_knn(const int32_t* __restrict__ Xi, long long nv, const int32_t* __restrict__ Ci,
                      const long long* __restrict__ W, const GridParams* __restrict__ gp,
                      const int64_t* __restrict__ start, const int32_t* __restrict__ ids,
                      const long long* __restrict__ cwmax, int K, int32_t* __restrict__ knn,
                      long long* __restrict__ dplus) {
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const GridParams g = *gp;
    const int3 x = ld_int3(Xi, v);
    const int3 c = cell_of(x, g);
    long long bd[RPD_MAXK];
    int bi[RPD_MAXK];
    int cnt = 0;
    long long dp = LLONG_MAX;
    for (int r = 0;; r++) {
        if (r > 0) {
            long long lb2 = ring_lb2(x, g, c, r);
            if (lb2 == LLONG_MAX) break;                 // every cell visited
            long long plb = lb2 - g.wmax;
            if (cnt == K && plb > bd[K - 1]) {
                dp = min(dp, plb);
                break;
            }
        }
        for_shell(g, c, r, [&](int qx, int qy, int qz) {
            int q = (qz * g.dim.y + qy) * g.dim.x + qx;
            long long s0 = start[q], s1 = start[q + 1];
            if (s0 == s1) return;
            long long plb = box_dist2(x, g, qx, qy, qz) - cwmax[q];
            if (cnt == K && plb > bd[K - 1]) {
                dp = min(dp, plb);
                return;
            }
            for (long long e = s0; e < s1; e++) {
                int s = ids[e];
                long long d = pd_exact(x, ld_int3(Ci, s), W[s]);
                if (cnt < K || d < bd[K - 1] || (d == bd[K - 1] && s < bi[K - 1])) {
                    if (cnt == K) dp = min(dp, bd[K - 1]);
                    int p = cnt < K ? cnt++ : K - 1;
                    while (p > 0 && (bd[p - 1] > d || (bd[p - 1] == d && bi[p - 1] > s))) {
                        bd[p] = bd[p - 1];
                        bi[p] = bi[p - 1];
                        p--;
                    }
                    bd[p] = d;
                    bi[p] = s;
                } else {
                    dp = min(dp, d);
                }
            }
        });
    }
    for (int j = 0; j < K; j++) knn[v * K + j] = j < cnt ? bi[j] : -1;
    dplus[v] = dp;
}

// ---------------------------------------------------------- candidates
struct Gathered {
    int id;
    long long D[4];
};

// Keep the gathered spheres that pass the exact corner test against every
// other gathered sphere; write them sorted by index.
// Also writes the clip order: slots sorted by power distance at the tet
// centroid (sum_a pd(X_a, s) = 4 pd(centroid, s) + a sphere-independent term).
template <int CAP>
__device__ void finish_candidates(Gathered* G, int n, long long t, int32_t* __restrict__ cand_cnt,
                                  int32_t* __restrict__ cand, uint8_t* __restrict__ cand_ord, DevState* st) {
    int kept[RPD_MAXC];   // indices into G, sorted by sphere index
    int nk = 0;
    for (int s = 0; s < n; s++) {
        bool ok = true;
        for (int j = 0; j < n && ok; j++) {
            if (j == s) continue;
            bool some = false;
#pragma unroll
            for (int a = 0; a < 4; a++) some |= (G[s].D[a] <= G[j].D[a]);
            ok = some;
        }
        if (!ok) continue;
        if (nk == RPD_MAXC) {
            dev_fail(st, RPD_E_OVERFLOW, CNT_OVERFLOW);
            cand_cnt[t] = 0;
            return;
        }
        int p = nk++;
        while (p > 0 && G[kept[p - 1]].id > G[s].id) {
            kept[p] = kept[p - 1];
            p--;
        }
        kept[p] = s;
    }
    uint8_t ord[RPD_MAXC];
    for (int j = 0; j < nk; j++) {
        cand[t * RPD_MAXC + j] = G[kept[j]].id;
        const Gathered& g = G[kept[j]];
        long long key = g.D[0] + g.D[1] + g.D[2] + g.D[3];
        int p = j;
        while (p > 0) {
            const Gathered& h = G[kept[ord[p - 1]]];
            long long hk = h.D[0] + h.D[1] + h.D[2] + h.D[3];
            if (hk <= key) break;
            ord[p] = ord[p - 1];
            p--;
        }
        ord[p] = (uint8_t)j;
    }
    for (int j = 0; j < nk; j++) cand_ord[t * RPD_MAXC + j] = ord[j];
    cand_cnt[t] = nk;
}

__device__ __forceinline__ bool load_tet(const int32_t* __restrict__ T, long long t, long long nv,
                                         const int32_t* __restrict__ Xi, int* v, int3* X) {
    for (int a = 0; a < 4; a++) {
        v[a] = T[4 * t + a];
        if (v[a] < 0 || v[a] >= nv) return false;
        X[a] = ld_int3(Xi, v[a]);
    }
    return true;
}

__global__ void __launch_bounds__(128) k_candidates(const int32_t* __restrict__ T, long long nt, long long nv,
                             const int32_t* __restrict__ Xi, const int32_t* __restrict__ Ci,
                             const long long* __restrict__ W, const int32_t* __restrict__ knn,
                             const long long* __restrict__ dplus, int K, int32_t* __restrict__ cand_cnt,
                             int32_t* __restrict__ cand, uint8_t* __restrict__ cand_ord, int32_t* __restrict__ fb_list,
                             int32_t* __restrict__ fb_count, DevState* st) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int v[4];
    int3 X[4];
    if (!load_tet(T, t, nv, Xi, v, X)) {
        cand_cnt[t] = 0;
        return;
    }
    int o[4];
    long long dp[4], M[4][4];
    for (int a = 0; a < 4; a++) {
        o[a] = knn[(long long)v[a] * K];
        dp[a] = dplus[v[a]];
    }
    for (int b = 0; b < 4; b++) {
        int3 cb = ld_int3(Ci, o[b]);
        long long wb = W[o[b]];
        for (int a = 0; a < 4; a++) M[a][b] = pd_exact(X[a], cb, wb);
    }
    int bstar = -1;
    long long best = LLONG_MAX;
    for (int b = 0; b < 4; b++) {
        bool complete = true;
        long long score = 0;
        for (int a = 0; a < 4; a++) {
            complete &= dp[a] > M[a][b];
            score = max(score, M[a][b] - M[a][a]);
        }
        if (complete && score < best) {
            best = score;
            bstar = b;
        }
    }
    if (bstar < 0) {
        int slot = atomicAdd(fb_count, 1);
        fb_list[slot] = (int32_t)t;
        cand_cnt[t] = 0;
        return;
    }
    Gathered G[RPD_GATHER];
    int n = 0;
    for (int a = 0; a < 4; a++) {
        long long thr = M[a][bstar];
        for (int j = 0; j < K; j++) {
            int s = knn[(long long)v[a] * K + j];
            if (s < 0) break;
            int3 cs = ld_int3(Ci, s);
            long long ws = W[s];
            long long d = pd_exact(X[a], cs, ws);
            if (d > thr) break;                       // lists are sorted by distance
            bool dup = false;
            for (int q = 0; q < n && !dup; q++) dup = (G[q].id == s);
            if (dup) continue;
            if (n == RPD_GATHER) {
                int slot = atomicAdd(fb_count, 1);
                fb_list[slot] = (int32_t)t;
                cand_cnt[t] = 0;
                return;
            }
            G[n].id = s;
            for (int c = 0; c < 4; c++) G[n].D[c] = pd_exact(X[c], cs, ws);
            n++;
        }
    }
    finish_candidates<RPD_GATHER>(G, n, t, cand_cnt, cand, cand_ord, st);
}

#define RPD_FB_GATHER 128

__device__ void fallback_one(const int32_t* __restrict__ T, long long nv, const int32_t* __restrict__ Xi,
                             const int32_t* __restrict__ Ci, const long long* __restrict__ W,
                             const int32_t* __restrict__ knn, int K, const GridParams* __restrict__ gp,
                             const int64_t* __restrict__ start, const int32_t* __restrict__ ids,
                             const long long* __restrict__ cwmax, long long t, int32_t* __restrict__ cand_cnt,
                             int32_t* __restrict__ cand, uint8_t* __restrict__ cand_ord, DevState* st);

__global__ void __launch_bounds__(64) k_candidates_fallback(const int32_t* __restrict__ T, long long nv,
                                      const int32_t* __restrict__ Xi, const int32_t* __restrict__ Ci,
                                      const long long* __restrict__ W, const int32_t* __restrict__ knn, int K,
                                      const GridParams* __restrict__ gp, const int64_t* __restrict__ start,
                                      const int32_t* __restrict__ ids, const long long* __restrict__ cwmax,
                                      const int32_t* __restrict__ fb_list, const int32_t* __restrict__ fb_count,
                                      int32_t* __restrict__ cand_cnt, int32_t* __restrict__ cand,
                                      uint8_t* __restrict__ cand_ord, DevState* st) {
    const long long nfb = *fb_count;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nfb;
         q += (long long)gridDim.x * blockDim.x)
        fallback_one(T, nv, Xi, Ci, W, knn, K, gp, start, ids, cwmax, fb_list[q], cand_cnt, cand, cand_ord, st);
}

__device__ void fallback_one(const int32_t* __restrict__ T, long long nv, const int32_t* __restrict__ Xi,
                             const int32_t* __restrict__ Ci, const long long* __restrict__ W,
                             const int32_t* __restrict__ knn, int K, const GridParams* __restrict__ gp,
                             const int64_t* __restrict__ start, const int32_t* __restrict__ ids,
                             const long long* __restrict__ cwmax, long long t, int32_t* __restrict__ cand_cnt,
                             int32_t* __restrict__ cand, uint8_t* __restrict__ cand_ord, DevState* st) {
    int v[4];
    int3 X[4];
    if (!load_tet(T, t, nv, Xi, v, X)) return;
    const GridParams g = *gp;
    int o[4];
    long long M[4][4];
    for (int a = 0; a < 4; a++) o[a] = knn[(long long)v[a] * K];
    for (int b = 0; b < 4; b++)
        for (int a = 0; a < 4; a++) M[a][b] = pd_exact(X[a], ld_int3(Ci, o[b]), W[o[b]]);
    int bstar = 0;
    long long best = LLONG_MAX;
    for (int b = 0; b < 4; b++) {
        long long score = 0;
        for (int a = 0; a < 4; a++) score = max(score, M[a][b] - M[a][a]);
        if (score < best) { best = score; bstar = b; }
    }
    Gathered G[RPD_FB_GATHER];
    int n = 0;
    bool over = false;
    for (int a = 0; a < 4 && !over; a++) {
        long long thr = M[a][bstar];
        int3 x = X[a];
        int3 c = cell_of(x, g);
        for (int r = 0; !over; r++) {
            if (r > 0) {
                long long lb2 = ring_lb2(x, g, c, r);
                if (lb2 == LLONG_MAX || lb2 - g.wmax > thr) break;
            }
            for_shell(g, c, r, [&](int qx, int qy, int qz) {
                int cq = (qz * g.dim.y + qy) * g.dim.x + qx;
                if (over || box_dist2(x, g, qx, qy, qz) - cwmax[cq] > thr) return;
                for (long long e = start[cq]; e < start[cq + 1]; e++) {
                    int s = ids[e];
                    int3 cs = ld_int3(Ci, s);
                    long long ws = W[s];
                    if (pd_exact(x, cs, ws) > thr) continue;
                    bool dup = false;
                    for (int z = 0; z < n && !dup; z++) dup = (G[z].id == s);
                    if (dup) continue;
                    if (n == RPD_FB_GATHER) { over = true; return; }
                    G[n].id = s;
                    for (int cc = 0; cc < 4; cc++) G[n].D[cc] = pd_exact(X[cc], cs, ws);
                    n++;
                }
            });
        }
    }
    if (over) {
        dev_fail(st, RPD_E_OVERFLOW, CNT_OVERFLOW);
        cand_cnt[t] = 0;
        return;
    }
    atomicAdd(&st->cnt[CNT_CAND_FALLBACK], 1ull);
    finish_candidates<RPD_FB_GATHER>(G, n, t, cand_cnt, cand, cand_ord, st);
}

}  // namespace

size_t grid_tmp_bytes(long long ns, long long ncap) {
    return al(sizeof(int32_t) * (ncap + 1)) * 2 + al(scan_tmp_bytes(ncap));
}

void launch_sphere_grid(const int32_t* Ci, const long long* W, long long ns, long long ncap, GridParams* gp,
                        int64_t* cell_start, int32_t* cell_ids, long long* cell_wmax, void* tmp, cudaStream_t s) {
    char* p = (char*)tmp;
    int32_t* count = (int32_t*)p; p += al(sizeof(int32_t) * (ncap + 1));
    int32_t* fill = (int32_t*)p; p += al(sizeof(int32_t) * (ncap + 1));
    void* stmp = p;
    k_bbox<<<1, 1024, 0, s>>>(Ci, W, ns, ncap, gp);
    cudaMemsetAsync(count, 0, sizeof(int32_t) * ncap, s);
    cudaMemsetAsync(fill, 0, sizeof(int32_t) * ncap, s);
    cudaMemsetAsync(cell_wmax, 0, sizeof(long long) * ncap, s);
    k_cell_count<<<nblk(ns, 256), 256, 0, s>>>(Ci, W, ns, gp, count, cell_wmax);
    scan_excl(count, cell_start, ncap, stmp, s);
    k_cell_fill<<<nblk(ns, 256), 256, 0, s>>>(Ci, ns, gp, cell_start, fill, cell_ids);
}

void launch_knn(const int32_t* Xi, long long nv, const int32_t* Ci, const long long* W, const GridParams* gp,
                const int64_t* cell_start, const int32_t* cell_ids, const long long* cell_wmax, int K,
                int32_t* knn, long long* dplus, cudaStream_t s) {
    if (nv == 0) return;
    k_knn<<<nblk(nv, 128), 128, 0, s>>>(Xi, nv, Ci, W, gp, cell_start, cell_ids, cell_wmax, K, knn, dplus);
}

void launch_candidates(const int32_t* d_tets, long long nt, long long nv, const int32_t* Xi, const int32_t* Ci,
                       const long long* W, const int32_t* knn, const long long* dplus, int K, const GridParams* gp,
                       const int64_t* cell_start, const int32_t* cell_ids, const long long* cell_wmax,
                       int32_t* cand_cnt, int32_t* cand, uint8_t* cand_ord, int32_t* fb_list, int32_t* fb_count,
                       DevState* st, cudaStream_t s) {
    if (nt == 0) return;
    cudaMemsetAsync(fb_count, 0, sizeof(int32_t), s);
    k_candidates<<<nblk(nt, 128), 128, 0, s>>>(d_tets, nt, nv, Xi, Ci, W, knn, dplus, K, cand_cnt, cand, cand_ord,
                                               fb_list, fb_count, st);
    k_candidates_fallback<<<152, 64, 0, s>>>(d_tets, nv, Xi, Ci, W, knn, K, gp, cell_start, cell_ids, cell_wmax,
                                             fb_list, fb_count, cand_cnt, cand, cand_ord, st);
}

// Batches of independent shapes in one context (the paper builds one shape at
// a time).  The shapes' vertices, tets and spheres are concatenated; every
// stage runs once over the union (one launch per stage, the pairs of all
// shapes binned together by candidate count), and a tet sees only the
// spheres of its own shape because the neighbour search walks a grid per
// shape (knn.cu).  These kernels check that no tet reaches into another
// shape and cut the sorted result tables into per-shape ranges.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"
#include "prim.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Every corner of a tet of shape s must be a vertex of shape s.
__global__ void k_batch_check(const int32_t* __restrict__ tets, const long long* __restrict__ toff,
                              const long long* __restrict__ voff, int nshapes, DevState* st) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= toff[nshapes]) return;
    int lo = 0, hi = nshapes - 1;   // the shape holding tet t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (toff[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    for (int k = 0; k < 4; k++) {
        const long long v = tets[4 * t + k];
        if (v < voff[lo] || v >= voff[lo + 1]) {
            dev_fail(st, RPD_E_INVALID, CNT_INVALID);
            return;
        }
    }
}

// Row ranges of a sorted table per shape: out[s] = the first row whose
// leading column (a sphere id, or a tet id for pieces) is >= bound[s], for
// s = 0..nshapes (bound[nshapes] = the total: out = rows).
__global__ void k_batch_cut(const int32_t* __restrict__ lead, long long rows, int stride,
                            const long long* __restrict__ bound, int nshapes, long long* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nshapes) return;
    const long long b = bound[s];
    long long lo = 0, hi = rows;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((long long)lead[mid * stride] < b) lo = mid + 1;
        else hi = mid;
    }
    out[s] = lo;
}

// Piece ranges: the pieces of shape s are those of its tets, i.e. of the
// pairs [pair_off[toff[s]], pair_off[toff[s + 1]]), compacted by piece_off.
__global__ void k_batch_cut_pieces(const int64_t* __restrict__ pair_off, const int64_t* __restrict__ piece_off,
                                   const long long* __restrict__ toff, int nshapes, long long* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nshapes) return;
    out[s] = piece_off[pair_off[toff[s]]];
}

}  // namespace

void launch_batch_check(const int32_t* tets, const long long* toff, const long long* voff, int nshapes,
                        long long nt, DevState* st, cudaStream_t s) {
    if (nt <= 0) return;
    k_batch_check<<<nblk(nt, 256), 256, 0, s>>>(tets, toff, voff, nshapes, st);
    note_launch();
}

void launch_batch_cut(const int32_t* lead, long long rows, int stride, const long long* bound, int nshapes,
                      long long* out, cudaStream_t s) {
    k_batch_cut<<<nblk(nshapes + 1, 128), 128, 0, s>>>(lead, rows, stride, bound, nshapes, out);
    note_launch();
}

void launch_batch_cut_pieces(const int64_t* pair_off, const int64_t* piece_off, const long long* toff, int nshapes,
                             long long* out, cudaStream_t s) {
    k_batch_cut_pieces<<<nblk(nshapes + 1, 128), 128, 0, s>>>(pair_off, piece_off, toff, nshapes, out);
    note_launch();
}

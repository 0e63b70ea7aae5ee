// A0: input snapping, validation, face adjacency and ownership bits.
//
// The fractional Euler weights of Sec. 4.1.2 are derived "from the
// combinatorial structure of the tetrahedral mesh": a mesh face shared by n
// tets weighs 1/n in each.  The library uses the equivalent integer form in
// which the whole weight goes to the lowest-numbered tet containing the face
// (every tet that contains a mesh face clips it to the same restricted set,
// so the n copies of 1/n and one copy of 1 sum to the same value).
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "prim.cuh"

namespace {

__global__ void k_snap_points(const double* __restrict__ x, long long n3, double scale, int32_t* __restrict__ out,
                              DevState* st) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    double v = x[i] * scale;
    if (!(fabs(v) <= (double)RPD_COORD_MAX)) {   // also rejects NaN
        dev_fail(st, RPD_E_INVALID, CNT_INVALID);
        out[i] = 0;
        return;
    }
    out[i] = (int32_t)rint(v);
}

__global__ void k_snap_radii(const double* __restrict__ r, long long n, double scale, long long* __restrict__ W,
                             DevState* st) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = r[i] * scale;
    if (!(v >= 0.0 && v <= (double)(1 << 22))) {
        dev_fail(st, RPD_E_INVALID, CNT_INVALID);
        W[i] = 0;
        return;
    }
    long long q = (long long)rint(v);
    W[i] = q * q;
}

// Exact orientation: det[p1-p0, p2-p0, p3-p0] > 0 with 128-bit integers.
__global__ void k_check_tets(const int32_t* __restrict__ T, long long nt, long long nv, const int32_t* __restrict__ Xi,
                             DevState* st) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int v[4];
    for (int a = 0; a < 4; a++) {
        v[a] = T[4 * t + a];
        if (v[a] < 0 || v[a] >= nv) {
            dev_fail(st, RPD_E_INVALID, CNT_INVALID);
            return;
        }
    }
    int3 p0 = ld_int3(Xi, v[0]), p1 = ld_int3(Xi, v[1]), p2 = ld_int3(Xi, v[2]), p3 = ld_int3(Xi, v[3]);
    long long ax = p1.x - p0.x, ay = p1.y - p0.y, az = p1.z - p0.z;
    long long bx = p2.x - p0.x, by = p2.y - p0.y, bz = p2.z - p0.z;
    long long cx = p3.x - p0.x, cy = p3.y - p0.y, cz = p3.z - p0.z;
    __int128 d = (__int128)ax * ((__int128)by * cz - (__int128)bz * cy) -
                 (__int128)ay * ((__int128)bx * cz - (__int128)bz * cx) +
                 (__int128)az * ((__int128)bx * cy - (__int128)by * cx);
    if (d <= 0) dev_fail(st, RPD_E_INVALID, CNT_INVALID);
}

__device__ __forceinline__ void sort3(unsigned long long& a, unsigned long long& b, unsigned long long& c) {
    unsigned long long t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
}

// Face f of a tet is the triangle opposite local vertex f.
// Vertex ids use vb bits (nv <= 2^vb), so a face key has 3 vb bits.
__global__ void k_face_keys(const int32_t* __restrict__ T, long long nt, int vb, uint64_t* __restrict__ key,
                            uint32_t* __restrict__ val) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * nt) return;
    long long t = i >> 2;
    int f = (int)(i & 3);
    unsigned long long v[3];
    int n = 0;
    for (int c = 0; c < 4; c++)
        if (c != f) v[n++] = (unsigned)T[4 * t + c] & ((1u << vb) - 1u);
    sort3(v[0], v[1], v[2]);
    key[i] = (v[0] << (2 * vb)) | (v[1] << vb) | v[2];
    val[i] = (uint32_t)i;
}

__global__ void k_edge_keys(const int32_t* __restrict__ T, long long nt, int vb, uint64_t* __restrict__ key,
                            uint32_t* __restrict__ val) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * nt) return;
    long long t = i / 6;
    int e = (int)(i - 6 * t);
    const int EA[6] = {0, 0, 0, 1, 1, 2}, EB[6] = {1, 2, 3, 2, 3, 3};
    unsigned long long a = (unsigned)T[4 * t + EA[e]] & ((1u << vb) - 1u);
    unsigned long long b = (unsigned)T[4 * t + EB[e]] & ((1u << vb) - 1u);
    if (a > b) { unsigned long long s = a; a = b; b = s; }
    key[i] = (a << vb) | b;
    val[i] = (uint32_t)i;
}

// Runs of equal face keys: adjacency, face ownership, > 2 tets -> error.
__global__ void k_face_runs(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, long long n,
                            int32_t* __restrict__ adj, uint32_t* __restrict__ own, DevState* st) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = key[i];
    bool first = (i == 0) || key[i - 1] != k;
    if (!first) return;
    long long j = i + 1;
    while (j < n && key[j] == k && j - i < 3) j++;
    long long cnt = j - i;
    if (cnt > 2) {
        dev_fail(st, RPD_E_NONMANIFOLD, CNT_NONMANIFOLD);
        return;
    }
    uint32_t a = val[i];
    atomicOr(&own[a >> 2], 1u << (10 + (a & 3)));
    if (cnt == 2) {
        uint32_t b = val[i + 1];
        adj[a] = (int32_t)(b >> 2);
        adj[b] = (int32_t)(a >> 2);
    }
}

__global__ void k_edge_runs(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, long long n,
                            uint32_t* __restrict__ own) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0 || key[i - 1] != key[i]) {
        uint32_t a = val[i];   // stable sort: lowest tet first
        atomicOr(&own[a / 6], 1u << (4 + a % 6));
    }
}

__global__ void k_vertex_min(const int32_t* __restrict__ T, long long nt, long long nv, int32_t* __restrict__ vmin) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * nt) return;
    int v = T[i];
    if (v >= 0 && v < nv) atomicMin(&vmin[v], (int32_t)(i >> 2));
}

__global__ void k_vertex_own(const int32_t* __restrict__ T, long long nt, long long nv,
                             const int32_t* __restrict__ vmin, uint32_t* __restrict__ own) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    uint32_t b = 0;
    for (int a = 0; a < 4; a++) {
        int v = T[4 * t + a];
        if (v >= 0 && v < nv && vmin[v] == (int32_t)t) b |= 1u << a;
    }
    atomicOr(&own[t], b);
}

__global__ void k_fill_i32(int32_t* p, long long n, int32_t v) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }
size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

void launch_snap(const double* d_verts, long long nv, const double* d_centers, const double* d_radii, long long ns,
                 int grid_bits, int32_t* Xi, int32_t* Ci, long long* W, DevState* st, cudaStream_t s) {
    double scale = ldexp(1.0, grid_bits);
    const int T = 256;
    if (nv) {
        k_snap_points<<<nblk(3 * nv, T), T, 0, s>>>(d_verts, 3 * nv, scale, Xi, st);
        note_launch();
    }
    if (ns) {
        k_snap_points<<<nblk(3 * ns, T), T, 0, s>>>(d_centers, 3 * ns, scale, Ci, st);
        note_launch();
        k_snap_radii<<<nblk(ns, T), T, 0, s>>>(d_radii, ns, scale, W, st);
        note_launch();
    }
}

size_t prep_tmp_bytes(long long nt, long long nv) {
    long long n = 6 * nt;
    return 2 * al(sizeof(uint64_t) * n) + 2 * al(sizeof(uint32_t) * n) + al(sizeof(int32_t) * nv) +
           al(radix_tmp_bytes(n));
}

void launch_prep_mesh(const int32_t* d_tets, long long nt, long long nv, const int32_t* Xi, int32_t* adj,
                      uint32_t* own, void* tmp, DevState* st, cudaStream_t s) {
    const int T = 256;
    long long n6 = 6 * nt;
    char* p = (char*)tmp;
    uint64_t* k0 = (uint64_t*)p; p += al(sizeof(uint64_t) * n6);
    uint64_t* k1 = (uint64_t*)p; p += al(sizeof(uint64_t) * n6);
    uint32_t* v0 = (uint32_t*)p; p += al(sizeof(uint32_t) * n6);
    uint32_t* v1 = (uint32_t*)p; p += al(sizeof(uint32_t) * n6);
    int32_t* vmin = (int32_t*)p; p += al(sizeof(int32_t) * nv);
    void* rtmp = p;
    k_check_tets<<<nblk(nt, T), T, 0, s>>>(d_tets, nt, nv, Xi, st);
    note_launch();
    cudaMemsetAsync(own, 0, sizeof(uint32_t) * nt, s);
    cudaMemsetAsync(adj, 0xff, sizeof(int32_t) * 4 * nt, s);
    int vb = 1;
    while ((1ll << vb) < nv) vb++;
    // faces
    k_face_keys<<<nblk(4 * nt, T), T, 0, s>>>(d_tets, nt, vb, k0, v0);
    note_launch();
    radix_sort_pairs(k0, v0, k1, v1, 4 * nt, 3 * vb, rtmp, &st->err, s);
    k_face_runs<<<nblk(4 * nt, T), T, 0, s>>>(k1, v1, 4 * nt, adj, own, st);
    note_launch();
    // edges
    k_edge_keys<<<nblk(n6, T), T, 0, s>>>(d_tets, nt, vb, k0, v0);
    note_launch();
    radix_sort_pairs(k0, v0, k1, v1, n6, 2 * vb, rtmp, &st->err, s);
    k_edge_runs<<<nblk(n6, T), T, 0, s>>>(k1, v1, n6, own);
    note_launch();
    // vertices
    k_fill_i32<<<nblk(nv, T), T, 0, s>>>(vmin, nv, 0x7fffffff);
    note_launch();
    k_vertex_min<<<nblk(4 * nt, T), T, 0, s>>>(d_tets, nt, nv, vmin);
    note_launch();
    k_vertex_own<<<nblk(nt, T), T, 0, s>>>(d_tets, nt, nv, vmin, own);
    note_launch();
}

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

// Mesh combinatorics by hashing: every tet inserts its 4 faces (sorted vertex
// triples) and 6 edges (sorted pairs) into open-addressing tables keyed by the
// packed vertex ids; per face the table keeps the (tet, face) indices of the
// (at most two) tets that hold it, per edge the lowest (tet, edge) index, per
// vertex the lowest tet.  A third tet on a face is a non-manifold error.  A
// second pass looks every entry up again: face adjacency and ownership by the
// lowest-numbered tet.  The results do not depend on the insertion order.
// A slot is 16 bytes, key and payload together, so an insertion or a lookup
// touches one 32-byte sector of the table (the probing and the atomics on the
// payload land on the same line).
struct MeshTables {
    uint64_t* ft;   // face slots: [key, (first index, second index)]
    uint64_t* et;   // edge slots: [key, (lowest index, unused)]
    uint32_t* vmin;   // lowest tet per vertex
    unsigned long long fmask, emask;
    int fshift, eshift;
    int vb;
};

constexpr uint32_t NONE32 = 0xffffffffu;

// Slot of `key` in a table of 16-byte slots (the key first), inserted if
// absent; -1 when the table is full.
__device__ __forceinline__ long long slot_insert(uint64_t* t, unsigned long long mask, int shift, uint64_t key) {
    unsigned long long h = hslot(key, shift);
    for (unsigned long long it = 0; it <= mask; it++) {
        const uint64_t k = t[2 * h];
        if (k == key) return (long long)h;
        if (k == HEMPTY) {
            const uint64_t old = atomicCAS((unsigned long long*)&t[2 * h], HEMPTY, key);
            if (old == HEMPTY || old == key) return (long long)h;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ long long slot_find(const uint64_t* t, unsigned long long mask, int shift, uint64_t key) {
    unsigned long long h = hslot(key, shift);
    for (unsigned long long it = 0; it <= mask; it++) {
        const uint64_t k = t[2 * h];
        if (k == key) return (long long)h;
        if (k == HEMPTY) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ void sort3(unsigned long long& a, unsigned long long& b, unsigned long long& c) {
    unsigned long long t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
}

// Face f of a tet is the triangle opposite local vertex f.
__device__ __forceinline__ uint64_t face_key(const int v[4], int f, int vb) {
    unsigned long long w[3];
    int n = 0;
#pragma unroll
    for (int c = 0; c < 4; c++)
        if (c != f) w[n++] = (unsigned)v[c];
    sort3(w[0], w[1], w[2]);
    return (w[0] << (2 * vb)) | (w[1] << vb) | w[2];
}

__device__ __forceinline__ uint64_t edge_key(const int v[4], int e, int vb) {
    const int ea = e < 3 ? 0 : (e < 5 ? 1 : 2);
    const int eb = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
    unsigned long long a = (unsigned)v[ea], b = (unsigned)v[eb];
    if (a > b) {
        const unsigned long long t = a;
        a = b;
        b = t;
    }
    return (a << vb) | b;
}

__device__ __forceinline__ bool load_tet_ids(const int32_t* __restrict__ T, long long t, long long nv, int v[4]) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        v[a] = T[4 * t + a];
        ok &= v[a] >= 0 && v[a] < nv;
    }
    return ok;
}

// Exact orientation (det[p1-p0, p2-p0, p3-p0] > 0 with 128-bit integers) and
// table insertion.
__global__ void k_mesh_insert(const int32_t* __restrict__ T, long long nt, long long nv,
                              const int32_t* __restrict__ Xi, MeshTables M, DevState* st) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int v[4];
    if (!load_tet_ids(T, t, nv, v)) {
        dev_fail(st, RPD_E_INVALID, CNT_INVALID);
        return;
    }
    const int3 p0 = ld_int3(Xi, v[0]), p1 = ld_int3(Xi, v[1]), p2 = ld_int3(Xi, v[2]), p3 = ld_int3(Xi, v[3]);
    const long long ax = p1.x - p0.x, ay = p1.y - p0.y, az = p1.z - p0.z;
    const long long bx = p2.x - p0.x, by = p2.y - p0.y, bz = p2.z - p0.z;
    const long long cx = p3.x - p0.x, cy = p3.y - p0.y, cz = p3.z - p0.z;
    const __int128 d = (__int128)ax * ((__int128)by * cz - (__int128)bz * cy) -
                       (__int128)ay * ((__int128)bx * cz - (__int128)bz * cx) +
                       (__int128)az * ((__int128)bx * cy - (__int128)by * cx);
    if (d <= 0) {
        dev_fail(st, RPD_E_INVALID, CNT_INVALID);
        return;
    }
#pragma unroll
    for (int a = 0; a < 4; a++) atomicMin(&M.vmin[v[a]], (uint32_t)t);
#pragma unroll
    for (int f = 0; f < 4; f++) {
        const long long h = slot_insert(M.ft, M.fmask, M.fshift, face_key(v, f, M.vb));
        if (h < 0) {
            dev_fail(st, RPD_E_OVERFLOW, CNT_CAPACITY);
            continue;
        }
        const uint32_t i = (uint32_t)(4 * t + f);
        uint32_t* ab = reinterpret_cast<uint32_t*>(&M.ft[2 * h + 1]);
        if (atomicCAS(&ab[0], NONE32, i) != NONE32 && atomicCAS(&ab[1], NONE32, i) != NONE32)
            dev_fail(st, RPD_E_NONMANIFOLD, CNT_NONMANIFOLD);   // a third tet on the face
    }
#pragma unroll
    for (int e = 0; e < 6; e++) {
        const long long h = slot_insert(M.et, M.emask, M.eshift, edge_key(v, e, M.vb));
        if (h < 0) {
            dev_fail(st, RPD_E_OVERFLOW, CNT_CAPACITY);
            continue;
        }
        atomicMin(reinterpret_cast<uint32_t*>(&M.et[2 * h + 1]), (uint32_t)(6 * t + e));
    }
}

// Adjacency (adj[4t+f] = tet across face f, or -1) and ownership bits:
// 0..3 vertices, 4..9 edges, 10..13 faces.
__global__ void k_mesh_finish(const int32_t* __restrict__ T, long long nt, long long nv, MeshTables M,
                              int32_t* __restrict__ adj, uint32_t* __restrict__ own, DevState* st) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int v[4];
    if (!load_tet_ids(T, t, nv, v)) {
        own[t] = 0;
#pragma unroll
        for (int f = 0; f < 4; f++) adj[4 * t + f] = -1;
        return;
    }
    uint32_t bits = 0;
#pragma unroll
    for (int a = 0; a < 4; a++)
        if (M.vmin[v[a]] == (uint32_t)t) bits |= 1u << a;
#pragma unroll
    for (int f = 0; f < 4; f++) {
        const uint32_t i = (uint32_t)(4 * t + f);
        int32_t nb = -1;
        const long long h = slot_find(M.ft, M.fmask, M.fshift, face_key(v, f, M.vb));
        if (h >= 0) {
            const uint64_t w = M.ft[2 * h + 1];
            const uint32_t a = (uint32_t)w, b = (uint32_t)(w >> 32);
            const uint32_t mn = min(a, b), mx = max(a, b);   // NONE32 sorts last
            if (mn == i) bits |= 1u << (10 + f);
            if (mx != NONE32) nb = (int32_t)((mn == i ? mx : mn) >> 2);
        }
        adj[4 * t + f] = nb;
    }
#pragma unroll
    for (int e = 0; e < 6; e++) {
        const long long h = slot_find(M.et, M.emask, M.eshift, edge_key(v, e, M.vb));
        if (h >= 0 && (uint32_t)M.et[2 * h + 1] == (uint32_t)(6 * t + e)) bits |= 1u << (4 + e);
    }
    own[t] = bits;
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

static int log2_cap(long long n) {
    int b = 4;
    while ((1ll << b) < n) b++;
    return b;
}

size_t prep_tmp_bytes(long long nt, long long nv) {
    const long long cf = 1ll << log2_cap(6 * nt), ce = 1ll << log2_cap(8 * nt);
    return al(2 * sizeof(uint64_t) * (cf + ce)) + al(sizeof(uint32_t) * nv);
}

void launch_prep_mesh(const int32_t* d_tets, long long nt, long long nv, const int32_t* Xi, int32_t* adj,
                      uint32_t* own, void* tmp, DevState* st, cudaStream_t s) {
    if (nt <= 0) return;
    const int T = 256;
    const int bf = log2_cap(6 * nt), be = log2_cap(8 * nt);
    const long long cf = 1ll << bf, ce = 1ll << be;
    char* p = (char*)tmp;
    MeshTables M;
    M.ft = (uint64_t*)p;
    M.et = M.ft + 2 * cf;
    p += al(2 * sizeof(uint64_t) * (cf + ce));
    M.vmin = (uint32_t*)p;
    M.fmask = (unsigned long long)(cf - 1);
    M.emask = (unsigned long long)(ce - 1);
    M.fshift = 64 - bf;
    M.eshift = 64 - be;
    int vb = 1;
    while ((1ll << vb) < nv) vb++;
    M.vb = vb;
    // every key empty, every payload NONE32
    cudaMemsetAsync(M.ft, 0xff, 2 * sizeof(uint64_t) * (cf + ce), s);
    cudaMemsetAsync(M.vmin, 0xff, sizeof(uint32_t) * nv, s);
    k_mesh_insert<<<nblk(nt, T), T, 0, s>>>(d_tets, nt, nv, Xi, M, st);
    note_launch();
    k_mesh_finish<<<nblk(nt, T), T, 0, s>>>(d_tets, nt, nv, M, adj, own, st);
    note_launch();
}

// Topology repair kernels: pin points of non-contractible restricted elements
// and sphere shrinking against the shape's boundary.
//
// Sec. 4.1.1: an element with beta0 > 1 gets a new sphere grown from a pin
// point on the surface of a component other than the one its sphere resides
// in; Sec. 4.1.2: an element with chi != 1 gets one grown from the surface
// triangle of the element furthest from its sphere.  Sec. 5.1: the new
// sphere is computed by sphere shrinking (the shrinking-ball algorithm of
// Ma et al. 2012): starting from a ball tangent to the surface at the pin p
// (centre p + r n, n the inward normal, r large), find the surface point q
// nearest to the centre; while q lies inside the ball, replace the ball by
// the one tangent at p that passes through q, of radius
//     r' = |p - q|^2 / (2 n.(q - p)),
// until the ball is empty; it then touches the surface at p and q.
//
// Surface = the boundary triangles of the tet mesh (tet faces without a
// neighbour); a pin is the centroid of such a triangle, its normal points
// into the tet.  Which component a piece belongs to is read from the
// union-find parents the finalisation left for that element kind.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <climits>

#include "internal.cuh"
#include "prim.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ void face_corners(int f, int& a, int& b, int& c) {
    a = f == 0 ? 1 : 0;
    b = f <= 1 ? 2 : 1;
    c = f <= 2 ? 3 : 2;
}

// ------------------------------------------------------- boundary triangles
__global__ void k_bnd_flag(const int32_t* __restrict__ adj, long long n4, uint8_t* __restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n4) flag[i] = adj[i] < 0 ? 1 : 0;
}

// Triangle k = (A, B, C) of boundary face 4t+f as 9 doubles (world units),
// ordered so that (B - A) x (C - A) points into the tet.
__global__ void k_bnd_fill(const int32_t* __restrict__ tets, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ Xi, long long nt, const int64_t* __restrict__ pos, double unit,
                           double* __restrict__ tri, int32_t* __restrict__ face_of) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * nt || adj[i] >= 0) return;
    const long long t = i >> 2;
    const int f = (int)(i & 3);
    int a, b, c;
    face_corners(f, a, b, c);
    const int3 A = ld_int3(Xi, tets[4 * t + a]), B = ld_int3(Xi, tets[4 * t + b]), C = ld_int3(Xi, tets[4 * t + c]);
    const int3 D = ld_int3(Xi, tets[4 * t + f]);
    // orientation of (B - A) x (C - A) against D - A, exact in 128 bits
    const long long ux = B.x - A.x, uy = B.y - A.y, uz = B.z - A.z;
    const long long vx = C.x - A.x, vy = C.y - A.y, vz = C.z - A.z;
    const long long wx = D.x - A.x, wy = D.y - A.y, wz = D.z - A.z;
    const __int128 det = (__int128)wx * ((__int128)uy * vz - (__int128)uz * vy) -
                         (__int128)wy * ((__int128)ux * vz - (__int128)uz * vx) +
                         (__int128)wz * ((__int128)ux * vy - (__int128)uy * vx);
    const int3 P1 = det > 0 ? B : C, P2 = det > 0 ? C : B;
    const long long k = pos[i];
    double* o = tri + 9 * k;
    o[0] = A.x * unit; o[1] = A.y * unit; o[2] = A.z * unit;
    o[3] = P1.x * unit; o[4] = P1.y * unit; o[5] = P1.z * unit;
    o[6] = P2.x * unit; o[7] = P2.y * unit; o[8] = P2.z * unit;
    face_of[k] = (int32_t)i;
}

// ----------------------------------------------------------------- pins
// Row of the element with this packed key (sorted key rows, binary search),
// or -1.
__device__ __forceinline__ long long find_row(const int32_t* __restrict__ keys, long long n, int kind, const int* q) {
    long long lo = 0, hi = n - 1;
    while (lo <= hi) {
        const long long mid = (lo + hi) >> 1;
        int cmp = 0;
        for (int k = 0; k < kind && cmp == 0; k++) {
            const int v = keys[mid * kind + k];
            cmp = v < q[k] ? -1 : (v > q[k] ? 1 : 0);
        }
        if (cmp == 0) return mid;
        if (cmp < 0) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

struct PinArgs {
    ClipArgs a;
    int kind;
    const int32_t* keys;      // [nkeys, kind] sorted
    const int32_t* beta;
    const int32_t* chi;
    long long nkeys;
    const int32_t* parent;    // union-find of the kind's nodes
    long long nmax;           // node capacity (pairs, or record capacity)
    const int64_t* fpos;      // failing elements' positions (scan of !flag)
    const uint8_t* flag;
    unsigned long long* anchor;   // per failing element: (tet << 32) | node
    unsigned long long* far2;     // per failing element: largest squared distance
    unsigned long long* best;     // per failing element: (tet << 2) | face
    int uf_limit;
    const uint8_t* used;          // [4 nt] boundary faces already grown from, or NULL
};

// Node n of the kind: its tet, its element's key, its link byte; false for
// an empty piece or a record past the count.
__device__ __forceinline__ bool node_of(const PinArgs& P, long long n, long long& t, int* key, unsigned& link) {
    const ClipArgs& a = P.a;
    if (P.kind == 1) {
        if (n >= P.nmax || a.pflag[n] != 1) return false;
        t = a.pair_tet[n];
        key[0] = a.cand[t * RPD_MAXC + (n - a.pair_off[t])];
        link = a.c_link[n];
        return true;
    }
    const int w = P.kind - 2;
    const long long cnt = (long long)a.rcount[w];
    if (n >= (cnt < P.nmax ? cnt : P.nmax)) return false;
    t = a.rtet[w][n];
    const uint64_t k = a.rkey[w][n];
    const uint64_t m = (1ull << a.key_bits) - 1;
    for (int z = 0; z < P.kind; z++) key[z] = (int)((k >> ((P.kind - 1 - z) * a.key_bits)) & m);
    link = a.rlink[w][n];
    return true;
}

// Failing-element index of node n, or -1.
__device__ __forceinline__ long long fail_of(const PinArgs& P, long long n, long long& t, int* key, unsigned& link) {
    if (!node_of(P, n, t, key, link)) return -1;
    const long long e = find_row(P.keys, P.nkeys, P.kind, key);
    if (e < 0 || P.flag[e]) return -1;
    return P.fpos[e];
}

__device__ __forceinline__ int uf_root(const int32_t* parent, int x, int limit) {
    for (int it = 0; it < limit; it++) {
        const int px = parent[x];
        if (px < 0) return x;
        x = px;
    }
    return -1;
}

// Tet faces without a neighbour that the element's piece in tet t touches,
// leaving out the faces already grown from (used[4t+f] != 0, if given).
__device__ __forceinline__ unsigned boundary_faces(const ClipArgs& a, long long t, unsigned link,
                                                   const uint8_t* used) {
    unsigned b = 0;
    for (int f = 0; f < 4; f++)
        if (((link >> (4 + f)) & 1) && a.adj[4 * t + f] < 0 && !(used && used[4 * t + f])) b |= 1u << f;
    return b;
}

// 3 x centroid of face f of tet t (grid units).
__device__ __forceinline__ void face_centroid3(const ClipArgs& a, long long t, int f, long long* g) {
    int i0, i1, i2;
    face_corners(f, i0, i1, i2);
    const int3 A = ld_int3(a.Xi, a.tets[4 * t + i0]), B = ld_int3(a.Xi, a.tets[4 * t + i1]),
               C = ld_int3(a.Xi, a.tets[4 * t + i2]);
    g[0] = (long long)A.x + B.x + C.x;
    g[1] = (long long)A.y + B.y + C.y;
    g[2] = (long long)A.z + B.z + C.z;
}

__global__ void k_pin_anchor(PinArgs P) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long t;
    int key[4];
    unsigned link;
    const long long f = fail_of(P, n, t, key, link);
    if (f < 0) return;
    atomicMin(&P.anchor[f], ((unsigned long long)t << 32) | (unsigned long long)n);
    // chi != 1 with one component: the boundary triangle furthest from the
    // element's (first) sphere
    const unsigned bf = boundary_faces(P.a, t, link, P.used);
    if (!bf) return;
    const long long e = find_row(P.keys, P.nkeys, P.kind, key);
    if (P.beta[e] > 1) return;
    const int3 c = ld_int3(P.a.Ci, key[0]);
    for (int q = 0; q < 4; q++) {
        if (!((bf >> q) & 1)) continue;
        long long g[3];
        face_centroid3(P.a, t, q, g);
        const long long dx = g[0] - 3ll * c.x, dy = g[1] - 3ll * c.y, dz = g[2] - 3ll * c.z;
        atomicMax(&P.far2[f], (unsigned long long)(dx * dx + dy * dy + dz * dz));
    }
}

__global__ void k_pin_pick(PinArgs P) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long t;
    int key[4];
    unsigned link;
    const long long f = fail_of(P, n, t, key, link);
    if (f < 0) return;
    const unsigned bf = boundary_faces(P.a, t, link, P.used);
    if (!bf) return;
    const long long e = find_row(P.keys, P.nkeys, P.kind, key);
    if (P.beta[e] > 1) {
        // a component other than the anchor's (the element's piece in the
        // lowest-numbered tet)
        const int an = (int)(P.anchor[f] & 0xffffffffu);
        const int r0 = uf_root(P.parent, an, P.uf_limit), r1 = uf_root(P.parent, (int)n, P.uf_limit);
        if (r0 < 0 || r1 < 0 || r0 == r1) return;
        const int q = __ffs(bf) - 1;
        atomicMin(&P.best[f], ((unsigned long long)t << 2) | (unsigned long long)q);
        return;
    }
    const int3 c = ld_int3(P.a.Ci, key[0]);
    for (int q = 0; q < 4; q++) {
        if (!((bf >> q) & 1)) continue;
        long long g[3];
        face_centroid3(P.a, t, q, g);
        const long long dx = g[0] - 3ll * c.x, dy = g[1] - 3ll * c.y, dz = g[2] - 3ll * c.z;
        if ((unsigned long long)(dx * dx + dy * dy + dz * dz) == P.far2[f])
            atomicMin(&P.best[f], ((unsigned long long)t << 2) | (unsigned long long)q);
    }
}

// Per element: key row, pin (face centroid), inward unit normal, face id
// 4t+f (-1 and NaN when the element touches no boundary triangle that
// qualifies).
__global__ void k_pin_emit(PinArgs P, int32_t* __restrict__ out_keys, double* __restrict__ pins,
                           double* __restrict__ normals, int32_t* __restrict__ faces) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.nkeys || P.flag[e]) return;
    const long long f = P.fpos[e];
    for (int k = 0; k < P.kind; k++) out_keys[f * P.kind + k] = P.keys[e * P.kind + k];
    const unsigned long long b = P.best[f];
    if (b == ~0ull) {
        for (int k = 0; k < 3; k++) pins[3 * f + k] = normals[3 * f + k] = nan("");
        faces[f] = -1;
        return;
    }
    const long long t = (long long)(b >> 2);
    const int q = (int)(b & 3);
    int i0, i1, i2;
    face_corners(q, i0, i1, i2);
    const int3 A = ld_int3(P.a.Xi, P.a.tets[4 * t + i0]), B = ld_int3(P.a.Xi, P.a.tets[4 * t + i1]),
               C = ld_int3(P.a.Xi, P.a.tets[4 * t + i2]), D = ld_int3(P.a.Xi, P.a.tets[4 * t + q]);
    const double u = P.a.unit;
    const double ux = (double)(B.x - A.x), uy = (double)(B.y - A.y), uz = (double)(B.z - A.z);
    const double vx = (double)(C.x - A.x), vy = (double)(C.y - A.y), vz = (double)(C.z - A.z);
    double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    const double side = nx * (D.x - A.x) + ny * (D.y - A.y) + nz * (D.z - A.z);
    const double s = (side < 0 ? -1.0 : 1.0) / sqrt(nx * nx + ny * ny + nz * nz);
    pins[3 * f + 0] = ((double)A.x + B.x + C.x) * u / 3.0;
    pins[3 * f + 1] = ((double)A.y + B.y + C.y) * u / 3.0;
    pins[3 * f + 2] = ((double)A.z + B.z + C.z) * u / 3.0;
    normals[3 * f + 0] = nx * s;
    normals[3 * f + 1] = ny * s;
    normals[3 * f + 2] = nz * s;
    faces[f] = (int32_t)(4 * t + q);
}

__global__ void k_not_flag(const uint8_t* __restrict__ flag, long long n, uint8_t* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = flag[i] ? 0 : 1;
}

// Bounding ball of each boundary triangle for the shrinking's cull: the
// centroid rounded to FP32, and a radius, measured in FP64 from that rounded
// centre to the corners, rounded up to FP32 with a 2^-20 relative margin.
__global__ void k_bnd_spheres(const double* __restrict__ tri, long long n, float4* __restrict__ bs) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* T = tri + 9 * i;
    float g[3];
    for (int k = 0; k < 3; k++) g[k] = (float)((T[k] + T[3 + k] + T[6 + k]) / 3.0);
    double r = 0.0;
    for (int v = 0; v < 3; v++) {
        double d2 = 0.0;
        for (int k = 0; k < 3; k++) {
            const double d = T[3 * v + k] - (double)g[k];
            d2 += d * d;
        }
        r = fmax(r, sqrt(d2));
    }
    bs[i] = make_float4(g[0], g[1], g[2], __double2float_ru(r * (1.0 + 0x1p-20)));
}

// ------------------------------------------------------------ shrinking
// Nearest point q to x on triangle (A, B, C).  With e1 = B - A, e2 = C - A
// the projection of x onto the triangle's plane is A + s e1 + t e2, where
// (s, t) solves the 2x2 normal equations; when s, t >= 0 and s + t <= 1 that
// is the answer, otherwise the nearest point lies on the boundary and is the
// nearest of the three edges' clamped projections.
__device__ __forceinline__ double seg_nearest(const double* P, const double* Q, const double* x, double* q) {
    double pq[3], px[3];
    for (int k = 0; k < 3; k++) {
        pq[k] = Q[k] - P[k];
        px[k] = x[k] - P[k];
    }
    const double l2 = pq[0] * pq[0] + pq[1] * pq[1] + pq[2] * pq[2];
    double u = l2 > 0 ? (px[0] * pq[0] + px[1] * pq[1] + px[2] * pq[2]) / l2 : 0.0;
    u = u < 0 ? 0 : (u > 1 ? 1 : u);
    double d = 0;
    for (int k = 0; k < 3; k++) {
        q[k] = P[k] + u * pq[k];
        d += (x[k] - q[k]) * (x[k] - q[k]);
    }
    return d;
}

__device__ __forceinline__ void nearest_on_triangle(const double* T, const double* x, double* q) {
    const double* A = T;
    const double* B = T + 3;
    const double* C = T + 6;
    double e1[3], e2[3], d[3];
    for (int k = 0; k < 3; k++) {
        e1[k] = B[k] - A[k];
        e2[k] = C[k] - A[k];
        d[k] = x[k] - A[k];
    }
    const double a11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
    const double a12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
    const double a22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
    const double b1 = e1[0] * d[0] + e1[1] * d[1] + e1[2] * d[2];
    const double b2 = e2[0] * d[0] + e2[1] * d[1] + e2[2] * d[2];
    const double det = a11 * a22 - a12 * a12;
    if (det > 0) {
        const double s = (b1 * a22 - b2 * a12) / det, t = (b2 * a11 - b1 * a12) / det;
        if (s >= 0 && t >= 0 && s + t <= 1) {
            for (int k = 0; k < 3; k++) q[k] = A[k] + s * e1[k] + t * e2[k];
            return;
        }
    }
    double q1[3], q2[3];
    double best = seg_nearest(A, B, x, q);
    const double d2 = seg_nearest(B, C, x, q1);
    if (d2 < best) {
        best = d2;
        for (int k = 0; k < 3; k++) q[k] = q1[k];
    }
    if (seg_nearest(C, A, x, q2) < best)
        for (int k = 0; k < 3; k++) q[k] = q2[k];
}

constexpr int SHRINK_THREADS = 256;
constexpr int SHRINK_ITERS = 100;
constexpr int SHRINK_CLUSTER = 8;   // CTAs per pin (a portable cluster size)

// (distance, triangle) pairs ordered by distance, then by the lower index; a
// pair with no triangle (-1) loses every tie.
__device__ __forceinline__ bool closer(double d, long long k, double bd, long long bk) {
    return d < bd || (d == bd && k >= 0 && (bk < 0 || k < bk));
}

// Sphere shrinking against all boundary triangles except the pin's own, one
// thread-block cluster of SHRINK_CLUSTER CTAs per pin.  Each CTA scans one
// contiguous part of the triangles for the one nearest to the current centre;
// the parts' results meet through distributed shared memory after a cluster
// barrier, and every CTA takes the same (distance, lowest index) minimum over
// them in rank order, so all CTAs follow the same radii and leave the loop
// together.  The minimum does not depend on how the triangles are split, so
// the result equals that of a single block scanning them all.
//
// Cull: a triangle whose bounding ball lies farther from the centre than the
// current radius r cannot be the nearest one, nor tie with it: the nearest
// one of a non-empty ball is within r, and an empty ball ends the shrinking
// whichever triangle is nearest.  The test runs in FP32 on the rounded centre
// with margins (2^-18 of the distance and 3 x 2^-18 of the centre's largest
// coordinate) far above the FP32 rounding of the test, so it never culls a
// triangle within r; only the triangles left are tested in FP64, and the
// result is that of testing them all.  Output centre and radius (NaN for a
// pin row without a face).
__global__ void __cluster_dims__(SHRINK_CLUSTER, 1, 1) __launch_bounds__(SHRINK_THREADS)
    k_shrink(const double* __restrict__ tri, const float4* __restrict__ bs, long long ntri,
             const int32_t* __restrict__ face_of, const double* __restrict__ pins, const double* __restrict__ normals, const int32_t* __restrict__ faces,
             double r0, const double* __restrict__ r_start, double* __restrict__ centres, double* __restrict__ radii,
             int32_t* __restrict__ iters, int32_t* __restrict__ restarted) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ double sd[SHRINK_THREADS / 32];
    __shared__ long long si[SHRINK_THREADS / 32];
    __shared__ double part_d[2];        // this CTA's nearest triangle, by iteration parity
    __shared__ long long part_k[2];
    __shared__ double sr;
    __shared__ int sdone, swarm;
    const unsigned rank = cluster.block_rank();
    const long long j = blockIdx.x / SHRINK_CLUSTER;   // the cluster's pin (uniform over the cluster)
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int own = faces[j];
    if (own < 0) {   // every CTA of the cluster leaves here, before any cluster barrier
        if (rank == 0 && tid == 0) {
            for (int k = 0; k < 3; k++) centres[3 * j + k] = nan("");
            radii[j] = nan("");
            iters[j] = 0;
            if (restarted) restarted[j] = 0;
        }
        return;
    }
    const long long per = (ntri + SHRINK_CLUSTER - 1) / SHRINK_CLUSTER;
    const long long lo = per * rank, hi = lo + per < ntri ? lo + per : ntri;
    const double p[3] = {pins[3 * j], pins[3 * j + 1], pins[3 * j + 2]};
    const double n[3] = {normals[3 * j], normals[3 * j + 1], normals[3 * j + 2]};
    int rs_flag = 0;
    if (tid == 0) {
        // a proposed first radius (0 < r < r0) replaces r0; the first ball
        // must then contain a surface point, otherwise it may lie below the
        // fixed point and the shrinking starts over from r0
        const double rs = r_start ? r_start[j] : 0.0;
        swarm = rs > 0.0 && rs < r0;
        sr = swarm ? rs : r0;
        sdone = 0;
    }
    __syncthreads();
    int it = 0;
    for (; it < SHRINK_ITERS; it++) {
        const double r = sr;
        const double c[3] = {p[0] + r * n[0], p[1] + r * n[1], p[2] + r * n[2]};
        const float cf[3] = {(float)c[0], (float)c[1], (float)c[2]};
        const float cslack = 3.0f * 0x1p-18f * fmaxf(fabsf(cf[0]), fmaxf(fabsf(cf[1]), fabsf(cf[2])));
        const float uf = __double2float_ru(r * (1.0 + 0x1p-20));
        double bd = INFINITY;
        long long bi = -1;
        for (long long k = lo + tid; k < hi; k += SHRINK_THREADS) {
            const float4 b = bs[k];
            const float dx = cf[0] - b.x, dy = cf[1] - b.y, dz = cf[2] - b.z;
            const float lb = sqrtf(dx * dx + dy * dy + dz * dz) * (1.0f - 0x1p-18f) - b.w - cslack;
            if (lb > uf) continue;   // the whole triangle lies farther than r
            if (face_of[k] == own) continue;
            double q[3];
            nearest_on_triangle(tri + 9 * k, c, q);
            const double d = (q[0] - c[0]) * (q[0] - c[0]) + (q[1] - c[1]) * (q[1] - c[1]) + (q[2] - c[2]) * (q[2] - c[2]);
            if (d < bd) {
                bd = d;
                bi = k;
            }
        }
        for (int off = 16; off; off >>= 1) {
            const double od = __shfl_down_sync(0xffffffffu, bd, off);
            const long long oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (closer(od, oi, bd, bi)) {
                bd = od;
                bi = oi;
            }
        }
        if (lane == 0) {
            sd[w] = bd;
            si[w] = bi;
        }
        __syncthreads();
        const int par = it & 1;
        if (tid == 0) {
            double d = INFINITY;
            long long k = -1;
            for (int z = 0; z < SHRINK_THREADS / 32; z++)
                if (closer(sd[z], si[z], d, k)) {
                    d = sd[z];
                    k = si[z];
                }
            part_d[par] = d;
            part_k[par] = k;
        }
        // the parts of this iteration are visible cluster-wide after the
        // barrier; a part slot is written again two iterations later, after
        // the next barrier, which every CTA reaches only once it has read it
        cluster.sync();
        if (tid == 0) {
            double d = INFINITY;
            long long k = -1;
            for (unsigned z = 0; z < SHRINK_CLUSTER; z++) {
                const double* pd = cluster.map_shared_rank(&part_d[par], z);
                const long long* pk = cluster.map_shared_rank(&part_k[par], z);
                const double od = *pd;
                const long long ok = *pk;
                if (closer(od, ok, d, k)) {
                    d = od;
                    k = ok;
                }
            }
            // empty ball (within rounding): done, unless it is a proposed one
            if (k < 0 || sqrt(d) >= r * (1.0 - 1e-12)) {
                if (swarm) {
                    sr = r0;
                    rs_flag = 1;
                } else {
                    sdone = 1;
                }
            } else {
                double q[3];
                nearest_on_triangle(tri + 9 * k, c, q);
                const double pq[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
                const double dn = pq[0] * n[0] + pq[1] * n[1] + pq[2] * n[2];
                const double rn = (pq[0] * pq[0] + pq[1] * pq[1] + pq[2] * pq[2]) / (2.0 * dn);
                if (!(dn > 0) || !(rn < r)) sdone = 1;   // no progress possible
                else sr = rn;
            }
            swarm = 0;
        }
        __syncthreads();
        if (sdone) break;
    }
    // peers may still be reading this CTA's parts: leave together
    cluster.sync();
    if (rank == 0 && tid == 0) {
        const double r = sr;
        for (int k = 0; k < 3; k++) centres[3 * j + k] = p[k] + r * n[k];
        radii[j] = r;
        iters[j] = it + 1;
        if (restarted) restarted[j] = rs_flag;
    }
}

__global__ void k_sphere_out(const int32_t* __restrict__ Ci, const long long* __restrict__ W, long long ns, double unit,
                             double* __restrict__ c, double* __restrict__ r) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    for (int k = 0; k < 3; k++) c[3 * i + k] = (double)Ci[3 * i + k] * unit;
    r[i] = sqrt((double)W[i]) * unit;   // W = (integer radius)^2 < 2^46: the root is exact
}

__global__ void k_fixed_to_world(const long long* __restrict__ in, double* __restrict__ out, long long n, double scale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i] * scale;
}

// Records of restricted power edges: add each segment's fixed-point length to
// its key's row (64-bit integer sums: the result does not depend on order).
__global__ void k_edge_len_sum(ClipArgs a, long long nmax, const int32_t* __restrict__ keys, long long nkeys,
                               unsigned long long* __restrict__ len) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cnt = (long long)a.rcount[1];
    if (r >= (cnt < nmax ? cnt : nmax)) return;
    const uint64_t k = a.rkey[1][r];
    const uint64_t m = (1ull << a.key_bits) - 1;
    int key[3];
    for (int z = 0; z < 3; z++) key[z] = (int)((k >> ((2 - z) * a.key_bits)) & m);
    const long long e = find_row(keys, nkeys, 3, key);
    if (e >= 0) atomicAdd(&len[e], (unsigned long long)a.elen[r]);
}

// Surface samples: centroid of each boundary triangle and its unit normal
// into the shape ((B - A) x (C - A) points into the tet, see k_bnd_fill).
__global__ void k_surface_samples(const double* __restrict__ tri, const int32_t* __restrict__ face_of, long long nb,
                                  double* __restrict__ pts, double* __restrict__ nrm, int32_t* __restrict__ faces) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const double* T = tri + 9 * k;
    const double ux = T[3] - T[0], uy = T[4] - T[1], uz = T[5] - T[2];
    const double vx = T[6] - T[0], vy = T[7] - T[1], vz = T[8] - T[2];
    const double nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    const double inv = 1.0 / sqrt(nx * nx + ny * ny + nz * nz);
    for (int z = 0; z < 3; z++) pts[3 * k + z] = (T[z] + T[3 + z] + T[6 + z]) / 3.0;
    nrm[3 * k] = nx * inv;
    nrm[3 * k + 1] = ny * inv;
    nrm[3 * k + 2] = nz * inv;
    faces[k] = face_of[k];
}

__global__ void k_mark_faces(const int32_t* __restrict__ faces, long long n, uint8_t* __restrict__ used,
                             long long n4) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && faces[i] >= 0 && faces[i] < n4) used[faces[i]] = 1;
}

}  // namespace

void launch_edge_length_sum(const ClipArgs& a, long long nmax, const int32_t* keys, long long nkeys, long long* len,
                            cudaStream_t s) {
    cudaMemsetAsync(len, 0, sizeof(long long) * (nkeys > 0 ? nkeys : 1), s);
    if (nmax <= 0 || nkeys <= 0 || !a.elen) return;
    k_edge_len_sum<<<nblk(nmax, 256), 256, 0, s>>>(a, nmax, keys, nkeys, (unsigned long long*)len);
    note_launch();
}

void launch_surface_samples(const double* tri, const int32_t* face_of, long long nb, double* pts, double* nrm,
                            int32_t* faces, cudaStream_t s) {
    if (nb <= 0) return;
    k_surface_samples<<<nblk(nb, 256), 256, 0, s>>>(tri, face_of, nb, pts, nrm, faces);
    note_launch();
}

void launch_mark_faces(const int32_t* faces, long long n, uint8_t* used, long long n4, cudaStream_t s) {
    if (n <= 0) return;
    k_mark_faces<<<nblk(n, 256), 256, 0, s>>>(faces, n, used, n4);
    note_launch();
}

void launch_fixed_to_world(const long long* in, double* out, long long n, double scale, cudaStream_t s) {
    if (n <= 0) return;
    k_fixed_to_world<<<nblk(n, 256), 256, 0, s>>>(in, out, n, scale);
    note_launch();
}

void launch_sphere_out(const int32_t* Ci, const long long* W, long long ns, double unit, double* c, double* r,
                       cudaStream_t s) {
    if (ns <= 0) return;
    k_sphere_out<<<nblk(ns, 256), 256, 0, s>>>(Ci, W, ns, unit, c, r);
    note_launch();
}

size_t boundary_tmp_bytes(long long nt) { return ((4 * nt + 255) & ~255ll) + scan_tmp_bytes(4 * nt) + 256; }

// Boundary flags and positions: pos[4 nt] = number of boundary triangles.
void launch_boundary_count(const int32_t* adj, long long nt, int64_t* pos, void* tmp, cudaStream_t s) {
    uint8_t* flag = (uint8_t*)tmp;
    void* stmp = (char*)tmp + ((4 * nt + 255) & ~255ll);
    if (nt > 0) {
        k_bnd_flag<<<nblk(4 * nt, 256), 256, 0, s>>>(adj, 4 * nt, flag);
        note_launch();
    }
    scan_excl(flag, pos, 4 * nt, stmp, s);
}

void launch_boundary_fill(const int32_t* tets, const int32_t* adj, const int32_t* Xi, long long nt, const int64_t* pos,
                          double unit, double* tri, int32_t* face_of, cudaStream_t s) {
    if (nt == 0) return;
    k_bnd_fill<<<nblk(4 * nt, 256), 256, 0, s>>>(tets, adj, Xi, nt, pos, unit, tri, face_of);
    note_launch();
}

size_t pins_tmp_bytes(long long nkeys) {
    const long long n = nkeys + 1;
    return 3 * ((8 * n + 255) & ~255ll) + ((n + 255) & ~255ll) + ((8 * n + 255) & ~255ll) + scan_tmp_bytes(n);
}

// Failing elements of one kind: fpos (scan of !flag); fpos[nkeys] = their count.
void launch_pins_count(const uint8_t* flag, long long nkeys, void* tmp, cudaStream_t s) {
    const long long n = nkeys + 1;
    char* p = (char*)tmp + 3 * ((8 * n + 255) & ~255ll);
    uint8_t* nf = (uint8_t*)p;
    p += (n + 255) & ~255ll;
    int64_t* fpos = (int64_t*)p;
    p += (8 * n + 255) & ~255ll;
    if (nkeys > 0) {
        k_not_flag<<<nblk(nkeys, 256), 256, 0, s>>>(flag, nkeys, nf);
        note_launch();
    }
    scan_excl(nf, fpos, nkeys, p, s);
}

const int64_t* pins_fpos(const void* tmp, long long nkeys) {
    const long long n = nkeys + 1;
    return (const int64_t*)((const char*)tmp + 3 * ((8 * n + 255) & ~255ll) + ((n + 255) & ~255ll));
}

void launch_pins(const ClipArgs& a, int kind, const int32_t* keys, const int32_t* beta, const int32_t* chi,
                 const uint8_t* flag, long long nkeys, long long nfail, const int32_t* parent, long long nmax,
                 int uf_limit, const uint8_t* used, void* tmp, int32_t* out_keys, double* pins, double* normals,
                 int32_t* faces, cudaStream_t s) {
    const long long n = nkeys + 1;
    PinArgs P;
    P.a = a;
    P.kind = kind;
    P.keys = keys;
    P.beta = beta;
    P.chi = chi;
    P.nkeys = nkeys;
    P.parent = parent;
    P.nmax = nmax;
    P.flag = flag;
    P.fpos = pins_fpos(tmp, nkeys);
    P.anchor = (unsigned long long*)tmp;
    P.far2 = (unsigned long long*)((char*)tmp + ((8 * n + 255) & ~255ll));
    P.best = (unsigned long long*)((char*)tmp + 2 * ((8 * n + 255) & ~255ll));
    P.uf_limit = uf_limit;
    P.used = used;
    if (nfail <= 0) return;
    cudaMemsetAsync(P.anchor, 0xff, 8 * nfail, s);
    cudaMemsetAsync(P.far2, 0, 8 * nfail, s);
    cudaMemsetAsync(P.best, 0xff, 8 * nfail, s);
    if (nmax > 0) {
        k_pin_anchor<<<nblk(nmax, 256), 256, 0, s>>>(P);
        note_launch();
        k_pin_pick<<<nblk(nmax, 256), 256, 0, s>>>(P);
        note_launch();
    }
    k_pin_emit<<<nblk(nkeys, 256), 256, 0, s>>>(P, out_keys, pins, normals, faces);
    note_launch();
}

void launch_boundary_spheres(const double* tri, long long n, float4* bs, cudaStream_t s) {
    if (n <= 0) return;
    k_bnd_spheres<<<nblk(n, 256), 256, 0, s>>>(tri, n, bs);
    note_launch();
}

void launch_shrink(const double* tri, const float4* bs, long long ntri, const int32_t* face_of, const double* pins,
                   const double* normals, const int32_t* faces, long long n, double r0, const double* r_start,
                   double* centres, double* radii, int32_t* iters, int32_t* restarted, cudaStream_t s) {
    // one cluster per pin, in launches of at most 2^24 pins (grid x < 2^31)
    for (long long b = 0; b < n; b += (1ll << 24)) {
        const long long m = n - b < (1ll << 24) ? n - b : (1ll << 24);
        k_shrink<<<(unsigned)(m * SHRINK_CLUSTER), SHRINK_THREADS, 0, s>>>(
            tri, bs, ntri, face_of, pins + 3 * b, normals + 3 * b, faces + b, r0, r_start ? r_start + b : nullptr,
            centres + 3 * b, radii + b, iters + b, restarted ? restarted + b : nullptr);
        note_launch();
    }
}

// ----------------------------------------------------- proposer features
// Features of a pin for the learned radius proposer: its position mapped to
// [-1, 1]^3 by the mesh's bounding box (centre bc, half of the longest side
// bh), its unit inward normal, and sin / cos of pi 2^o u for octaves o = 0..3
// of each mapped coordinate u.  With radii, also the regression target
// log2(r / diag), diag the box's diagonal.
__global__ void k_pin_features(const double* __restrict__ pins, const double* __restrict__ normals,
                               const double* __restrict__ radii, long long n, double bcx, double bcy, double bcz,
                               double bh, double diag, float* __restrict__ x, float* __restrict__ t) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float* f = x + j * RPD_PIN_FEATURES;
    const double bc[3] = {bcx, bcy, bcz};
    float u[3];
    for (int a = 0; a < 3; a++) {
        u[a] = (float)((pins[3 * j + a] - bc[a]) / bh);
        f[a] = u[a];
        f[3 + a] = (float)normals[3 * j + a];
    }
    for (int o = 0; o < 4; o++)
        for (int a = 0; a < 3; a++) {
            float sv, cv;
            sincospif(u[a] * (float)(1 << o), &sv, &cv);
            f[6 + 6 * o + 2 * a] = sv;
            f[6 + 6 * o + 2 * a + 1] = cv;
        }
    if (radii && t) t[j] = (float)log2(radii[j] / diag);
}

// Proposed first radius of the shrinking from the network's output y:
// margin * diag * 2^y (0 for a non-finite y: the plain start).
__global__ void k_radius_start(const float* __restrict__ y, long long n, double diag, double margin,
                               double* __restrict__ rs) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double v = (double)y[j];
    rs[j] = isfinite(v) ? margin * diag * exp2(fmin(fmax(v, -60.0), 4.0)) : 0.0;
}

// Bounding box of the grid vertices: lo in b[0..2], hi in b[3..5] (b starts
// at INT_MAX / INT_MIN).
__global__ void k_bbox(const int32_t* __restrict__ X, long long nv, int* __restrict__ b) {
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; a++) {
            lo[a] = min(lo[a], X[3 * i + a]);
            hi[a] = max(hi[a], X[3 * i + a]);
        }
    for (int a = 0; a < 3; a++) {
        for (int off = 16; off; off >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&b[a], lo[a]);
            atomicMax(&b[3 + a], hi[a]);
        }
    }
}

void launch_pin_features(const double* pins, const double* normals, const double* radii, long long n,
                         const double* bc, double bh, double diag, float* x, float* t, cudaStream_t s) {
    if (n <= 0) return;
    k_pin_features<<<nblk(n, 256), 256, 0, s>>>(pins, normals, radii, n, bc[0], bc[1], bc[2], bh, diag, x, t);
    note_launch();
}

void launch_radius_start(const float* y, long long n, double diag, double margin, double* rs, cudaStream_t s) {
    if (n <= 0) return;
    k_radius_start<<<nblk(n, 256), 256, 0, s>>>(y, n, diag, margin, rs);
    note_launch();
}

void launch_bbox(const int32_t* X, long long nv, int* b, cudaStream_t s) {
    const int init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    cudaMemcpyAsync(b, init, sizeof(init), cudaMemcpyHostToDevice, s);
    k_bbox<<<(unsigned)std::max<long long>(1, std::min<long long>(nblk(nv, 256), 152 * 4)), 256, 0, s>>>(X, nv, b);
    note_launch();
}

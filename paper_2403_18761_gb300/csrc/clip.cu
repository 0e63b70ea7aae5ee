// A3-A4: Tet-Cell clipping of every candidate (tet, sphere) pair with the
// fractional Euler characteristic emitted on the fly.
//
// Sec. 5.2 (Tet-Cell): the piece P(t,i) = t cap cell_i is computed for every
// (tet, sphere) pair independently, by clipping t with the radical
// half-spaces {pd(x,i) <= pd(x,k)} of the other spheres k (Sec. 4.1.2).  The
// polytope is stored as in the paper's data structure (Sec. 5.2): one integer
// triplet of plane ids per vertex.  Triplets are oriented so that they form a
// closed triangulated surface in the dual; each vertex also keeps its three
// dual neighbours (the vertex across each of its edges), so a clip removes
// the outside vertices, walks the boundary of the removed region once and
// closes it with a fan of new vertices on the new plane, all in O(V).
//
// Geometry lives in the barycentric coordinates of the tet.  Plane ids 0..3
// are the tet faces (face f opposite corner f, i.e. beta_f = 0); id 4+s is the
// radical plane of the s-th candidate sphere, given by its exact values at the
// corners F_s[c] = pd(X_c, i) - pd(X_c, s) (|F| < 2^47, exact int64).  A
// vertex on bisector rows J and tet faces A has homogeneous barycentric
// coordinates C = cofactor vector of the rows J over the free columns (not in
// A); its side of plane u is sign(F_u . C) once C is oriented so that
// sum(C) > 0.  The first stage evaluates this in FP32 (or FP64) on rows scaled
// by powers of two, with a forward error bound; an uncertified sign is
// recomputed in FP64 and then in exact 256-bit integers.
//
// Fractional Euler (Sec. 4.1.2, Eq. 7): each element of the piece inherits
// the weight of the mesh face that carries it (tet corner / edge / face /
// interior), here as ownership bits (the lowest tet containing a mesh face
// counts it once).  Per piece the kernel emits the RPC contribution
// V - E + F - C, an RPF record per radical face (i < j), an RPE record per
// radical edge (i < j, k), an RPV record per radical vertex, and the tet
// faces each element crosses (component links, Sec. 4.1.1).
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <type_traits>

#include "dfloat.cuh"
#include "exact.cuh"
#include "internal.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename Real>
struct PrecTraits;
template <>
struct PrecTraits<float> {
    static constexpr int VW = 7;   // words per slot: trip, nb, C0..C3, bound
    __device__ static float u() { return 0x1p-24f; }
};
template <>
struct PrecTraits<double> {
    static constexpr int VW = 12;  // trip, nb, C0..C3 (8 words), bound (2 words)
    __device__ static double u() { return 0x1p-53; }
};

constexpr uint32_t DEAD = 0xff000000u;   // flag in the triplet word of a free slot

// ---------------------------------------------------------------- lane state
struct Lane {
    long long t;
    int i;          // sphere index of this piece
    int si;         // its slot among the tet's candidates
    int n;          // number of candidates of the tet
    const int32_t* cand;
    int3 X[4];
    long long di[4];
    uint32_t own;
};

__device__ __forceinline__ void row_i64(const Lane& L, const int32_t* __restrict__ Ci, const long long* __restrict__ W,
                                        int slot, long long F[4]) {
    int s = L.cand[slot];
    int3 c = ld_int3(Ci, s);
    long long w = W[s];
#pragma unroll
    for (int k = 0; k < 4; k++) F[k] = L.di[k] - pd_exact(L.X[k], c, w);
}

// Scale a row by a power of two so that every |entry| <= 1, with an absolute
// error below the unit roundoff u of Real per entry.
template <typename Real>
__device__ __forceinline__ void scale_row(const long long F[4], Real R[4]);

template <>
__device__ __forceinline__ void scale_row<double>(const long long F[4], double R[4]) {
    unsigned long long m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) m = max(m, (unsigned long long)(F[k] < 0 ? -F[k] : F[k]));
    int e = m ? 64 - __clzll(m) : 0;                  // |F| < 2^e <= 2^48: exact in FP64
    double sc = __longlong_as_double((long long)(1023 - e) << 52);
#pragma unroll
    for (int k = 0; k < 4; k++) R[k] = (double)F[k] * sc;
}

// FP32 without FP64 or 64-bit conversions: drop the low e-24 bits with an
// arithmetic shift (floor, error < 2^(e-24)), convert the 24-bit integer
// exactly, scale by 2^-24 (exact); the result differs from F 2^-e by < 2^-24.
template <>
__device__ __forceinline__ void scale_row<float>(const long long F[4], float R[4]) {
    unsigned long long m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) m = max(m, (unsigned long long)(F[k] < 0 ? -F[k] : F[k]));
    int e = m ? 64 - __clzll(m) : 0;
    if (e <= 24) {
        float sc = __int_as_float((127 - e) << 23);
#pragma unroll
        for (int k = 0; k < 4; k++) R[k] = __int2float_rn((int)F[k]) * sc;
    } else {
        int sh = e - 24;
#pragma unroll
        for (int k = 0; k < 4; k++) R[k] = __int2float_rn((int)(F[k] >> sh)) * 0x1p-24f;
    }
}

// Triplet word: plane ids in bytes 0..2 (byte 3 = 0xff marks a free slot).
// Neighbour word: byte k = slot across dual edge trip[k] -> trip[k+1].
__device__ __forceinline__ int tb(uint32_t tw, int k) { return (tw >> (8 * k)) & 0xff; }
__device__ __forceinline__ uint32_t pack3(int a, int b, int c) { return (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)c << 16); }
__device__ __forceinline__ bool is_dead(uint32_t tw) { return (tw & DEAD) == DEAD; }

// Register-friendly access to 4-vectors with a run-time index (selects
// instead of local-memory indexing).
template <typename T>
__device__ __forceinline__ T get4(const T v[4], int i) {
    return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}
template <typename T>
__device__ __forceinline__ void set4(T v[4], int i, T x) {
    v[0] = i == 0 ? x : v[0];
    v[1] = i == 1 ? x : v[1];
    v[2] = i == 2 ? x : v[2];
    v[3] = i == 3 ? x : v[3];
}

// Free columns (ascending) and bisector planes of a triplet; returns m.
__device__ __forceinline__ int split_planes(int a, int b, int c, int* fc, int* bis) {
    const unsigned fmask = (a < 4 ? 1u << a : 0u) | (b < 4 ? 1u << b : 0u) | (c < 4 ? 1u << c : 0u);
    const int m = (a >= 4) + (b >= 4) + (c >= 4);
    // bisectors in (a, b, c) order
    bis[0] = a >= 4 ? a : (b >= 4 ? b : c);
    bis[1] = (a >= 4 && b >= 4) ? b : c;
    bis[2] = c;
    unsigned fr = (~fmask) & 15u;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        fc[k] = fr ? __ffs(fr) - 1 : 3;
        fr &= fr - 1;
    }
    return m;
}

// Cofactor vector (over the free columns, scattered to 4 entries) of m scaled
// rows, in floating point.
template <typename Real>
__device__ __forceinline__ void cof_real(int m, const Real (*R)[4], const int* fc, Real C[4]) {
    C[0] = C[1] = C[2] = C[3] = (Real)0;
    if (m == 1) {
        set4(C, fc[0], get4(R[0], fc[1]));
        set4(C, fc[1], -get4(R[0], fc[0]));
    } else if (m == 2) {
        const Real x0 = get4(R[0], fc[0]), x1 = get4(R[0], fc[1]), x2 = get4(R[0], fc[2]);
        const Real y0 = get4(R[1], fc[0]), y1 = get4(R[1], fc[1]), y2 = get4(R[1], fc[2]);
        set4(C, fc[0], fma(x1, y2, -(x2 * y1)));
        set4(C, fc[1], fma(x2, y0, -(x0 * y2)));
        set4(C, fc[2], fma(x0, y1, -(x1 * y0)));
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int c0 = k == 0 ? 1 : 0, c1 = k <= 1 ? 2 : 1, c2 = k <= 2 ? 3 : 2;
            Real m0 = fma(R[1][c1], R[2][c2], -(R[1][c2] * R[2][c1]));
            Real m1 = fma(R[1][c0], R[2][c2], -(R[1][c2] * R[2][c0]));
            Real m2 = fma(R[1][c0], R[2][c1], -(R[1][c1] * R[2][c0]));
            Real d = fma(R[0][c0], m0, fma(-R[0][c1], m1, R[0][c2] * m2));
            C[k] = (k & 1) ? -d : d;
        }
    }
}

// Absolute error bound of each cofactor entry for rows with |entry| <= 1.
template <typename Real>
__device__ __forceinline__ Real cof_err(int m) {
    const Real u = PrecTraits<Real>::u();
    return m == 1 ? 2 * u : (m == 2 ? 16 * u : 96 * u);
}

// Bound on |computed F.C - exact| for a scaled row F (|F| <= 1).
template <typename Real>
__device__ __forceinline__ Real dot_bound(int m, const Real C[4]) {
    const Real u = PrecTraits<Real>::u();
    Real sa = fabs(C[0]) + fabs(C[1]) + fabs(C[2]) + fabs(C[3]);
    return ((Real)(m + 1) * cof_err<Real>(m) + 6 * u * sa) * (1 + 8 * u);
}

// ------------------------------------------------------------- slow paths
struct Slow {
    const int32_t* Ci;
    const long long* W;
    DevState* st;
};

struct Row4 {
    long long v[4];
};

// Exact-or-FP64 sign of (F_u . C) * sign(sum C) for the vertex on planes
// (a,b,c); has_u == false asks for sign(sum C) alone.  Returns 0 only when
// the exact value is zero (degenerate input).  Arguments are passed by value
// so that the caller's lane state stays in registers.
__device__ __noinline__ int slow_sign_impl(Lane L, Slow S, int a, int b, int c, Row4 U, bool has_u, bool try_fp64,
                                           unsigned* cnt) {
    const long long* Fu = has_u ? U.v : nullptr;
    unsigned& n64 = cnt[0];
    unsigned& nex = cnt[1];
    int fc[4], bis[3];
    int m = split_planes(a, b, c, fc, bis);
    long long R[3][4];
    for (int k = 0; k < m; k++) row_i64(L, S.Ci, S.W, bis[k] - 4, R[k]);
    if (try_fp64) {
        double Rd[3][4], Cd[4], Fd[4];
        for (int k = 0; k < m; k++) scale_row<double>(R[k], Rd[k]);
        cof_real<double>(m, Rd, fc, Cd);
        const double u = 0x1p-53, em = cof_err<double>(m);
        double sum = Cd[0] + Cd[1] + Cd[2] + Cd[3];
        double sa = fabs(Cd[0]) + fabs(Cd[1]) + fabs(Cd[2]) + fabs(Cd[3]);
        double bs = ((m + 1) * em + 4 * u * sa) * (1 + 8 * u);
        if (fabs(sum) > bs) {
            int ss = sum > 0 ? 1 : -1;
            if (!Fu) {
                n64++;
                return ss;
            }
            scale_row<double>(Fu, Fd);
            double v = fma(Fd[0], Cd[0], fma(Fd[1], Cd[1], fma(Fd[2], Cd[2], Fd[3] * Cd[3])));
            if (fabs(v) > dot_bound<double>(m, Cd)) {
                n64++;
                return (v > 0 ? 1 : -1) * ss;
            }
        }
    }
    nex++;
    I256 C[4];
    exact_cofactors(m, R, fc, C);
    I256 sum = C[0];
    for (int k = 1; k <= m; k++) sum = i256_add(sum, C[k]);
    int ss = i256_sign(sum);
    if (!Fu || ss == 0) return ss;
    I256 v = i256_mul_i64(C[0], Fu[fc[0]]);
    for (int k = 1; k <= m; k++) v = i256_add(v, i256_mul_i64(C[k], Fu[fc[k]]));
    return i256_sign(v) * ss;
}

__device__ __forceinline__ int slow_sign(const Lane& L, const Slow& S, int a, int b, int c, const long long* Fu,
                                         bool try_fp64, unsigned& n64, unsigned& nex) {
    Row4 U;
    if (Fu)
        for (int k = 0; k < 4; k++) U.v[k] = Fu[k];
    else
        for (int k = 0; k < 4; k++) U.v[k] = 0;
    unsigned cnt[2] = {0, 0};
    const int r = slow_sign_impl(L, S, a, b, c, U, Fu != nullptr, try_fp64, cnt);
    n64 += cnt[0];
    nex += cnt[1];
    return r;
}

// ------------------------------------------------------------ smem access
// Per warp: [VMAX][VW][32] slot words followed by [VMAX][32] scratch words.
template <typename Real, int VMAX>
struct Store {
    uint32_t* base;
    int lane;
    static constexpr int VW = PrecTraits<Real>::VW;
    __device__ __forceinline__ uint32_t& w(int v, int k) const { return base[(v * VW + k) * 32 + lane]; }
    __device__ __forceinline__ uint32_t& scratch(int j) const { return base[(VMAX * VW + j) * 32 + lane]; }
    __device__ __forceinline__ uint32_t trip(int v) const { return w(v, 0); }
    __device__ __forceinline__ void set_trip(int v, uint32_t t) const { w(v, 0) = t; }
    __device__ __forceinline__ uint32_t nb(int v) const { return w(v, 1); }
    __device__ __forceinline__ void set_nb(int v, uint32_t t) const { w(v, 1) = t; }
    __device__ __forceinline__ void put_real(int v, int k, float x) const { w(v, 2 + k) = __float_as_uint(x); }
    __device__ __forceinline__ void put_real(int v, int k, double x) const {
        unsigned long long b = __double_as_longlong(x);
        w(v, 2 + 2 * k) = (uint32_t)b;
        w(v, 3 + 2 * k) = (uint32_t)(b >> 32);
    }
    __device__ __forceinline__ void get_real(int v, int k, float& x) const { x = __uint_as_float(w(v, 2 + k)); }
    __device__ __forceinline__ void get_real(int v, int k, double& x) const {
        unsigned long long b = (unsigned long long)w(v, 2 + 2 * k) | ((unsigned long long)w(v, 3 + 2 * k) << 32);
        x = __longlong_as_double(b);
    }
};

// Weight (0/1 ownership) of the mesh face carrying the element defined by the
// tet-face planes in `fmask` (bits 0..3); interior elements weigh 1.
__device__ __forceinline__ int carrier_weight(unsigned fmask, uint32_t own) {
    int nf = __popc(fmask);
    if (nf == 0) return 1;
    if (nf == 1) return (own >> (10 + __ffs(fmask) - 1)) & 1;
    unsigned rest = (~fmask) & 15u;
    if (nf == 2) {
        int a = __ffs(rest) - 1;
        int b = __ffs(rest & (rest - 1)) - 1;
        return (own >> (4 + tet_edge_index(a, b))) & 1;
    }
    return (own >> (__ffs(rest) - 1)) & 1;   // the corner not on the three faces
}

__device__ __forceinline__ unsigned fbits(int p) { return p < 4 ? (1u << p) : 0u; }
__device__ __forceinline__ unsigned tfbits(uint32_t tw) { return fbits(tb(tw, 0)) | fbits(tb(tw, 1)) | fbits(tb(tw, 2)); }
__device__ __forceinline__ int pos_of(uint32_t tw, int p) { return tb(tw, 0) == p ? 0 : (tb(tw, 1) == p ? 1 : (tb(tw, 2) == p ? 2 : -1)); }

__device__ __forceinline__ __int128 tet_det6(const int3* X) {
    long long ax = X[1].x - X[0].x, ay = X[1].y - X[0].y, az = X[1].z - X[0].z;
    long long bx = X[2].x - X[0].x, by = X[2].y - X[0].y, bz = X[2].z - X[0].z;
    long long cx = X[3].x - X[0].x, cy = X[3].y - X[0].y, cz = X[3].z - X[0].z;
    return (__int128)ax * ((__int128)by * cz - (__int128)bz * cy) - (__int128)ay * ((__int128)bx * cz - (__int128)bz * cx) +
           (__int128)az * ((__int128)bx * cy - (__int128)by * cx);
}

__device__ __forceinline__ double tet_volume6(const int3* X) {
    long long ax = X[1].x - X[0].x, ay = X[1].y - X[0].y, az = X[1].z - X[0].z;
    long long bx = X[2].x - X[0].x, by = X[2].y - X[0].y, bz = X[2].z - X[0].z;
    long long cx = X[3].x - X[0].x, cy = X[3].y - X[0].y, cz = X[3].z - X[0].z;
    __int128 d = (__int128)ax * ((__int128)by * cz - (__int128)bz * cy) -
                 (__int128)ay * ((__int128)bx * cz - (__int128)bz * cx) +
                 (__int128)az * ((__int128)bx * cy - (__int128)by * cx);
    return (double)d;
}

// Warp-wide exclusive scan of a per-lane count + one atomic reservation.
__device__ __forceinline__ long long warp_reserve(unsigned cnt, unsigned long long* counter) {
    int lane = threadIdx.x & 31;
    unsigned inc = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        unsigned o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += o;
    }
    unsigned total = __shfl_sync(0xffffffffu, inc, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return (long long)base + (inc - cnt);
}

__device__ __forceinline__ bool bit(unsigned long long m0, unsigned long long m1, int v) {
    return v < 64 ? ((m0 >> v) & 1) : ((m1 >> (v - 64)) & 1);
}

// Fractional Euler records of one cut piece (Sec. 4.1.2): the RPC contribution
// V - E + F - 1 with carrier weights and its links through tet faces, one RPF
// record per radical face of a sphere j > i (polygon V - E + 1), one RPE
// record per edge on two radical planes of spheres > i, one RPV record per
// vertex on three.  All lanes call it (warp-wide reservations); inactive
// lanes emit nothing.
template <int VMAX, typename S>
__device__ __forceinline__ void emit_records(const ClipArgs& A, const Lane& L, const S& V, int nslot, long long p,
                                             bool active) {
    const int b = A.key_bits;
    unsigned long long fmask = 0;   // planes present as faces
    unsigned nF = 0, nE = 0, nV = 0;
    if (active) {
        for (int v = 0; v < nslot; v++) {
            const uint32_t tw = V.trip(v);
            if (is_dead(tw)) continue;
            const int x0 = tb(tw, 0), x1 = tb(tw, 1), x2 = tb(tw, 2);
            fmask |= (1ull << x0) | (1ull << x1) | (1ull << x2);
            if (x0 >= 4 && x1 >= 4 && x2 >= 4 && L.cand[x0 - 4] > L.i && L.cand[x1 - 4] > L.i && L.cand[x2 - 4] > L.i)
                nV++;
            const int ex[3] = {x0, x1, x2}, ey[3] = {x1, x2, x0};
#pragma unroll
            for (int e = 0; e < 3; e++)
                if (ex[e] < ey[e] && ex[e] >= 4 && L.cand[ex[e] - 4] > L.i && L.cand[ey[e] - 4] > L.i) nE++;
        }
        for (int pl = 4; pl < 4 + L.n; pl++)
            if (((fmask >> pl) & 1) && L.cand[pl - 4] > L.i) nF++;
    }
    const long long fb = warp_reserve(nF, &A.rcount[0]);
    const long long eb = warp_reserve(nE, &A.rcount[1]);
    const long long vb = warp_reserve(nV, &A.rcount[2]);
    if (!active) return;
    A.f_off[p] = (int32_t)fb;
    A.f_cnt[p] = (uint8_t)nF;
    A.e_off[p] = (int32_t)eb;
    A.e_cnt[p] = (uint8_t)nE;
    const int32_t* adj = A.adj + 4 * L.t;
    // RPC contribution V - E + F - C and links through tet faces
    {
        int sv = 0, se = 0, sf = 0;
        for (int v = 0; v < nslot; v++) {
            const uint32_t tw = V.trip(v);
            if (is_dead(tw)) continue;
            sv += carrier_weight(tfbits(tw), L.own);
#pragma unroll
            for (int e = 0; e < 3; e++) {
                const int x = tb(tw, e), y = tb(tw, (e + 1) % 3);
                if (x < y) se += carrier_weight(fbits(x) | fbits(y), L.own);
            }
        }
        unsigned lk = 0;
        for (int f = 0; f < 4; f++)
            if ((fmask >> f) & 1) {
                sf += carrier_weight(1u << f, L.own);
                if (adj[f] >= 0) lk |= 1u << f;
                lk |= 16u << f;   // the piece has a face on tet face f
            }
        sf += __popcll(fmask >> 4);   // radical faces are interior (weight 1)
        A.c_val[p] = sv - se + sf - 1;
        A.c_link[p] = (uint8_t)lk;
    }
    // RPF records: walk the polygon on the radical plane of each sphere j > i
    {
        long long wr = fb;
        for (int pl = 4; pl < 4 + L.n; pl++) {
            if (!((fmask >> pl) & 1)) continue;
            const int j = L.cand[pl - 4];
            if (j <= L.i) continue;
            int v0 = 0;
            while (is_dead(V.trip(v0)) || pos_of(V.trip(v0), pl) < 0) v0++;
            int sv = 0, se = 0, v = v0;
            unsigned lk = 0;
            for (int guard = 0; guard < VMAX; guard++) {
                const uint32_t tw = V.trip(v);
                const int kp = pos_of(tw, pl);
                const int r = tb(tw, (kp + 2) % 3);          // edge (r -> pl) leads to the next vertex
                sv += carrier_weight(tfbits(tw), L.own);
                se += carrier_weight(fbits(r), L.own);
                if (r < 4 && adj[r] >= 0) lk |= 1u << r;
                if (r < 4) lk |= 16u << r;   // the polygon has an edge on tet face r
                v = tb(V.nb(v), (kp + 2) % 3);
                if (v == v0) break;
            }
            if (wr < A.rcap[0]) {
                A.rkey[0][wr] = ((unsigned long long)L.i << b) | (unsigned long long)j;
                A.rtet[0][wr] = (int32_t)L.t;
                A.rval[0][wr] = (int16_t)(sv - se + 1);
                A.rlink[0][wr] = (uint8_t)lk;
            }
            wr++;
        }
    }
    // RPE records (edges on two radical planes) and RPV records
    {
        long long we = eb, wv = vb;
        for (int v = 0; v < nslot; v++) {
            const uint32_t tw = V.trip(v);
            if (is_dead(tw)) continue;
            const uint32_t nw = V.nb(v);
#pragma unroll
            for (int e = 0; e < 3; e++) {
                const int x = tb(tw, e), y = tb(tw, (e + 1) % 3), z = tb(tw, (e + 2) % 3);
                if (!(x < y && x >= 4)) continue;
                const int j = L.cand[x - 4], k = L.cand[y - 4];
                if (j <= L.i || k <= L.i) continue;
                const uint32_t tw2 = V.trip(tb(nw, e));       // other end point (holds y -> x)
                const int tz = tb(tw2, 0) + tb(tw2, 1) + tb(tw2, 2) - x - y;
                const int sv = carrier_weight(fbits(z), L.own) + carrier_weight(fbits(tz), L.own);
                unsigned lk = 0;
                if (z < 4 && adj[z] >= 0) lk |= 1u << z;
                if (tz < 4 && adj[tz] >= 0) lk |= 1u << tz;
                if (z < 4) lk |= 16u << z;     // an end point lies on tet face z
                if (tz < 4) lk |= 16u << tz;
                const int lo = min(j, k), hi = max(j, k);
                if (we < A.rcap[1]) {
                    A.rkey[1][we] = ((unsigned long long)L.i << (2 * b)) | ((unsigned long long)lo << b) |
                                    (unsigned long long)hi;
                    A.rtet[1][we] = (int32_t)L.t;
                    A.rval[1][we] = (int16_t)(sv - 1);
                    A.rlink[1][we] = (uint8_t)lk;
                }
                we++;
            }
            const int x0 = tb(tw, 0), x1 = tb(tw, 1), x2 = tb(tw, 2);
            if (x0 >= 4 && x1 >= 4 && x2 >= 4) {
                const int j = L.cand[x0 - 4], k = L.cand[x1 - 4], m3 = L.cand[x2 - 4];
                if (j > L.i && k > L.i && m3 > L.i) {
                    const int s0 = min(j, min(k, m3)), s2 = max(j, max(k, m3)), s1 = j + k + m3 - s0 - s2;
                    if (wv < A.rcap[2] && 4 * b <= 64) {
                        A.rkey[2][wv] = ((unsigned long long)L.i << (3 * b)) |
                                        ((unsigned long long)s0 << (2 * b)) | ((unsigned long long)s1 << b) |
                                        (unsigned long long)s2;
                        A.rtet[2][wv] = (int32_t)L.t;
                        A.rval[2][wv] = 1;
                        A.rlink[2][wv] = 0;
                    }
                    wv++;
                }
            }
        }
    }
}

// ----------------------------------------------------------- clip kernel
template <typename Real, int VMAX>
__device__ __forceinline__ void clip_one(const ClipArgs& A, const int32_t* __restrict__ pairs, long long q, bool active,
                                         const Store<Real, VMAX>& V) {
    Lane L;
    long long p = 0;
    int nslot = 0, nlive = 0;
    bool alive = active, whole = true, degenerate = false;
    unsigned nfast = 0, n64 = 0, nex = 0;
    unsigned nvp = 0;   // constructed vertices with m = 1, 2, 3 radical planes, 10 bits each
    const Slow S{A.Ci, A.W, A.st};
    if (active) {
        p = pairs[q];
        L.t = A.pair_tet[p];
        L.si = (int)(p - A.pair_off[L.t]);
        L.n = A.cand_cnt[L.t];
        L.cand = A.cand + L.t * RPD_MAXC;
        L.i = L.cand[L.si];
        L.own = A.own[L.t];
        const int3 ci = ld_int3(A.Ci, L.i);
        const long long wi = A.W[L.i];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            L.X[k] = ld_int3(A.Xi, A.tets[4 * L.t + k]);
            L.di[k] = pd_exact(L.X[k], ci, wi);
        }
        // the tet: corner a lies on the three faces != a; neighbours across
        // the dual edges trip[0]->trip[1], trip[1]->trip[2], trip[2]->trip[0]
        V.set_trip(0, pack3(1, 2, 3));
        V.set_nb(0, pack3(3, 1, 2));
        V.set_trip(1, pack3(0, 3, 2));
        V.set_nb(1, pack3(2, 0, 3));
        V.set_trip(2, pack3(0, 1, 3));
        V.set_nb(2, pack3(3, 0, 1));
        V.set_trip(3, pack3(0, 2, 1));
        V.set_nb(3, pack3(1, 0, 2));
        nslot = nlive = 4;
    }
    // ---------------------------------------------------------- clipping
    const uint8_t* ord = active ? A.cand_ord + L.t * RPD_MAXC : nullptr;
    for (int k = 0; alive && k < L.n; k++) {
        const int s = ord[k];
        if (s == L.si) continue;
        long long F[4];
        row_i64(L, A.Ci, A.W, s, F);
        if (F[0] < 0 && F[1] < 0 && F[2] < 0 && F[3] < 0) continue;   // plane misses the tet
        if (F[0] > 0 && F[1] > 0 && F[2] > 0 && F[3] > 0) {            // tet inside cell s
            alive = false;
            break;
        }
        Real Fr[4];
        scale_row<Real>(F, Fr);
        const int l = 4 + s;
        unsigned long long out0 = 0, out1 = 0;
        int nout = 0;
        for (int v = 0; v < nslot; v++) {
            const uint32_t tw = V.trip(v);
            if (is_dead(tw)) continue;
            const int a = tb(tw, 0), b = tb(tw, 1), c = tb(tw, 2);
            int sg;
            if (a < 4 && b < 4 && c < 4) {
                const long long fv = get4(F, 6 - a - b - c);
                sg = (fv > 0) - (fv < 0);
            } else {
                Real C0, C1, C2, C3, B;
                V.get_real(v, 0, C0);
                V.get_real(v, 1, C1);
                V.get_real(v, 2, C2);
                V.get_real(v, 3, C3);
                V.get_real(v, 4, B);
                const Real val = fma(Fr[0], C0, fma(Fr[1], C1, fma(Fr[2], C2, Fr[3] * C3)));
                if (fabs(val) > B && !A.force_slow) {
                    sg = val > 0 ? 1 : -1;
                    nfast++;
                } else {
                    sg = slow_sign(L, S, a, b, c, F, sizeof(Real) == 4 && A.force_slow < 2, n64, nex);
                }
            }
            if (sg == 0) {
                degenerate = true;
                break;
            }
            if (sg > 0) {
                if (v < 64) out0 |= 1ull << v;
                else out1 |= 1ull << (v - 64);
                nout++;
            }
        }
        if (degenerate) {
            alive = false;
            break;
        }
        if (nout == 0) continue;
        if (nout == nlive) {
            alive = false;
            break;
        }
        whole = false;
        // boundary of the removed region: dual edges x->y of removed vertices
        // whose neighbour w is kept; one new vertex (x, y, l) each
        int nbd = 0;
        for (int r = 0; r < nslot; r++) {
            if (!bit(out0, out1, r)) continue;
            const uint32_t tw = V.trip(r), nw = V.nb(r);
#pragma unroll
            for (int e = 0; e < 3; e++) {
                const int w = tb(nw, e);
                if (bit(out0, out1, w)) continue;
                if (nbd == VMAX) {
                    nbd = VMAX + 1;
                    break;
                }
                V.scratch(nbd++) = (uint32_t)tb(tw, e) | ((uint32_t)tb(tw, (e + 1) % 3) << 8) | ((uint32_t)w << 16);
            }
            V.set_trip(r, DEAD);
        }
        if (nbd > VMAX) {
            dev_fail(A.st, RPD_E_OVERFLOW, CNT_CAPACITY);
            alive = false;
            break;
        }
        // slots: free slots first, then append
        int cur = 0;
        for (int j = 0; j < nbd; j++) {
            while (cur < nslot && !is_dead(V.trip(cur))) cur++;
            int h;
            if (cur < nslot) {
                h = cur++;
            } else {
                h = nslot++;
                cur = nslot;
            }
            if (h >= VMAX) {
                dev_fail(A.st, RPD_E_OVERFLOW, CNT_CAPACITY);
                alive = false;
                break;
            }
            V.scratch(j) |= (uint32_t)h << 24;
            V.set_trip(h, DEAD | 0x00ffffffu);   // reserved (still free for the scan below)
        }
        if (!alive) break;
        for (int j = 0; j < nbd; j++) {
            const uint32_t e = V.scratch(j);
            const int x = e & 0xff, y = (e >> 8) & 0xff, w = (e >> 16) & 0xff, h = e >> 24;
            int n1 = -1, n2 = -1;
            for (int j2 = 0; j2 < nbd; j2++) {
                const uint32_t e2 = V.scratch(j2);
                if ((int)(e2 & 0xff) == y) n1 = e2 >> 24;          // next: starts at y
                if ((int)((e2 >> 8) & 0xff) == x) n2 = e2 >> 24;   // previous: ends at x
            }
            // w held the dual edge y -> x towards the removed vertex
            const uint32_t tww = V.trip(w);
            const int kk = (tb(tww, 0) == y && tb(tww, 1) == x)   ? 0
                           : (tb(tww, 1) == y && tb(tww, 2) == x) ? 1
                           : (tb(tww, 2) == y && tb(tww, 0) == x) ? 2
                                                                  : -1;
            if (n1 < 0 || n2 < 0 || kk < 0) {   // not a closed dual surface: cannot happen for exact signs
                dev_fail(A.st, RPD_E_DEGENERATE, CNT_CAPACITY);
                degenerate = true;
                alive = false;
                break;
            }
            V.set_trip(h, pack3(x, y, l));
            V.set_nb(h, pack3(w, n1, n2));
            V.set_nb(w, (V.nb(w) & ~(0xffu << (8 * kk))) | ((uint32_t)h << (8 * kk)));
            // homogeneous barycentric coordinates of the new vertex
            int fc[4], bis[3];
            const int m = split_planes(x, y, l, fc, bis);
            nvp += 1u << (10 * (m - 1));
            Real R[3][4];
#pragma unroll
            for (int z = 0; z < 3; z++) {
                if (z >= m) break;
                if (bis[z] == l) {
#pragma unroll
                    for (int c = 0; c < 4; c++) R[z][c] = Fr[c];
                } else {
                    long long Fk[4];
                    row_i64(L, A.Ci, A.W, bis[z] - 4, Fk);
                    scale_row<Real>(Fk, R[z]);
                }
            }
            Real C[4];
            cof_real<Real>(m, R, fc, C);
            const Real u = PrecTraits<Real>::u();
            const Real sum = C[0] + C[1] + C[2] + C[3];
            const Real sa = fabs(C[0]) + fabs(C[1]) + fabs(C[2]) + fabs(C[3]);
            const Real bs = ((Real)(m + 1) * cof_err<Real>(m) + 4 * u * sa) * (1 + 8 * u);
            int ss;
            if (fabs(sum) > bs && !A.force_slow) {
                ss = sum > 0 ? 1 : -1;
                nfast++;
            } else {
                ss = slow_sign(L, S, x, y, l, nullptr, sizeof(Real) == 4 && A.force_slow < 2, n64, nex);
            }
            if (ss == 0) {
                degenerate = true;
                alive = false;
                break;
            }
            if (ss < 0) {
#pragma unroll
                for (int z = 0; z < 4; z++) C[z] = -C[z];
            }
#pragma unroll
            for (int z = 0; z < 4; z++) V.put_real(h, z, C[z]);
            V.put_real(h, 4, dot_bound<Real>(m, C));
        }
        if (!alive) break;
        nlive += nbd - nout;
    }
    if (degenerate) dev_fail(A.st, RPD_E_DEGENERATE, CNT_DEGENERATE);
    if (active && nlive < 4) alive = false;
    dev_count(A.st, CNT_PRED_FAST, nfast);
    dev_count(A.st, CNT_PRED_FP64, n64);
    dev_count(A.st, CNT_PRED_EXACT, nex);
    dev_count(A.st, CNT_NEWVERT1, nvp & 1023u);
    dev_count(A.st, CNT_NEWVERT2, (nvp >> 10) & 1023u);
    dev_count(A.st, CNT_NEWVERT3, nvp >> 20);

    // ------------------------- whole pieces here; cut pieces to the queue
    // (their fractional Euler records are emitted by k_records, their volume
    // by k_volume)
    const bool queued = alive && !whole;
    const long long qb = warp_reserve(queued ? 1u : 0u, A.qcount);
    if (queued && qb < A.qcap) {
        A.qpair[qb] = (int32_t)p;
        A.qnv[qb] = (uint8_t)nslot;
        for (int v = 0; v < nslot; v++) {
            A.qtrip[(2LL * v) * A.qcap + qb] = V.trip(v);
            A.qtrip[(2LL * v + 1) * A.qcap + qb] = V.nb(v);
        }
    }
    if (!active) return;
    A.pflag[p] = alive ? 1 : 0;
    if (!alive) {
        A.c_val[p] = 0;
        A.c_link[p] = 0;
        A.f_off[p] = A.e_off[p] = 0;
        A.f_cnt[p] = A.e_cnt[p] = 0;
        A.p_vol[p] = 0.0;
        A.p_mom[3 * p] = A.p_mom[3 * p + 1] = A.p_mom[3 * p + 2] = 0.0;
        return;
    }
    if (!whole) return;
    {   // the whole tet: V - E + F - 1 from the ownership bits, links on every shared face
        const int32_t* adj = A.adj + 4 * L.t;
        unsigned lk = 0xf0u;   // the whole tet has a face on each tet face
        for (int f = 0; f < 4; f++)
            if (adj[f] >= 0) lk |= 1u << f;
        A.c_val[p] = __popc(L.own & 0xfu) - __popc(L.own & 0x3f0u) + __popc(L.own & 0x3c00u) - 1;
        A.c_link[p] = (uint8_t)lk;
        A.f_off[p] = A.e_off[p] = 0;
        A.f_cnt[p] = A.e_cnt[p] = 0;
    }
    // whole tets: volume and moment in closed form; cut pieces were queued
    if (whole) {
        const double vt = tet_volume6(L.X) / 6.0;
        const double u3 = A.unit * A.unit * A.unit;
        A.p_vol[p] = vt * u3;
        A.p_mom[3 * p + 0] = vt * 0.25 * ((double)L.X[0].x + L.X[1].x + L.X[2].x + L.X[3].x) * u3 * A.unit;
        A.p_mom[3 * p + 1] = vt * 0.25 * ((double)L.X[0].y + L.X[1].y + L.X[2].y + L.X[3].y) * u3 * A.unit;
        A.p_mom[3 * p + 2] = vt * 0.25 * ((double)L.X[0].z + L.X[1].z + L.X[2].z + L.X[3].z) * u3 * A.unit;
    }
}

template <typename Real, int VMAX>
__global__ void __launch_bounds__(128) k_clip(ClipArgs A, const int32_t* __restrict__ pairs,
                                              const int32_t* __restrict__ d_n) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Store<Real, VMAX> V{smem + (size_t)warp * VMAX * (PrecTraits<Real>::VW + 1) * 32, lane};
    const long long n = *d_n;
    // grid-stride over pairs; q0 is warp-uniform so warp collectives stay converged
    for (long long q0 = (long long)blockIdx.x * blockDim.x + warp * 32; q0 < n;
         q0 += (long long)gridDim.x * blockDim.x) {
        const long long q = q0 + lane;
        clip_one<Real, VMAX>(A, pairs, q, q < n, V);
        __syncwarp();
    }
}

// ------------------------------------------------------ fractional Euler records
// One lane per cut piece of a bin's queue: the piece's slot words (triplet,
// dual neighbours) are staged in shared memory, then emit_records runs on them.
struct QStore {
    uint32_t* base;
    int lane;
    __device__ __forceinline__ uint32_t& w(int v, int k) const { return base[(v * 2 + k) * 32 + lane]; }
    __device__ __forceinline__ uint32_t trip(int v) const { return base[(v * 2) * 32 + lane]; }
    __device__ __forceinline__ uint32_t nb(int v) const { return base[(v * 2 + 1) * 32 + lane]; }
};

template <int VMAX>
__global__ void __launch_bounds__(128) k_records(ClipArgs A) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const QStore V{smem + (size_t)warp * VMAX * 2 * 32, lane};
    const long long qn = (long long)*A.qcount;
    const long long n = qn < A.qcap ? qn : A.qcap;
    const long long q0 = (long long)blockIdx.x * blockDim.x + warp * 32;
    if (q0 >= n) return;   // warp-uniform
    const long long q = q0 + lane;
    const bool active = q < n;
    Lane L{};
    long long p = 0;
    int nslot = 0;
    if (active) {
        p = A.qpair[q];
        nslot = A.qnv[q];
        L.t = A.pair_tet[p];
        L.si = (int)(p - A.pair_off[L.t]);
        L.n = A.cand_cnt[L.t];
        L.cand = A.cand + L.t * RPD_MAXC;
        L.i = L.cand[L.si];
        L.own = A.own[L.t];
        for (int v = 0; v < nslot; v++) {
            V.w(v, 0) = A.qtrip[(2LL * v) * A.qcap + q];
            V.w(v, 1) = A.qtrip[(2LL * v + 1) * A.qcap + q];
        }
    }
    emit_records<VMAX>(A, L, V, nslot, p, active);
}

// ------------------------------------------------------ volume and moment
// Chart coordinates of the tet: x = X0 + sum_{c=1..3} beta_c (X_c - X0), with
// Jacobian 6 vol(t).  With P_v = beta_v - beta_a (chart, relative to an apex
// vertex a of the piece), the piece is the union of the tets (a, R, v, v')
// over the fan triangles (R, v, v') of every face not through a, R being the
// face's first vertex; faces are walked through the dual adjacency.
//   vol(P) = vol(t) |sum d|,  d = det(P_R, P_v, P_v')
//   int_P x = vol(P) X0 + vol(t) sum_c (X_c - X0) (beta_a,c |sum d| + sign * sum d (P_R+P_v+P_v')_c / 4)
// Exact rows F_s[c] = pd(X_c, i) - pd(X_c, s) of a candidate plane, computed
// where a vertex coordinate needs them (the sphere's centre and weight come
// from the L1/L2-resident sphere arrays).  Keeping them in shared memory
// instead cost 1 KB per warp per candidate and halved the occupancy of the
// middle bins.
struct RowCache {
    const Lane& L;
    const int32_t* __restrict__ Ci;
    const long long* __restrict__ W;
    __device__ __forceinline__ long long get(int slot, int c) const {
        const int s = L.cand[slot];
        const int3 x = c == 0 ? L.X[0] : (c == 1 ? L.X[1] : (c == 2 ? L.X[2] : L.X[3]));
        const long long d = c == 0 ? L.di[0] : (c == 1 ? L.di[1] : (c == 2 ? L.di[2] : L.di[3]));
        return d - pd_exact(x, ld_int3(Ci, s), W[s]);
    }
    __device__ __forceinline__ void row(int slot, long long F[4]) const { row_i64(L, Ci, W, slot, F); }
};

template <typename Real>
struct VolAcc;

// Double-float accumulation (FP32 pipes) for the FP32-filtered mode.
template <>
struct VolAcc<float> {
    df s0{0, 0}, s1{0, 0}, s2{0, 0}, s3{0, 0};
    static __device__ __forceinline__ void beta(const Lane& L, const RowCache& RC, int a, int b, int c, df out[3]) {
        int fc[4], bis[3];
        const int m = split_planes(a, b, c, fc, bis);
        df be[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        if (m == 0) {
            set4(be, 6 - a - b - c, df_make(1.0f));
        } else if (m == 1) {
            // on the tet edge between corners c0 and c1: the exact row entries
            // F0, F1 of the one radical plane give beta_c0 = F1 / (F1 - F0)
            const int c0 = fc[0], c1 = fc[1];
            const long long F0 = RC.get(bis[0] - 4, c0);
            const long long F1 = RC.get(bis[0] - 4, c1);
            const df b0 = df_div_fast(df_from_i64(F1), df_from_i64(F1 - F0));
            set4(be, c0, b0);
            set4(be, c1, df_sub(df_make(1.0f), b0));
        } else if (m == 2) {
            // on a tet face: the cofactors of two exact rows over the three
            // free columns, in exact 128-bit integers (|entry| < 2^47)
            long long F[4], G[4];
            RC.row(bis[0] - 4, F);
            RC.row(bis[1] - 4, G);
            const long long f0 = get4(F, fc[0]), f1 = get4(F, fc[1]), f2 = get4(F, fc[2]);
            const long long g0 = get4(G, fc[0]), g1 = get4(G, fc[1]), g2 = get4(G, fc[2]);
            const __int128 k0 = (__int128)f1 * g2 - (__int128)f2 * g1;
            const __int128 k1 = (__int128)f2 * g0 - (__int128)f0 * g2;
            const __int128 k2 = (__int128)f0 * g1 - (__int128)f1 * g0;
            const df inv = df_div_fast(df_make(1.0f), df_from_i128(k0 + k1 + k2));
            set4(be, fc[0], df_mul(df_from_i128(k0), inv));
            set4(be, fc[1], df_mul(df_from_i128(k1), inv));
            set4(be, fc[2], df_mul(df_from_i128(k2), inv));
        } else {
            df R[3][4];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k >= m) break;
                long long F[4];
                RC.row(bis[k] - 4, F);
                unsigned long long mx = 0;
#pragma unroll
                for (int z = 0; z < 4; z++) mx = max(mx, (unsigned long long)(F[z] < 0 ? -F[z] : F[z]));
                const int e = mx ? 64 - __clzll(mx) : 0;
                const float sc = __int_as_float((127 - e) << 23);
#pragma unroll
                for (int z = 0; z < 4; z++) R[k][z] = df_scale(df_from_i64(F[z]), sc);
            }
            df C[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
            if (m == 1) {
                set4(C, fc[0], get4(R[0], fc[1]));
                set4(C, fc[1], df_neg(get4(R[0], fc[0])));
            } else if (m == 2) {
                const df x0 = get4(R[0], fc[0]), x1 = get4(R[0], fc[1]), x2 = get4(R[0], fc[2]);
                const df y0 = get4(R[1], fc[0]), y1 = get4(R[1], fc[1]), y2 = get4(R[1], fc[2]);
                set4(C, fc[0], df_sub(df_mul(x1, y2), df_mul(x2, y1)));
                set4(C, fc[1], df_sub(df_mul(x2, y0), df_mul(x0, y2)));
                set4(C, fc[2], df_sub(df_mul(x0, y1), df_mul(x1, y0)));
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int c0 = k == 0 ? 1 : 0, c1 = k <= 1 ? 2 : 1, c2 = k <= 2 ? 3 : 2;
                    const df m0 = df_sub(df_mul(R[1][c1], R[2][c2]), df_mul(R[1][c2], R[2][c1]));
                    const df m1 = df_sub(df_mul(R[1][c0], R[2][c2]), df_mul(R[1][c2], R[2][c0]));
                    const df m2 = df_sub(df_mul(R[1][c0], R[2][c1]), df_mul(R[1][c1], R[2][c0]));
                    const df d = df_add(df_sub(df_mul(R[0][c0], m0), df_mul(R[0][c1], m1)), df_mul(R[0][c2], m2));
                    C[k] = (k & 1) ? df_neg(d) : d;
                }
            }
            const df inv = df_div_fast(df_make(1.0f), df_add(df_add(C[0], C[1]), df_add(C[2], C[3])));
#pragma unroll
            for (int z = 1; z < 4; z++) be[z] = df_mul(C[z], inv);
        }
        out[0] = be[1];
        out[1] = be[2];
        out[2] = be[3];
    }
    __device__ __forceinline__ void term(const df* P1, const df* P2, const df* P3) {
        const df c0 = df_sub(df_mul(P2[1], P3[2]), df_mul(P2[2], P3[1]));
        const df c1 = df_sub(df_mul(P2[2], P3[0]), df_mul(P2[0], P3[2]));
        const df c2 = df_sub(df_mul(P2[0], P3[1]), df_mul(P2[1], P3[0]));
        const df d = df_add(df_add(df_mul(P1[0], c0), df_mul(P1[1], c1)), df_mul(P1[2], c2));
        s0 = df_add(s0, d);
        s1 = df_add(s1, df_mul(d, df_add(df_add(P1[0], P2[0]), P3[0])));
        s2 = df_add(s2, df_mul(d, df_add(df_add(P1[1], P2[1]), P3[1])));
        s3 = df_add(s3, df_mul(d, df_add(df_add(P1[2], P2[2]), P3[2])));
    }
    __device__ __forceinline__ void result(double* S) const {
        S[0] = df_to_double(s0);
        S[1] = df_to_double(s1);
        S[2] = df_to_double(s2);
        S[3] = df_to_double(s3);
    }
};

// Native FP64 for the FP64 mode.
template <>
struct VolAcc<double> {
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    static __device__ __forceinline__ void beta(const Lane& L, const RowCache& RC, int a, int b, int c, double out[3]) {
        int fc[4], bis[3];
        const int m = split_planes(a, b, c, fc, bis);
        double be[4] = {0, 0, 0, 0};
        if (m == 0) {
            set4(be, 6 - a - b - c, 1.0);
        } else {
            double Rd[3][4], Cd[4];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k >= m) break;
                long long Fk[4];
                RC.row(bis[k] - 4, Fk);
                scale_row<double>(Fk, Rd[k]);
            }
            cof_real<double>(m, Rd, fc, Cd);
            const double inv = 1.0 / (Cd[0] + Cd[1] + Cd[2] + Cd[3]);
#pragma unroll
            for (int z = 0; z < 4; z++) be[z] = Cd[z] * inv;
        }
        out[0] = be[1];
        out[1] = be[2];
        out[2] = be[3];
    }
    __device__ __forceinline__ void term(const double* P1, const double* P2, const double* P3) {
        const double d = P1[0] * (P2[1] * P3[2] - P2[2] * P3[1]) - P1[1] * (P2[0] * P3[2] - P2[2] * P3[0]) +
                         P1[2] * (P2[0] * P3[1] - P2[1] * P3[0]);
        s0 += d;
        s1 += d * (P1[0] + P2[0] + P3[0]);
        s2 += d * (P1[1] + P2[1] + P3[1]);
        s3 += d * (P1[2] + P2[2] + P3[2]);
    }
    __device__ __forceinline__ void result(double* S) const {
        S[0] = s0;
        S[1] = s1;
        S[2] = s2;
        S[3] = s3;
    }
};

// Volume-kernel storage per warp: [vmax][8][32] words: trip, nb, P (3 values).
template <typename T>
struct VStore {
    uint32_t* base;
    int lane;
    __device__ __forceinline__ uint32_t& w(int v, int k) const { return base[(v * 8 + k) * 32 + lane]; }
    __device__ __forceinline__ void put(int v, int k, df x) const {
        w(v, 2 + 2 * k) = __float_as_uint(x.hi);
        w(v, 3 + 2 * k) = __float_as_uint(x.lo);
    }
    __device__ __forceinline__ void put(int v, int k, double x) const {
        unsigned long long b = __double_as_longlong(x);
        w(v, 2 + 2 * k) = (uint32_t)b;
        w(v, 3 + 2 * k) = (uint32_t)(b >> 32);
    }
    __device__ __forceinline__ void get(int v, int k, df& x) const {
        x.hi = __uint_as_float(w(v, 2 + 2 * k));
        x.lo = __uint_as_float(w(v, 3 + 2 * k));
    }
    __device__ __forceinline__ void get(int v, int k, double& x) const {
        x = __longlong_as_double((long long)((unsigned long long)w(v, 2 + 2 * k) |
                                             ((unsigned long long)w(v, 3 + 2 * k) << 32)));
    }
};

// Volume and first moment of a piece cut by one radical plane only (every
// vertex on tet faces and the plane of one sphere s): the part F . beta <= 0
// of the tet in barycentric coordinates beta, F the exact row of s.  With K
// the corners where F < 0 and s_ax = F_a / (F_a - F_x) the position of the
// cut along edge a -> x:
//   |K| = 1, K = {a}: the tet (a, p_ab, p_ac, p_ad), fraction s_ab s_ac s_ad;
//   |K| = 3: the tet minus that tet at the fourth corner;
//   |K| = 2, K = {a, b}: the wedge between the triangles (a, p_ac, p_ad) and
//     (b, p_bc, p_bd), split into the tets (a, p_ac, p_ad, b),
//     (p_ac, p_ad, b, p_bc) and (p_ad, b, p_bc, p_bd) of fractions
//     s_ac s_ad, s_ad s_bc (1 - s_ac) and s_bc s_bd (1 - s_ad), all positive.
// The barycentric first moment is the fraction-weighted vertex mean of those
// tets.  T is double-float in the FP32-filtered mode (FP32 pipes; native
// FP64 runs at 1/64 of the rate) and double in the FP64 mode.
template <typename T>
struct Arith;
template <>
struct Arith<df> {
    static __device__ __forceinline__ df add(df a, df b) { return df_add(a, b); }
    static __device__ __forceinline__ df sub(df a, df b) { return df_sub(a, b); }
    static __device__ __forceinline__ df mul(df a, df b) { return df_mul(a, b); }
    static __device__ __forceinline__ df div(df a, df b) { return df_div_fast(a, b); }
    static __device__ __forceinline__ df from_i64(long long v) { return df_from_i64(v); }
    static __device__ __forceinline__ df num(float v) { return df_make(v); }
    static __device__ __forceinline__ double dbl(df v) { return df_to_double(v); }
};
template <>
struct Arith<double> {
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double from_i64(long long v) { return (double)v; }
    static __device__ __forceinline__ double num(float v) { return (double)v; }
    static __device__ __forceinline__ double dbl(double v) { return v; }
};

// fr = volume / vol(t); m[k] = (first moment / vol(t))_k - fr X0_k, in grid
// units: sum over corners l of M_l (X_l - X0)_k.
template <typename T>
__device__ __forceinline__ void one_plane_piece(const long long F[4], const int3* X, T& fr, T m[3]) {
    typedef Arith<T> A;
    const int neg = (F[0] < 0) + (F[1] < 0) + (F[2] < 0) + (F[3] < 0);
    auto cut = [&](int a, int x) {
        const long long fa = get4(F, a), fx = get4(F, x);
        return A::div(A::from_i64(fa), A::from_i64(fa - fx));   // |fa - fx| < 2^48: exact operands
    };
    // corners of the tet relative to corner 0, as exact FP32 values (< 2^22)
    auto dX = [&](int l, int k) {
        const int3 p = l == 0 ? X[0] : (l == 1 ? X[1] : (l == 2 ? X[2] : X[3]));
        const int v = k == 0 ? p.x - X[0].x : (k == 1 ? p.y - X[0].y : p.z - X[0].z);
        return A::num((float)v);
    };
    for (int k = 0; k < 3; k++) m[k] = A::num(0.f);
    auto acc = [&](T M, int l) {   // mom += M (X_l - X0)
        if (l == 0) return;
        for (int k = 0; k < 3; k++) m[k] = A::add(m[k], A::mul(M, dX(l, k)));
    };
    if (neg == 1 || neg == 3) {
        // the corner a on the minority side and the tet it cuts off
        const bool want = neg == 1;
        const int a = ((F[0] < 0) == want) ? 0 : (((F[1] < 0) == want) ? 1 : (((F[2] < 0) == want) ? 2 : 3));
        const int x1 = (a + 1) & 3, x2 = (a + 2) & 3, x3 = (a + 3) & 3;
        const T s1 = cut(a, x1), s2 = cut(a, x2), s3 = cut(a, x3);
        const T fs = A::mul(A::mul(s1, s2), s3);
        const T q = A::mul(fs, A::num(0.25f));
        const T ca = A::mul(q, A::sub(A::num(4.f), A::add(A::add(s1, s2), s3)));   // fs * centroid_a
        if (want) {
            fr = fs;
            acc(ca, a);
            acc(A::mul(q, s1), x1);
            acc(A::mul(q, s2), x2);
            acc(A::mul(q, s3), x3);
        } else {   // the whole tet's moment (1/4 each) minus the corner tet's
            fr = A::sub(A::num(1.f), fs);
            const T qt = A::num(0.25f);
            acc(A::sub(qt, ca), a);
            acc(A::sub(qt, A::mul(q, s1)), x1);
            acc(A::sub(qt, A::mul(q, s2)), x2);
            acc(A::sub(qt, A::mul(q, s3)), x3);
        }
    } else {
        int a = -1, b = -1, c = -1, d = -1;
        for (int l = 0; l < 4; l++) {
            if (F[l] < 0) (a < 0 ? a : b) = l;
            else (c < 0 ? c : d) = l;
        }
        const T sac = cut(a, c), sad = cut(a, d), sbc = cut(b, c), sbd = cut(b, d);
        const T one = A::num(1.f);
        const T f1 = A::mul(sac, sad), f2 = A::mul(A::mul(sad, sbc), A::sub(one, sac)),
                f3 = A::mul(A::mul(sbc, sbd), A::sub(one, sad));
        fr = A::add(A::add(f1, f2), f3);
        const T q = A::num(0.25f);
        // vertex sums of the three tets, corner by corner
        const T Ma = A::mul(q, A::add(A::add(A::mul(f1, A::sub(A::num(3.f), A::add(sac, sad))),
                                             A::mul(f2, A::sub(A::num(2.f), A::add(sac, sad)))),
                                      A::mul(f3, A::sub(one, sad))));
        const T Mb = A::mul(q, A::add(A::add(f1, A::mul(f2, A::sub(A::num(2.f), sbc))),
                                      A::mul(f3, A::sub(A::num(3.f), A::add(sbc, sbd)))));
        const T Mc = A::mul(q, A::add(A::add(A::mul(f1, sac), A::mul(f2, A::add(sac, sbc))), A::mul(f3, sbc)));
        const T Md = A::mul(q, A::add(A::mul(A::add(f1, f2), sad), A::mul(f3, A::add(sad, sbd))));
        acc(Ma, a);
        acc(Mb, b);
        acc(Mc, c);
        acc(Md, d);
    }
}

template <typename Real>
__global__ void __launch_bounds__(128) k_volume(ClipArgs A, int vmax, int rmax) {
    typedef typename std::conditional<sizeof(Real) == 4, df, double>::type T;
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const VStore<T> V{smem + (size_t)warp * vmax * 8 * 32, lane};
    (void)rmax;
    (void)nwarps;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)*A.qcount;
    if (q >= n || q >= A.qcap) return;
    const long long p = A.qpair[q];
    Lane L;
    L.t = A.pair_tet[p];
    L.si = (int)(p - A.pair_off[L.t]);
    L.n = A.cand_cnt[L.t];
    L.cand = A.cand + L.t * RPD_MAXC;
    L.i = L.cand[L.si];
    const int3 ci = ld_int3(A.Ci, L.i);
    const long long wi = A.W[L.i];
    for (int k = 0; k < 4; k++) {
        L.X[k] = ld_int3(A.Xi, A.tets[4 * L.t + k]);
        L.di[k] = pd_exact(L.X[k], ci, wi);
    }
    if (L.n == 2) {   // two candidates (a whole bin): one radical plane, closed form
        // the only plane that can cut the piece is the other candidate's, so
        // the queued polytope is not read
        long long F[4];
        row_i64(L, A.Ci, A.W, 1 - L.si, F);
        T fr, mom[3];
        one_plane_piece<T>(F, L.X, fr, mom);
        const double u3 = A.unit * A.unit * A.unit;
        const int x0[3] = {L.X[0].x, L.X[0].y, L.X[0].z};
        if constexpr (sizeof(Real) == 4) {   // double-float to the end, one conversion per output
            const df vt6 = df_from_i128(tet_det6(L.X));
            A.p_vol[p] = df_to_double(df_mul(vt6, fr)) * (u3 / 6.0);
            for (int k = 0; k < 3; k++)
                A.p_mom[3 * p + k] =
                    df_to_double(df_mul(vt6, df_add(df_mul(fr, df_from_i64(x0[k])), mom[k]))) * (u3 * A.unit / 6.0);
        } else {
            const double vt = tet_volume6(L.X) / 6.0;
            A.p_vol[p] = vt * fr * u3;
            for (int k = 0; k < 3; k++) A.p_mom[3 * p + k] = vt * (fr * (double)x0[k] + mom[k]) * u3 * A.unit;
        }
        return;
    }
    const int nslot = A.qnv[q];
    int apex = -1;
    for (int v = 0; v < nslot; v++) {
        const uint32_t tw = A.qtrip[(2LL * v) * A.qcap + q];
        V.w(v, 0) = tw;
        V.w(v, 1) = A.qtrip[(2LL * v + 1) * A.qcap + q];
        if (apex < 0 && !is_dead(tw)) apex = v;
    }
    const RowCache RC{L, A.Ci, A.W};
    // chart coordinates relative to the apex vertex
    T O[3];
    const uint32_t ta = V.w(apex, 0);
    VolAcc<Real>::beta(L, RC, tb(ta, 0), tb(ta, 1), tb(ta, 2), O);
    unsigned long long fm = 0;
    // Coordinates by class of vertex (radical planes through it: 0-1, 2, 3):
    // the cheap class in one pass, the others in passes of their own, so a
    // lane on an expensive vertex holds up its warp only for that class.
    unsigned long long h2lo = 0, h2hi = 0, h3lo = 0, h3hi = 0;   // slots of the m = 2 and m = 3 vertices
    auto coords = [&](int v, uint32_t tw) {
        T be[3];
        VolAcc<Real>::beta(L, RC, tb(tw, 0), tb(tw, 1), tb(tw, 2), be);
        for (int k = 0; k < 3; k++) {
            if constexpr (sizeof(Real) == 4) V.put(v, k, df_sub(be[k], O[k]));
            else V.put(v, k, be[k] - O[k]);
        }
    };
    for (int v = 0; v < nslot; v++) {
        const uint32_t tw = V.w(v, 0);
        if (is_dead(tw) || v == apex) continue;
        fm |= (1ull << tb(tw, 0)) | (1ull << tb(tw, 1)) | (1ull << tb(tw, 2));
        const int m = (tb(tw, 0) >= 4) + (tb(tw, 1) >= 4) + (tb(tw, 2) >= 4);
        const unsigned long long bit = 1ull << (v & 63);
        if (m <= 1) coords(v, tw);
        else if (m == 2) (v < 64 ? h2lo : h2hi) |= bit;
        else (v < 64 ? h3lo : h3hi) |= bit;
    }
    auto pass = [&](unsigned long long bits, int base) {
        for (; bits; bits &= bits - 1) {
            const int v = base + __ffsll((long long)bits) - 1;
            coords(v, V.w(v, 0));
        }
    };
    pass(h2lo, 0);
    pass(h2hi, 64);
    pass(h3lo, 0);
    pass(h3hi, 64);
    // Length of every restricted-power-edge segment this piece emitted (its
    // records, in the order emit_records wrote them from e_off[p]): the end
    // points' chart coordinates P (the apex's is 0) give the world vector
    // sum_c (X_c - X0) dP_c in grid units; stored as fixed point x 2^24.
    if (A.elen && A.e_cnt[p]) {
        // in the chart type: double-float on the FP32 pipes in the
        // FP32-filtered mode (native FP64 runs at 1/64 of the rate there)
        long long we = A.e_off[p];
        auto chart = [&](int v, int k) {
            T x;
            if (v == apex) {
                if constexpr (sizeof(Real) == 4) x = df_make(0.0f);
                else x = 0.0;
            } else {
                V.get(v, k, x);
            }
            return x;
        };
        for (int v = 0; v < nslot; v++) {
            const uint32_t tw = V.w(v, 0);
            if (is_dead(tw)) continue;
            const uint32_t nw = V.w(v, 1);
            for (int e = 0; e < 3; e++) {
                const int x = tb(tw, e), y = tb(tw, (e + 1) % 3);
                if (!(x < y && x >= 4)) continue;
                if (L.cand[x - 4] <= L.i || L.cand[y - 4] <= L.i) continue;
                const int u = tb(nw, e);
                double len;
                if constexpr (sizeof(Real) == 4) {
                    df w3[3] = {df_make(0.f), df_make(0.f), df_make(0.f)};
                    for (int c = 1; c <= 3; c++) {
                        const df d = df_sub(chart(v, c - 1), chart(u, c - 1));
                        const float ex = (float)(L.X[c].x - L.X[0].x), ey = (float)(L.X[c].y - L.X[0].y),
                                    ez = (float)(L.X[c].z - L.X[0].z);   // exact: < 2^22
                        w3[0] = df_add(w3[0], df_mul(d, df_make(ex)));
                        w3[1] = df_add(w3[1], df_mul(d, df_make(ey)));
                        w3[2] = df_add(w3[2], df_mul(d, df_make(ez)));
                    }
                    const df l2 = df_add(df_add(df_mul(w3[0], w3[0]), df_mul(w3[1], w3[1])), df_mul(w3[2], w3[2]));
                    len = df_to_double(df_sqrt(l2));
                } else {
                    double dx = 0, dy = 0, dz = 0;
                    for (int c = 1; c <= 3; c++) {
                        const double d = chart(v, c - 1) - chart(u, c - 1);
                        dx += d * (double)(L.X[c].x - L.X[0].x);
                        dy += d * (double)(L.X[c].y - L.X[0].y);
                        dz += d * (double)(L.X[c].z - L.X[0].z);
                    }
                    len = sqrt(dx * dx + dy * dy + dz * dz);
                }
                if (we < A.rcap[1]) A.elen[we] = llrint(len * 0x1p24);
                we++;
            }
        }
    }
    fm &= ~((1ull << tb(ta, 0)) | (1ull << tb(ta, 1)) | (1ull << tb(ta, 2)));   // faces through the apex
    VolAcc<Real> acc;
    while (fm) {
        const int pl = __ffsll((long long)fm) - 1;
        fm &= fm - 1;
        int R = 0;
        while (is_dead(V.w(R, 0)) || pos_of(V.w(R, 0), pl) < 0) R++;
        // successor around face pl: across the dual edge (r -> pl)
        auto next = [&](int v) {
            const int kp = pos_of(V.w(v, 0), pl);
            return (int)tb(V.w(v, 1), (kp + 2) % 3);
        };
        T PR[3];
        for (int k = 0; k < 3; k++) V.get(R, k, PR[k]);
        int prev = next(R);
        int cur = next(prev);
        for (int guard = 0; guard < vmax && cur != R; guard++) {
            T P2[3], P3[3];
            for (int k = 0; k < 3; k++) {
                V.get(prev, k, P2[k]);
                V.get(cur, k, P3[k]);
            }
            acc.term(PR, P2, P3);
            prev = cur;
            cur = next(cur);
        }
    }
    if constexpr (sizeof(Real) == 4) {
        // the tail in double-float too (FP32 pipes), one conversion per output
        const bool neg = acc.s0.hi < 0.0f;
        const df frac = neg ? df_neg(acc.s0) : acc.s0;
        const df Sc[3] = {neg ? df_neg(acc.s1) : acc.s1, neg ? df_neg(acc.s2) : acc.s2, neg ? df_neg(acc.s3) : acc.s3};
        const df vt6 = df_from_i128(tet_det6(L.X));   // 6 vol(t), grid units
        const double u3 = A.unit * A.unit * A.unit;
        A.p_vol[p] = df_to_double(df_mul(vt6, frac)) * (u3 / 6.0);
        const int xs[4][3] = {{L.X[0].x, L.X[0].y, L.X[0].z}, {L.X[1].x, L.X[1].y, L.X[1].z},
                              {L.X[2].x, L.X[2].y, L.X[2].z}, {L.X[3].x, L.X[3].y, L.X[3].z}};
        df wc[3];
        for (int cc = 0; cc < 3; cc++) wc[cc] = df_add(df_mul(O[cc], frac), df_scale(Sc[cc], 0.25f));
        for (int k = 0; k < 3; k++) {
            const int x0 = xs[0][k];
            df m = df_mul(frac, df_from_i64(x0));
            for (int cc = 1; cc <= 3; cc++) m = df_add(m, df_mul(wc[cc - 1], df_make((float)(xs[cc][k] - x0))));
            A.p_mom[3 * p + k] = df_to_double(df_mul(vt6, m)) * (u3 * A.unit / 6.0);
        }
        return;
    }
    double S[4];
    acc.result(S);
    double Od[3];
    for (int k = 0; k < 3; k++) {
        if constexpr (sizeof(Real) == 4) Od[k] = df_to_double(O[k]);
        else Od[k] = O[k];
    }
    const double sgn = S[0] < 0 ? -1.0 : 1.0;
    const double vt = tet_volume6(L.X) / 6.0;
    const double frac = fabs(S[0]);
    const double u3 = A.unit * A.unit * A.unit;
    A.p_vol[p] = vt * frac * u3;
    const int xs[4][3] = {{L.X[0].x, L.X[0].y, L.X[0].z}, {L.X[1].x, L.X[1].y, L.X[1].z},
                          {L.X[2].x, L.X[2].y, L.X[2].z}, {L.X[3].x, L.X[3].y, L.X[3].z}};
    for (int k = 0; k < 3; k++) {
        const double x0 = (double)xs[0][k];
        double m = vt * frac * x0;
        for (int cc = 1; cc <= 3; cc++)
            m += vt * ((double)xs[cc][k] - x0) * (Od[cc - 1] * frac + sgn * S[cc] * 0.25);
        A.p_mom[3 * p + k] = m * u3 * A.unit;
    }
}

// Whole-tet pieces: a tet with a single candidate lies inside one cell.
__device__ __forceinline__ void whole_one(const ClipArgs& A, long long p) {
    const long long t = A.pair_tet[p];
    const uint32_t own = A.own[t];
    int3 X[4];
    for (int k = 0; k < 4; k++) X[k] = ld_int3(A.Xi, A.tets[4 * t + k]);
    const int32_t* adj = A.adj + 4 * t;
    unsigned lk = 0xf0u;   // the whole tet has a face on each tet face
    for (int f = 0; f < 4; f++)
        if (adj[f] >= 0) lk |= 1u << f;
    A.pflag[p] = 1;
    A.c_val[p] = __popc(own & 0xfu) - __popc(own & 0x3f0u) + __popc(own & 0x3c00u) - 1;
    A.c_link[p] = (uint8_t)lk;
    A.f_off[p] = 0;
    A.f_cnt[p] = 0;
    A.e_off[p] = 0;
    A.e_cnt[p] = 0;
    const double vt = tet_volume6(X) / 6.0;
    const double u3 = A.unit * A.unit * A.unit;
    A.p_vol[p] = vt * u3;
    A.p_mom[3 * p + 0] = vt * 0.25 * ((double)X[0].x + X[1].x + X[2].x + X[3].x) * u3 * A.unit;
    A.p_mom[3 * p + 1] = vt * 0.25 * ((double)X[0].y + X[1].y + X[2].y + X[3].y) * u3 * A.unit;
    A.p_mom[3 * p + 2] = vt * 0.25 * ((double)X[0].z + X[1].z + X[2].z + X[3].z) * u3 * A.unit;
}

__global__ void k_whole(ClipArgs A, const int32_t* __restrict__ pairs, const int32_t* __restrict__ d_n) {
    const long long n = *d_n;
    unsigned cnt = 0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        whole_one(A, pairs[q]);
        cnt++;
    }
    dev_count(A.st, CNT_WHOLE, cnt);
}

// Bins by candidate count n: 0: n = 1 (whole tet), 1..3: n = 2..4,
// 4: 5-6, 5: 7-8, 6: 9-16, 7: 17-32.
__device__ __forceinline__ int bin_of(int n) {
    return n <= 4 ? n - 1 : (n <= 6 ? 4 : (n <= 8 ? 5 : (n <= 16 ? 6 : 7)));
}

// Warp-aggregated atomicAdd of n on counter[b] (lanes with n <= 0 skip);
// returns this lane's base.
__device__ __forceinline__ int warp_bin_add(int n, int b, int32_t* counter) {
    const unsigned peers = __match_any_sync(0xffffffffu, n > 0 ? b : -1);
    const int lane = threadIdx.x & 31;
    const unsigned lt = peers & ((1u << lane) - 1u);
    int pre = 0, tot = 0;
    for (int k = 0; k < 32; k++) {
        const int nk = __shfl_sync(0xffffffffu, n, k);
        if ((peers >> k) & 1) {
            tot += nk;
            if ((lt >> k) & 1) pre += nk;
        }
    }
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader && n > 0 && tot > 0) base = atomicAdd(&counter[b], tot);
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + pre;
}

// only != NULL restricts the binning to the tets it marks (partial update).
__global__ void k_bin_count(const int32_t* __restrict__ cand_cnt, long long nt, int32_t* __restrict__ bin_count,
                            const uint8_t* __restrict__ only) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = (t < nt && (!only || only[t])) ? cand_cnt[t] : 0;
    warp_bin_add(n, n > 0 ? bin_of(n) : 0, bin_count);
}

__global__ void k_bin_prefix(const int32_t* __restrict__ bin_count, int32_t* __restrict__ bin_fill,
                             unsigned long long* __restrict__ rcount, unsigned long long* __restrict__ qcount) {
    int run = 0;
    for (int b = 0; b < RPD_NBINS; b++) {
        bin_fill[b] = run;
        run += bin_count[b];
        if (qcount) qcount[b] = 0;
    }
    if (rcount)
        for (int k = 0; k < 3; k++) rcount[k] = 0;
}

// Writes past cap are dropped (the caller bins again with room for all pairs).
// Every pair gets its tet in pair_tet; only the pairs of the tets `only`
// marks (all when NULL) are put into the bins.
__global__ void k_bin_pairs(const int32_t* __restrict__ cand_cnt, const int64_t* __restrict__ pair_off, long long nt,
                            int32_t* __restrict__ pair_tet, int32_t* __restrict__ bins, int32_t* __restrict__ bin_fill,
                            long long cap, const uint8_t* __restrict__ only) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = t < nt ? cand_cnt[t] : 0;
    const int nb = (t < nt && (!only || only[t])) ? n : 0;
    const int base = warp_bin_add(nb, nb > 0 ? bin_of(nb) : 0, bin_fill);
    if (n <= 0) return;
    const long long off = pair_off[t];
    for (int k = 0; k < n; k++) {
        if (off + k < cap) pair_tet[off + k] = (int32_t)t;
        if (k < nb && base + k < cap) bins[base + k] = (int32_t)(off + k);
    }
}

inline unsigned grid_for(long long n, int tpb) {
    long long b = (n + tpb - 1) / tpb;
    const long long cap = 152LL * 64;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

// Dynamic shared memory above 48 KB needs the kernel's limit raised; the
// attribute belongs to the current device, so it is raised once per device
// (thread-safe).
struct SmemLimit {
    std::mutex mu;
    size_t set[64] = {};
};

inline void raise_smem_limit(const void* fn, size_t bytes, SmemLimit& L) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(L.mu);
    if (bytes > L.set[dev]) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        L.set[dev] = bytes;
    }
}

template <typename Real, int VMAX, int WARPS>
void launch_clip_t(const ClipArgs& a, const int32_t* pairs, const int32_t* d_n, long long n, cudaStream_t s) {
    if (n <= 0) return;
    const size_t smem = (size_t)WARPS * VMAX * (PrecTraits<Real>::VW + 1) * 32 * sizeof(uint32_t);
    static SmemLimit lim;
    raise_smem_limit((const void*)k_clip<Real, VMAX>, smem, lim);
    k_clip<Real, VMAX><<<grid_for(n, 32 * WARPS), 32 * WARPS, smem, s>>>(a, pairs, d_n);
    note_launch();
}

template <typename Real>
void launch_volume_t(const ClipArgs& a, int vmax, int rmax, int warps, long long nmax, cudaStream_t s) {
    if (nmax <= 0) return;
    const size_t smem = (size_t)warps * vmax * 8 * 32 * sizeof(uint32_t);
    static SmemLimit lim;
    raise_smem_limit((const void*)k_volume<Real>, smem, lim);
    k_volume<Real><<<nblk(nmax, 32 * warps), 32 * warps, smem, s>>>(a, vmax, rmax);
    note_launch();
}

}  // namespace

// Slot capacity per bin: a piece of a tet with n candidates is a simple
// polytope with at most n + 3 faces, hence at most 2(n + 3) - 4 = 2n + 2
// vertices; new vertices fill freed slots first, so 2n + 2 slots suffice.
int clip_vmax(int bin) {
    static const int v[RPD_NBINS] = {4, 6, 8, 10, 14, 18, 34, 66};
    return v[bin];
}

void launch_bin_count(const int32_t* cand_cnt, long long nt, int32_t* bin_count, cudaStream_t s, const uint8_t* only) {
    cudaMemsetAsync(bin_count, 0, sizeof(int32_t) * RPD_NBINS, s);
    if (nt == 0) return;
    k_bin_count<<<nblk(nt, 256), 256, 0, s>>>(cand_cnt, nt, bin_count, only);
    note_launch();
}

void launch_bin_pairs(const int32_t* cand_cnt, const int64_t* pair_off, long long nt, int32_t* pair_tet, int32_t* bins,
                      const int32_t* bin_count, int32_t* bin_fill, long long cap, unsigned long long* rcount,
                      unsigned long long* qcount, cudaStream_t s, const uint8_t* only) {
    k_bin_prefix<<<1, 1, 0, s>>>(bin_count, bin_fill, rcount, qcount);
    note_launch();
    if (nt == 0) return;
    k_bin_pairs<<<nblk(nt, 256), 256, 0, s>>>(cand_cnt, pair_off, nt, pair_tet, bins, bin_fill, cap, only);
    note_launch();
}

void launch_whole_tets(const ClipArgs& a, const int32_t* pairs, const int32_t* d_n, long long nmax, cudaStream_t s) {
    if (nmax <= 0) return;
    k_whole<<<grid_for(nmax, 256), 256, 0, s>>>(a, pairs, d_n);
    note_launch();
}

void launch_clip(const ClipArgs& a, int bin, int precision, const int32_t* pairs, const int32_t* d_n, long long n,
                 cudaStream_t s) {
    if (precision == RPD_FP32_FILTERED) {
        switch (bin) {
            case 1: launch_clip_t<float, 6, 4>(a, pairs, d_n, n, s); break;
            case 2: launch_clip_t<float, 8, 4>(a, pairs, d_n, n, s); break;
            case 3: launch_clip_t<float, 10, 4>(a, pairs, d_n, n, s); break;
            case 4: launch_clip_t<float, 14, 4>(a, pairs, d_n, n, s); break;
            case 5: launch_clip_t<float, 18, 4>(a, pairs, d_n, n, s); break;
            case 6: launch_clip_t<float, 34, 2>(a, pairs, d_n, n, s); break;
            case 7: launch_clip_t<float, 66, 1>(a, pairs, d_n, n, s); break;
        }
    } else {
        switch (bin) {
            case 1: launch_clip_t<double, 6, 4>(a, pairs, d_n, n, s); break;
            case 2: launch_clip_t<double, 8, 4>(a, pairs, d_n, n, s); break;
            case 3: launch_clip_t<double, 10, 4>(a, pairs, d_n, n, s); break;
            case 4: launch_clip_t<double, 14, 2>(a, pairs, d_n, n, s); break;
            case 5: launch_clip_t<double, 18, 2>(a, pairs, d_n, n, s); break;
            case 6: launch_clip_t<double, 34, 1>(a, pairs, d_n, n, s); break;
            case 7: launch_clip_t<double, 66, 1>(a, pairs, d_n, n, s); break;
        }
    }
}

template <int VMAX, int WARPS>
void launch_records_t(const ClipArgs& a, long long nmax, cudaStream_t s) {
    if (nmax <= 0) return;
    const size_t smem = (size_t)WARPS * VMAX * 2 * 32 * sizeof(uint32_t);
    k_records<VMAX><<<nblk(nmax, 32 * WARPS), 32 * WARPS, smem, s>>>(a);
    note_launch();
}

void launch_records(const ClipArgs& a, int bin, long long n, cudaStream_t s) {
    switch (bin) {
        case 1: launch_records_t<6, 4>(a, n, s); break;
        case 2: launch_records_t<8, 4>(a, n, s); break;
        case 3: launch_records_t<10, 4>(a, n, s); break;
        case 4: launch_records_t<14, 4>(a, n, s); break;
        case 5: launch_records_t<18, 4>(a, n, s); break;
        case 6: launch_records_t<34, 4>(a, n, s); break;
        case 7: launch_records_t<66, 2>(a, n, s); break;
        default: break;
    }
}

void launch_volume(const ClipArgs& a, int bin, int precision, long long n, cudaStream_t s) {
    if (bin < 1) return;
    static const int rmax[RPD_NBINS] = {1, 2, 3, 4, 6, 8, 16, 32};   // most candidates of a bin's tets
    const int vw = bin <= 5 ? 4 : (bin == 6 ? 2 : 1);
    if (precision == RPD_FP32_FILTERED) launch_volume_t<float>(a, clip_vmax(bin), rmax[bin], vw, n, s);
    else launch_volume_t<double>(a, clip_vmax(bin), rmax[bin], vw, n, s);
}

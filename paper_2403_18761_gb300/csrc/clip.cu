// A3-A4: Tet-Cell clipping of every candidate (tet, sphere) pair with the
// fractional Euler characteristic emitted on the fly.
//
// Sec. 5.2 (Tet-Cell): the piece P(t,i) = t cap cell_i is computed for every
// (tet, sphere) pair independently, by clipping t with the radical
// half-spaces {pd(x,i) <= pd(x,k)} of the other spheres k (Sec. 4.1.2).  The
// polytope is stored as in the paper's data structure (Sec. 5.2): a list of
// planes and one integer triplet of plane ids per vertex.  Triplets are kept
// consistently oriented so that they form a closed triangulated surface in
// the dual; a clip removes the triangles of the outside vertices and closes
// the hole with a fan of new triplets on the new plane.
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

#include "exact.cuh"
#include "internal.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename Real>
struct PrecTraits;
template <>
struct PrecTraits<float> {
    static constexpr int VW = 7;   // words per vertex: trip, C0..C3, bound, spare
    __device__ static float u() { return 0x1p-24f; }
};
template <>
struct PrecTraits<double> {
    static constexpr int VW = 11;  // trip, C0..C3 (8 words), bound (2 words)
    __device__ static double u() { return 0x1p-53; }
};

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

// Scale a row by a power of two so that every |entry| < 1.
template <typename Real>
__device__ __forceinline__ void scale_row(const long long F[4], Real R[4]) {
    unsigned long long m = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) m = max(m, (unsigned long long)(F[k] < 0 ? -F[k] : F[k]));
    int e = m ? 64 - __clzll(m) : 0;
    Real sc = (Real)ldexp(1.0, -e);
#pragma unroll
    for (int k = 0; k < 4; k++) R[k] = (Real)F[k] * sc;
}

// Decode a triplet word: plane ids in bytes 0..2.
__device__ __forceinline__ void unpack3(uint32_t tw, int& a, int& b, int& c) {
    a = tw & 0xff;
    b = (tw >> 8) & 0xff;
    c = (tw >> 16) & 0xff;
}
__device__ __forceinline__ uint32_t pack3(int a, int b, int c) { return (uint32_t)a | ((uint32_t)b << 8) | ((uint32_t)c << 16); }

// Free columns (ascending) and bisector planes of a triplet; returns m.
__device__ __forceinline__ int split_planes(int a, int b, int c, int* fc, int* bis) {
    int pl[3] = {a, b, c};
    unsigned fmask = 0;
    int m = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (pl[k] < 4) fmask |= 1u << pl[k];
        else bis[m++] = pl[k];
    }
    int nf = 0;
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (!(fmask & (1u << k))) fc[nf++] = k;
    return m;
}

// Cofactor vector (over the free columns, scattered to 4 entries) of m scaled
// rows, in floating point.
template <typename Real>
__device__ __forceinline__ void cof_real(int m, const Real (*R)[4], const int* fc, Real C[4]) {
    C[0] = C[1] = C[2] = C[3] = (Real)0;
    if (m == 1) {
        C[fc[0]] = R[0][fc[1]];
        C[fc[1]] = -R[0][fc[0]];
    } else if (m == 2) {
        Real x0 = R[0][fc[0]], x1 = R[0][fc[1]], x2 = R[0][fc[2]];
        Real y0 = R[1][fc[0]], y1 = R[1][fc[1]], y2 = R[1][fc[2]];
        C[fc[0]] = fma(x1, y2, -(x2 * y1));
        C[fc[1]] = fma(x2, y0, -(x0 * y2));
        C[fc[2]] = fma(x0, y1, -(x1 * y0));
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            int c0 = k == 0 ? 1 : 0;
            int c1 = k <= 1 ? 2 : 1;
            int c2 = k <= 2 ? 3 : 2;
            Real m0 = fma(R[1][c1], R[2][c2], -(R[1][c2] * R[2][c1]));
            Real m1 = fma(R[1][c0], R[2][c2], -(R[1][c2] * R[2][c0]));
            Real m2 = fma(R[1][c0], R[2][c1], -(R[1][c1] * R[2][c0]));
            Real d = fma(R[0][c0], m0, fma(-R[0][c1], m1, R[0][c2] * m2));
            C[k] = (k & 1) ? -d : d;
        }
    }
}

// Absolute error bound of each cofactor entry for rows with |entry| < 1.
template <typename Real>
__device__ __forceinline__ Real cof_err(int m) {
    const Real u = PrecTraits<Real>::u();
    return m == 1 ? 2 * u : (m == 2 ? 16 * u : 96 * u);
}

// Bound on |computed F.C - exact| for a scaled row F (|F| < 1).
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

// Exact-or-FP64 sign of (F_u . C) * sign(sum C) for the vertex on planes
// (a,b,c); F_u == nullptr asks for sign(sum C) alone.  Returns 0 only when the
// exact value is zero (degenerate input).
__device__ __noinline__ int slow_sign(const Lane& L, const Slow& S, int a, int b, int c, const long long* Fu,
                                      bool try_fp64, unsigned& n64, unsigned& nex) {
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

// ------------------------------------------------------------ smem access
template <typename Real, int VMAX>
struct Store {
    uint32_t* base;   // this warp's region: [VMAX][VW][32]
    int lane;
    static constexpr int VW = PrecTraits<Real>::VW;
    __device__ __forceinline__ uint32_t& w(int v, int k) const { return base[(v * VW + k) * 32 + lane]; }
    __device__ __forceinline__ uint32_t trip(int v) const { return w(v, 0); }
    __device__ __forceinline__ void set_trip(int v, uint32_t t) const { w(v, 0) = t; }
    __device__ __forceinline__ void put_real(int v, int k, float x) const { w(v, 1 + k) = __float_as_uint(x); }
    __device__ __forceinline__ void put_real(int v, int k, double x) const {
        unsigned long long b = __double_as_longlong(x);
        w(v, 1 + 2 * k) = (uint32_t)b;
        w(v, 2 + 2 * k) = (uint32_t)(b >> 32);
    }
    __device__ __forceinline__ void get_real(int v, int k, float& x) const { x = __uint_as_float(w(v, 1 + k)); }
    __device__ __forceinline__ void get_real(int v, int k, double& x) const {
        unsigned long long b = (unsigned long long)w(v, 1 + 2 * k) | ((unsigned long long)w(v, 2 + 2 * k) << 32);
        x = __longlong_as_double(b);
    }
    // chart coordinates (3 doubles) reuse words 1..6
    __device__ __forceinline__ void put_beta(int v, int k, double x) const {
        unsigned long long b = __double_as_longlong(x);
        w(v, 1 + 2 * k) = (uint32_t)b;
        w(v, 2 + 2 * k) = (uint32_t)(b >> 32);
    }
    __device__ __forceinline__ double get_beta(int v, int k) const {
        unsigned long long b = (unsigned long long)w(v, 1 + 2 * k) | ((unsigned long long)w(v, 2 + 2 * k) << 32);
        return __longlong_as_double(b);
    }
    __device__ __forceinline__ void copy(int dst, int src) const {
#pragma unroll
        for (int k = 0; k < VW; k++) w(dst, k) = w(src, k);
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

// Does triplet (a,b,c) contain the directed edge x -> y?
__device__ __forceinline__ bool has_dir(int a, int b, int c, int x, int y) {
    return (a == x && b == y) || (b == x && c == y) || (c == x && a == y);
}
__device__ __forceinline__ bool has_plane(int a, int b, int c, int p) { return a == p || b == p || c == p; }

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

// ----------------------------------------------------------- clip kernel
template <typename Real, int VMAX>
__device__ __forceinline__ void clip_one(const ClipArgs& A, const int32_t* __restrict__ pairs, long long q, bool active,
                                         const Store<Real, VMAX>& V) {
    Lane L;
    long long p = 0;
    int nv = 0;
    bool alive = active, whole = true, degenerate = false;
    unsigned nfast = 0, n64 = 0, nex = 0;
    const Slow S{A.Ci, A.W, A.st};
    if (active) {
        p = pairs[q];
        L.t = A.pair_tet[p];
        L.si = (int)(p - A.pair_off[L.t]);
        L.n = A.cand_cnt[L.t];
        L.cand = A.cand + L.t * RPD_MAXC;
        L.i = L.cand[L.si];
        L.own = A.own[L.t];
        int3 ci = ld_int3(A.Ci, L.i);
        long long wi = A.W[L.i];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            L.X[k] = ld_int3(A.Xi, A.tets[4 * L.t + k]);
            L.di[k] = pd_exact(L.X[k], ci, wi);
        }
        // the tet: corner a lies on the three faces != a (oriented triplets)
        V.set_trip(0, pack3(1, 2, 3));
        V.set_trip(1, pack3(0, 3, 2));
        V.set_trip(2, pack3(0, 1, 3));
        V.set_trip(3, pack3(0, 2, 1));
        nv = 4;
    }
    // ---------------------------------------------------------- clipping
    for (int s = 0; alive && s < L.n; s++) {
        if (s == L.si) continue;
        long long F[4];
        row_i64(L, A.Ci, A.W, s, F);
        bool allneg = F[0] < 0 && F[1] < 0 && F[2] < 0 && F[3] < 0;
        if (allneg) continue;                            // plane misses the tet
        if (F[0] > 0 && F[1] > 0 && F[2] > 0 && F[3] > 0) {
            alive = false;                               // tet entirely in cell s
            break;
        }
        Real Fr[4];
        scale_row<Real>(F, Fr);
        const int l = 4 + s;
        unsigned long long out0 = 0, out1 = 0;
        int nout = 0;
        for (int v = 0; v < nv; v++) {
            int a, b, c;
            unpack3(V.trip(v), a, b, c);
            int sg;
            if (a < 4 && b < 4 && c < 4) {
                long long fv = F[6 - a - b - c];
                sg = (fv > 0) - (fv < 0);
            } else {
                Real C0, C1, C2, C3, B;
                V.get_real(v, 0, C0);
                V.get_real(v, 1, C1);
                V.get_real(v, 2, C2);
                V.get_real(v, 3, C3);
                V.get_real(v, 4, B);
                Real val = fma(Fr[0], C0, fma(Fr[1], C1, fma(Fr[2], C2, Fr[3] * C3)));
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
        if (nout == nv) {
            alive = false;
            break;
        }
        whole = false;
        // boundary edges of the removed region -> new vertices (x, y, l)
        int nnew = 0;
        for (int r = 0; r < nv && alive; r++) {
            bool isout = r < 64 ? ((out0 >> r) & 1) : ((out1 >> (r - 64)) & 1);
            if (!isout) continue;
            int a, b, c;
            unpack3(V.trip(r), a, b, c);
            const int ex[3] = {a, b, c}, ey[3] = {b, c, a};
            for (int e = 0; e < 3; e++) {
                int x = ex[e], y = ey[e];
                int twin = -1;
                for (int w = 0; w < nv; w++) {
                    int a2, b2, c2;
                    unpack3(V.trip(w), a2, b2, c2);
                    if (has_dir(a2, b2, c2, y, x)) {
                        twin = w;
                        break;
                    }
                }
                if (twin < 0) continue;
                bool twin_out = twin < 64 ? ((out0 >> twin) & 1) : ((out1 >> (twin - 64)) & 1);
                if (twin_out) continue;
                int dst = nv + nnew;
                if (dst >= VMAX) {
                    dev_fail(A.st, RPD_E_OVERFLOW, CNT_CAPACITY);
                    alive = false;
                    break;
                }
                nnew++;
                V.set_trip(dst, pack3(x, y, l));
                // homogeneous barycentric coordinates of the new vertex
                int fc[4], bis[3];
                int m = split_planes(x, y, l, fc, bis);
                Real R[3][4];
                for (int k = 0; k < m; k++) {
                    if (bis[k] == l) {
                        for (int z = 0; z < 4; z++) R[k][z] = Fr[z];
                    } else {
                        long long Fk[4];
                        row_i64(L, A.Ci, A.W, bis[k] - 4, Fk);
                        scale_row<Real>(Fk, R[k]);
                    }
                }
                Real C[4];
                cof_real<Real>(m, R, fc, C);
                const Real u = PrecTraits<Real>::u();
                Real sum = C[0] + C[1] + C[2] + C[3];
                Real sa = fabs(C[0]) + fabs(C[1]) + fabs(C[2]) + fabs(C[3]);
                Real bs = ((Real)(m + 1) * cof_err<Real>(m) + 4 * u * sa) * (1 + 8 * u);
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
                if (ss < 0)
                    for (int z = 0; z < 4; z++) C[z] = -C[z];
                for (int z = 0; z < 4; z++) V.put_real(dst, z, C[z]);
                V.put_real(dst, 4, dot_bound<Real>(m, C));
            }
        }
        if (!alive) break;
        // compact: keep inside vertices and append the new ones
        int wpos = 0;
        for (int r = 0; r < nv + nnew; r++) {
            bool isout = r < nv && (r < 64 ? ((out0 >> r) & 1) : ((out1 >> (r - 64)) & 1));
            if (isout) continue;
            if (r != wpos) V.copy(wpos, r);
            wpos++;
        }
        nv = wpos;
    }
    if (degenerate) dev_fail(A.st, RPD_E_DEGENERATE, CNT_DEGENERATE);
    if (active && nv < 4) alive = false;
    dev_count(A.st, CNT_PRED_FAST, nfast);
    dev_count(A.st, CNT_PRED_FP64, n64);
    dev_count(A.st, CNT_PRED_EXACT, nex);

    // --------------------------------------------- fractional Euler records
    const int b = A.key_bits;
    unsigned long long fmask = 0;   // planes present as faces
    unsigned nF = 0, nE = 0, nV = 0;
    if (alive) {
        for (int v = 0; v < nv; v++) {
            int a, bb, c;
            unpack3(V.trip(v), a, bb, c);
            fmask |= (1ull << a) | (1ull << bb) | (1ull << c);
            // radical vertex (3 bisectors, all of larger index)
            if (a >= 4 && bb >= 4 && c >= 4 && L.cand[a - 4] > L.i && L.cand[bb - 4] > L.i && L.cand[c - 4] > L.i) nV++;
            // radical edges x<y (directed edge counted once)
            const int ex[3] = {a, bb, c}, ey[3] = {bb, c, a};
            for (int e = 0; e < 3; e++)
                if (ex[e] < ey[e] && ex[e] >= 4 && L.cand[ex[e] - 4] > L.i && L.cand[ey[e] - 4] > L.i) nE++;
        }
        for (int pl = 4; pl < 4 + L.n; pl++)
            if (((fmask >> pl) & 1) && L.cand[pl - 4] > L.i) nF++;
    }
    long long fb = warp_reserve(nF, &A.rcount[0]);
    long long eb = warp_reserve(nE, &A.rcount[1]);
    long long vb = warp_reserve(nV, &A.rcount[2]);
    if (active) {
        A.pflag[p] = alive ? 1 : 0;
        A.f_off[p] = (int32_t)fb;
        A.f_cnt[p] = (uint8_t)nF;
        A.e_off[p] = (int32_t)eb;
        A.e_cnt[p] = (uint8_t)nE;
    }
    if (!alive) {
        if (active) {
            A.c_val[p] = 0;
            A.c_link[p] = 0;
            A.p_vol[p] = 0.0;
            A.p_mom[3 * p] = A.p_mom[3 * p + 1] = A.p_mom[3 * p + 2] = 0.0;
        }
        return;
    }
    const int32_t* adj = A.adj + 4 * L.t;
    // RPC contribution and links
    {
        int sv = 0, se = 0, sf = 0;
        for (int v = 0; v < nv; v++) {
            int a, bb, c;
            unpack3(V.trip(v), a, bb, c);
            sv += carrier_weight(fbits(a) | fbits(bb) | fbits(c), L.own);
            const int ex[3] = {a, bb, c}, ey[3] = {bb, c, a};
            for (int e = 0; e < 3; e++)
                if (ex[e] < ey[e]) se += carrier_weight(fbits(ex[e]) | fbits(ey[e]), L.own);
        }
        unsigned lk = 0;
        for (int f = 0; f < 4; f++)
            if ((fmask >> f) & 1) {
                sf += carrier_weight(1u << f, L.own);
                if (adj[f] >= 0) lk |= 1u << f;
            }
        sf += __popcll(fmask >> 4);   // radical faces are interior (weight 1)
        A.c_val[p] = sv - se + sf - 1;
        A.c_link[p] = (uint8_t)lk;
    }
    // RPF records: face on the radical plane of sphere j > i
    {
        long long w = fb;
        for (int pl = 4; pl < 4 + L.n; pl++) {
            if (!((fmask >> pl) & 1)) continue;
            int j = L.cand[pl - 4];
            if (j <= L.i) continue;
            int sv = 0, se = 0;
            unsigned lk = 0;
            for (int v = 0; v < nv; v++) {
                int a, bb, c;
                unpack3(V.trip(v), a, bb, c);
                if (!has_plane(a, bb, c, pl)) continue;
                sv += carrier_weight(fbits(a) | fbits(bb) | fbits(c), L.own);
                const int ex[3] = {a, bb, c}, ey[3] = {bb, c, a};
                for (int e = 0; e < 3; e++) {
                    int x = ex[e], y = ey[e];
                    if (x < y && (x == pl || y == pl)) {
                        int other = x == pl ? y : x;
                        se += carrier_weight(fbits(other), L.own);
                        if (other < 4 && adj[other] >= 0) lk |= 1u << other;
                    }
                }
            }
            if (w < A.rcap[0]) {
                A.rkey[0][w] = ((unsigned long long)L.i << b) | (unsigned long long)j;
                A.rtet[0][w] = (int32_t)L.t;
                A.rval[0][w] = (int16_t)(sv - se + 1);
                A.rlink[0][w] = (uint8_t)lk;
            }
            w++;
        }
    }
    // RPE records (edges on two radical planes) and RPV records
    {
        long long w = eb, wv = vb;
        for (int v = 0; v < nv; v++) {
            int a, bb, c;
            unpack3(V.trip(v), a, bb, c);
            const int ex[3] = {a, bb, c}, ey[3] = {bb, c, a}, ez[3] = {c, a, bb};
            for (int e = 0; e < 3; e++) {
                int x = ex[e], y = ey[e];
                if (!(x < y && x >= 4)) continue;
                int j = L.cand[x - 4], k = L.cand[y - 4];
                if (j <= L.i || k <= L.i) continue;
                // the other endpoint holds the directed edge y -> x
                int twin = -1, tz = -1;
                for (int u2 = 0; u2 < nv && twin < 0; u2++) {
                    int a2, b2, c2;
                    unpack3(V.trip(u2), a2, b2, c2);
                    if (has_dir(a2, b2, c2, y, x)) {
                        twin = u2;
                        tz = (a2 != x && a2 != y) ? a2 : ((b2 != x && b2 != y) ? b2 : c2);
                    }
                }
                if (twin < 0) continue;
                int z = ez[e];
                int sv = carrier_weight(fbits(z), L.own) + carrier_weight(fbits(tz), L.own);
                unsigned lk = 0;
                if (z < 4 && adj[z] >= 0) lk |= 1u << z;
                if (tz >= 0 && tz < 4 && adj[tz] >= 0) lk |= 1u << tz;
                int lo = min(j, k), hi = max(j, k);
                if (w < A.rcap[1]) {
                    A.rkey[1][w] = ((unsigned long long)L.i << (2 * b)) | ((unsigned long long)lo << b) |
                                   (unsigned long long)hi;
                    A.rtet[1][w] = (int32_t)L.t;
                    A.rval[1][w] = (int16_t)(sv - 1);
                    A.rlink[1][w] = (uint8_t)lk;
                }
                w++;
            }
            if (a >= 4 && bb >= 4 && c >= 4) {
                int j = L.cand[a - 4], k = L.cand[bb - 4], m3 = L.cand[c - 4];
                if (j > L.i && k > L.i && m3 > L.i) {
                    int s0 = min(j, min(k, m3)), s2 = max(j, max(k, m3)), s1 = j + k + m3 - s0 - s2;
                    if (wv < A.rcap[2] && 4 * b <= 64) {
                        A.rkey[2][wv] = ((unsigned long long)L.i << (3 * b)) | ((unsigned long long)s0 << (2 * b)) |
                                        ((unsigned long long)s1 << b) | (unsigned long long)s2;
                        A.rtet[2][wv] = (int32_t)L.t;
                        A.rval[2][wv] = 1;
                        A.rlink[2][wv] = 0;
                    }
                    wv++;
                }
            }
        }
    }
    // ------------------------------------------------ volume and moment (FP64)
    const double vol6 = tet_volume6(L.X);    // 6 vol(t), grid units
    const double u3 = A.unit * A.unit * A.unit;
    if (whole) {
        double vt = vol6 / 6.0;
        A.p_vol[p] = vt * u3;
        for (int k = 0; k < 3; k++) {
            double cx = 0.25 * ((double)(&L.X[0].x)[k] + (&L.X[1].x)[k] + (&L.X[2].x)[k] + (&L.X[3].x)[k]);
            A.p_mom[3 * p + k] = vt * cx * u3 * A.unit;
        }
        return;
    }
    // chart coordinates beta_1..3 of every vertex (exact rows, FP64 cofactors)
    for (int v = 0; v < nv; v++) {
        int a, bb, c;
        unpack3(V.trip(v), a, bb, c);
        double beta[4] = {0, 0, 0, 0};
        int fc[4], bis[3];
        int m = split_planes(a, bb, c, fc, bis);
        if (m == 0) {
            beta[6 - a - bb - c] = 1.0;
        } else {
            double Rd[3][4], Cd[4];
            for (int k = 0; k < m; k++) {
                long long Fk[4];
                row_i64(L, A.Ci, A.W, bis[k] - 4, Fk);
                scale_row<double>(Fk, Rd[k]);
            }
            cof_real<double>(m, Rd, fc, Cd);
            double sum = Cd[0] + Cd[1] + Cd[2] + Cd[3];
            double inv = 1.0 / sum;
            for (int z = 0; z < 4; z++) beta[z] = Cd[z] * inv;
        }
        V.put_beta(v, 0, beta[1]);
        V.put_beta(v, 1, beta[2]);
        V.put_beta(v, 2, beta[3]);
    }
    int a0, b0, c0;
    unpack3(V.trip(0), a0, b0, c0);
    const double O[3] = {V.get_beta(0, 0), V.get_beta(0, 1), V.get_beta(0, 2)};
    double S0 = 0, S1 = 0, S2 = 0, S3 = 0;
    for (int v = 1; v < nv; v++) {
        int a, bb, c;
        unpack3(V.trip(v), a, bb, c);
        const int ex[3] = {a, bb, c}, ey[3] = {bb, c, a};
        for (int e = 0; e < 3; e++) {
            int pf = ex[e], qf = ey[e];
            if (has_plane(a0, b0, c0, pf)) continue;          // face through the apex
            int R = -1, twin = -1;
            for (int u2 = 0; u2 < nv && (R < 0 || twin < 0); u2++) {
                int a2, b2, c2;
                unpack3(V.trip(u2), a2, b2, c2);
                if (R < 0 && has_plane(a2, b2, c2, pf)) R = u2;
                if (twin < 0 && has_dir(a2, b2, c2, qf, pf)) twin = u2;
            }
            if (v == R || twin == R || twin < 0) continue;
            double P1[3], P2[3], P3[3];
            for (int k = 0; k < 3; k++) {
                P1[k] = V.get_beta(v, k) - O[k];
                P2[k] = V.get_beta(twin, k) - O[k];
                P3[k] = V.get_beta(R, k) - O[k];
            }
            double d = P1[0] * (P2[1] * P3[2] - P2[2] * P3[1]) - P1[1] * (P2[0] * P3[2] - P2[2] * P3[0]) +
                       P1[2] * (P2[0] * P3[1] - P2[1] * P3[0]);
            S0 += d;
            S1 += d * (4 * O[0] + P1[0] + P2[0] + P3[0]);
            S2 += d * (4 * O[1] + P1[1] + P2[1] + P3[1]);
            S3 += d * (4 * O[2] + P1[2] + P2[2] + P3[2]);
        }
    }
    double sgn = S0 < 0 ? -1.0 : 1.0;
    double vt = vol6 / 6.0;
    double vol = vt * fabs(S0);
    const double Sc[3] = {S1 * sgn, S2 * sgn, S3 * sgn};
    A.p_vol[p] = vol * u3;
    for (int k = 0; k < 3; k++) {
        double x0 = (double)(&L.X[0].x)[k];
        double acc = vol * x0;
        for (int cc = 1; cc <= 3; cc++) acc += vt * ((double)(&L.X[cc].x)[k] - x0) * Sc[cc - 1] * 0.25;
        A.p_mom[3 * p + k] = acc * u3 * A.unit;
    }
}

template <typename Real, int VMAX>
__global__ void __launch_bounds__(128) k_clip(ClipArgs A, const int32_t* __restrict__ pairs,
                                              const int32_t* __restrict__ d_n) {
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Store<Real, VMAX> V{smem + (size_t)warp * VMAX * PrecTraits<Real>::VW * 32, lane};
    const long long n = *d_n;
    // grid-stride over pairs; q0 is warp-uniform so warp collectives stay converged
    for (long long q0 = (long long)blockIdx.x * blockDim.x + warp * 32; q0 < n;
         q0 += (long long)gridDim.x * blockDim.x) {
        long long q = q0 + lane;
        clip_one<Real, VMAX>(A, pairs, q, q < n, V);
        __syncwarp();
    }
}

// Whole-tet pieces: a tet with a single candidate lies inside one cell.
__device__ __forceinline__ void whole_one(const ClipArgs& A, long long p) {
    long long t = A.pair_tet[p];
    uint32_t own = A.own[t];
    int3 X[4];
    for (int k = 0; k < 4; k++) X[k] = ld_int3(A.Xi, A.tets[4 * t + k]);
    const int32_t* adj = A.adj + 4 * t;
    unsigned lk = 0;
    for (int f = 0; f < 4; f++)
        if (adj[f] >= 0) lk |= 1u << f;
    A.pflag[p] = 1;
    A.c_val[p] = __popc(own & 0xfu) - __popc(own & 0x3f0u) + __popc(own & 0x3c00u) - 1;
    A.c_link[p] = (uint8_t)lk;
    A.f_off[p] = 0;
    A.f_cnt[p] = 0;
    A.e_off[p] = 0;
    A.e_cnt[p] = 0;
    double vt = tet_volume6(X) / 6.0;
    double u3 = A.unit * A.unit * A.unit;
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

__device__ __forceinline__ int bin_of(int n) {
    return n <= 1 ? 0 : (n <= 4 ? 1 : (n <= 8 ? 2 : (n <= 16 ? 3 : 4)));
}

__global__ void k_bin_pairs(const int32_t* __restrict__ cand_cnt, const int64_t* __restrict__ pair_off, long long nt,
                            int32_t* __restrict__ pair_tet, int32_t* __restrict__ bins, long long stride,
                            int32_t* __restrict__ bin_count) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int n = t < nt ? cand_cnt[t] : 0;
    int b = bin_of(n);
    // warp-aggregated reservation per bin
    unsigned peers = __match_any_sync(0xffffffffu, n > 0 ? b : -1);
    int lane = threadIdx.x & 31;
    unsigned lt = peers & ((1u << lane) - 1u);
    // prefix of n over lower peers
    int pre = 0, tot = 0;
    for (int k = 0; k < 32; k++) {
        int nk = __shfl_sync(0xffffffffu, n, k);
        if ((peers >> k) & 1) {
            tot += nk;
            if ((lt >> k) & 1) pre += nk;
        }
    }
    int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader && n > 0 && tot > 0) base = atomicAdd(&bin_count[b], tot);
    base = __shfl_sync(0xffffffffu, base, leader);
    if (n <= 0) return;
    long long off = pair_off[t];
    for (int k = 0; k < n; k++) {
        pair_tet[off + k] = (int32_t)t;
        bins[(long long)b * stride + base + pre + k] = (int32_t)(off + k);
    }
}

inline unsigned grid_for(long long n, int tpb) {
    long long b = (n + tpb - 1) / tpb;
    const long long cap = 152LL * 64;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename Real, int VMAX, int WARPS>
void launch_clip_t(const ClipArgs& a, const int32_t* pairs, const int32_t* d_n, long long n, cudaStream_t s) {
    if (n <= 0) return;
    size_t smem = (size_t)WARPS * VMAX * PrecTraits<Real>::VW * 32 * sizeof(uint32_t);
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_clip<Real, VMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    k_clip<Real, VMAX><<<grid_for(n, 32 * WARPS), 32 * WARPS, smem, s>>>(a, pairs, d_n);
}

}  // namespace

void launch_bin_pairs(const int32_t* cand_cnt, const int64_t* pair_off, long long nt, int32_t* pair_tet, int32_t* bins,
                      long long bin_stride, int32_t* bin_count, cudaStream_t s) {
    cudaMemsetAsync(bin_count, 0, sizeof(int32_t) * RPD_NBINS, s);
    if (nt == 0) return;
    k_bin_pairs<<<nblk(nt, 256), 256, 0, s>>>(cand_cnt, pair_off, nt, pair_tet, bins, bin_stride, bin_count);
}

void launch_whole_tets(const ClipArgs& a, const int32_t* pairs, const int32_t* d_n, long long nmax, cudaStream_t s) {
    if (nmax <= 0) return;
    k_whole<<<grid_for(nmax, 256), 256, 0, s>>>(a, pairs, d_n);
}

// Vertex capacity per bin: a piece of a tet with n candidates has at most
// 2n vertices before a clip and the new face adds at most n + 2, so 3n + 2
// slots always suffice.
void launch_clip(const ClipArgs& a, int bin, int precision, const int32_t* pairs, const int32_t* d_n, long long n,
                 cudaStream_t s) {
    if (precision == RPD_FP32_FILTERED) {
        switch (bin) {
            case 1: launch_clip_t<float, 14, 4>(a, pairs, d_n, n, s); break;
            case 2: launch_clip_t<float, 26, 4>(a, pairs, d_n, n, s); break;
            case 3: launch_clip_t<float, 50, 2>(a, pairs, d_n, n, s); break;
            case 4: launch_clip_t<float, 98, 1>(a, pairs, d_n, n, s); break;
        }
    } else {
        switch (bin) {
            case 1: launch_clip_t<double, 14, 4>(a, pairs, d_n, n, s); break;
            case 2: launch_clip_t<double, 26, 2>(a, pairs, d_n, n, s); break;
            case 3: launch_clip_t<double, 50, 1>(a, pairs, d_n, n, s); break;
            case 4: launch_clip_t<double, 98, 1>(a, pairs, d_n, n, s); break;
        }
    }
}

// Geometric preservation (Sec. 4.3): distance from surface samples to the
// enveloping volume of the medial mesh.
//
// The medial mesh's primitives (Sec. 3.1, 3.2) are its vertices (spheres
// m_i = (c_i, r_i), one per RPC), its edges (medial cones, the spheres
// interpolated linearly between two vertices, one per RPF) and its triangles
// (medial slabs, interpolated between three, one per RPE).  The signed
// distance of a point s to a primitive is the minimum over its interpolated
// spheres of |s - c| - r; the sample's distance is the minimum over all
// primitives (negative inside the envelope).  Sec. 4.3 inserts a sphere at a
// sample whose distance exceeds delta times the bounding-box diagonal.
//
// |s - c(l)| - r(l) is convex in the interpolation weights l, so its minimum
// over a cone or slab is either at an interior stationary point or on the
// primitive's boundary, which is made of lower primitives (a cone's ends are
// spheres, a slab's edges are cones; every edge of an RPE is an RPF, every
// end of an RPF an RPC).  So each primitive contributes only its interior
// stationary point, found in closed form:
//  * cone (c1, r1) -> (c2, r2), axis u = (c2 - c1) / L, slope k = (r2 - r1) / L,
//    s at axial coordinate x and radial distance y from the axis: the
//    stationary point is at axial coordinate z = x + k y / sqrt(1 - k^2);
//    it counts when 0 < z < L (and |k| < 1);
//  * slab: the unit vector v from c(l) to s satisfies v.(c_j - c_1) = r_1 - r_j
//    (j = 2, 3), i.e. v is the normal of a plane tangent to the three
//    spheres; with v known, c(l) = s - rho v is solved in the plane of the
//    centres; it counts when l lies inside the triangle and rho > 0, and the
//    distance is then v.(s - c_1) - r_1.
//
// FP32 arithmetic on coordinates relative to mesh vertex 0 (the distances
// only decide a threshold); one thread per sample, the samples in Morton
// order, the Morton-sorted primitives staged through shared memory in tiles,
// scanned outwards from the block's position and skipped when their bounding
// ball is already farther than every sample's best distance.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"
#include "prim.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int ENV_THREADS = 256;
constexpr int ENV_TILE = 64;    // primitives per shared-memory tile (64 measured fastest of 64, 128, 256)

// A primitive: up to three spheres (x, y, z, r) and its kind (1, 2, 3).
struct Prim {
    float4 s[3];
    int kind;
};

__device__ __forceinline__ float sphere_d(float3 p, float4 c) {
    const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
    return sqrtf(dx * dx + dy * dy + dz * dz) - c.w;
}

// Interior stationary value of a cone, or +inf.
__device__ __forceinline__ float cone_d(float3 p, float4 a, float4 b) {
    const float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
    const float L2 = ex * ex + ey * ey + ez * ez;
    if (!(L2 > 0)) return INFINITY;
    const float L = sqrtf(L2), k = (b.w - a.w) / L;
    if (!(fabsf(k) < 1.0f)) return INFINITY;
    const float ax = p.x - a.x, ay = p.y - a.y, az = p.z - a.z;
    const float x = (ax * ex + ay * ey + az * ez) / L;
    const float y = sqrtf(fmaxf(ax * ax + ay * ay + az * az - x * x, 0.0f));
    const float z = x + k * y / sqrtf(1.0f - k * k);
    if (!(z > 0 && z < L)) return INFINITY;
    const float t = z / L;
    const float4 c = make_float4(a.x + t * ex, a.y + t * ey, a.z + t * ez, a.w + t * (b.w - a.w));
    return sphere_d(p, c);
}

// Interior stationary value of a slab, or +inf.
__device__ __forceinline__ float slab_d(float3 p, float4 c1, float4 c2, float4 c3) {
    const float3 e2 = make_float3(c2.x - c1.x, c2.y - c1.y, c2.z - c1.z);
    const float3 e3 = make_float3(c3.x - c1.x, c3.y - c1.y, c3.z - c1.z);
    const float g22 = e2.x * e2.x + e2.y * e2.y + e2.z * e2.z, g23 = e2.x * e3.x + e2.y * e3.y + e2.z * e3.z;
    const float g33 = e3.x * e3.x + e3.y * e3.y + e3.z * e3.z;
    const float det = g22 * g33 - g23 * g23;
    if (!(det > 1e-20f * g22 * g33)) return INFINITY;
    // in-plane part w = al e2 + be e3 of v: w.e2 = r1 - r2, w.e3 = r1 - r3
    const float b2 = c1.w - c2.w, b3 = c1.w - c3.w;
    const float al = (b2 * g33 - b3 * g23) / det, be = (b3 * g22 - b2 * g23) / det;
    const float3 w = make_float3(al * e2.x + be * e3.x, al * e2.y + be * e3.y, al * e2.z + be * e3.z);
    const float ww = w.x * w.x + w.y * w.y + w.z * w.z;
    if (!(ww < 1.0f)) return INFINITY;
    float3 n = make_float3(e2.y * e3.z - e2.z * e3.y, e2.z * e3.x - e2.x * e3.z, e2.x * e3.y - e2.y * e3.x);
    const float nn = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
    n = make_float3(n.x / nn, n.y / nn, n.z / nn);
    const float3 a = make_float3(p.x - c1.x, p.y - c1.y, p.z - c1.z);
    const float h = a.x * n.x + a.y * n.y + a.z * n.z;
    const float gm = copysignf(sqrtf(1.0f - ww), h);
    const float3 v = make_float3(w.x + gm * n.x, w.y + gm * n.y, w.z + gm * n.z);
    // c1 + l2 e2 + l3 e3 + rho v = s: rho from the normal component, then the
    // in-plane weights from the 2x2 Gram system
    const float vn = v.x * n.x + v.y * n.y + v.z * n.z;
    if (!(fabsf(vn) > 0)) return INFINITY;
    const float rho = h / vn;
    if (!(rho > 0)) return INFINITY;
    const float3 q = make_float3(a.x - rho * v.x, a.y - rho * v.y, a.z - rho * v.z);
    const float q2 = q.x * e2.x + q.y * e2.y + q.z * e2.z, q3 = q.x * e3.x + q.y * e3.y + q.z * e3.z;
    const float l2 = (q2 * g33 - q3 * g23) / det, l3 = (q3 * g22 - q2 * g23) / det;
    if (!(l2 > 0 && l3 > 0 && l2 + l3 < 1)) return INFINITY;
    return a.x * v.x + a.y * v.y + a.z * v.z - c1.w;
}

__device__ __forceinline__ float prim_d(float3 p, const Prim& q) {
    if (q.kind == 1) return sphere_d(p, q.s[0]);
    if (q.kind == 2) return cone_d(p, q.s[0], q.s[1]);
    return slab_d(p, q.s[0], q.s[1], q.s[2]);
}

// Primitive table: kinds 1..3 from the element keys, sphere data relative to
// the centre `o` (grid units x unit, in FP32).
__global__ void k_env_prims(const int32_t* __restrict__ k1, long long n1, const int32_t* __restrict__ k2, long long n2,
                            const int32_t* __restrict__ k3, long long n3, const int32_t* __restrict__ Ci,
                            const long long* __restrict__ W, double unit, double3 o, Prim* __restrict__ out,
                            uint64_t* __restrict__ morton, uint32_t* __restrict__ idx, int3 gmin, int shift) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n1 + n2 + n3) return;
    Prim q;
    const int32_t* key;
    int kind;
    if (i < n1) {
        kind = 1;
        key = k1 + i;
    } else if (i < n1 + n2) {
        kind = 2;
        key = k2 + 2 * (i - n1);
    } else {
        kind = 3;
        key = k3 + 3 * (i - n1 - n2);
    }
    q.kind = kind;
    long long cx = 0, cy = 0, cz = 0;
    for (int z = 0; z < 3; z++) {
        const int s = key[z < kind ? z : 0];
        const int3 c = ld_int3(Ci, s);
        q.s[z] = make_float4((float)(c.x * unit - o.x), (float)(c.y * unit - o.y), (float)(c.z * unit - o.z),
                             (float)(sqrt((double)W[s]) * unit));
        if (z < kind) {
            cx += c.x;
            cy += c.y;
            cz += c.z;
        }
    }
    out[i] = q;
    // Morton code of the primitive's mean centre (21 bits per axis)
    auto spread = [](unsigned long long v) {
        v &= 0x1fffffull;
        v = (v | v << 32) & 0x1f00000000ffffull;
        v = (v | v << 16) & 0x1f0000ff0000ffull;
        v = (v | v << 8) & 0x100f00f00f00f00full;
        v = (v | v << 4) & 0x10c30c30c30c30c3ull;
        v = (v | v << 2) & 0x1249249249249249ull;
        return v;
    };
    const unsigned long long ux = (unsigned long long)((cx / kind - gmin.x) >> shift);
    const unsigned long long uy = (unsigned long long)((cy / kind - gmin.y) >> shift);
    const unsigned long long uz = (unsigned long long)((cz / kind - gmin.z) >> shift);
    morton[i] = spread(ux) | (spread(uy) << 1) | (spread(uz) << 2);
    idx[i] = (uint32_t)i;
}

// Morton code of a sample (world coordinates), in the primitives' code space.
__device__ __forceinline__ unsigned long long spread21(unsigned long long v) {
    v &= 0x1fffffull;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
}

__global__ void k_env_sample_keys(const double* __restrict__ samples, long long ns, double scale, int3 gmin, int shift,
                                  uint64_t* __restrict__ morton, uint32_t* __restrict__ idx) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    unsigned long long u[3];
    const int gm[3] = {gmin.x, gmin.y, gmin.z};
    for (int a = 0; a < 3; a++) {
        double g = rint(samples[3 * i + a] * scale);
        g = fmin(fmax(g, (double)gm[a]), (double)(-gm[a] - 1));   // inside the code's range
        u[a] = (unsigned long long)(((long long)g - gm[a]) >> shift);
    }
    morton[i] = spread21(u[0]) | (spread21(u[1]) << 1) | (spread21(u[2]) << 2);
    idx[i] = (uint32_t)i;
}

__global__ void k_env_gather(const Prim* __restrict__ in, const uint32_t* __restrict__ order, long long n,
                             Prim* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[order[i]];
}

// Bounding ball (centre, radius) of each tile of sorted primitives: every
// point of a primitive's envelope lies within (distance to the ball centre
// + the sphere radius) of it.
__global__ void k_env_tiles(const Prim* __restrict__ p, long long n, float4* __restrict__ tiles) {
    const long long t = blockIdx.x;
    const long long b = t * ENV_TILE, e = b + ENV_TILE < n ? b + ENV_TILE : n;
    __shared__ float sx, sy, sz;
    if (threadIdx.x == 0) {
        double ax = 0, ay = 0, az = 0;
        for (long long i = b; i < e; i++) {
            ax += p[i].s[0].x;
            ay += p[i].s[0].y;
            az += p[i].s[0].z;
        }
        const double m = (double)(e - b);
        sx = (float)(ax / m);
        sy = (float)(ay / m);
        sz = (float)(az / m);
    }
    __syncthreads();
    float r = 0;
    for (long long i = b + threadIdx.x; i < e; i += blockDim.x)
        for (int z = 0; z < p[i].kind; z++) {
            const float4 c = p[i].s[z];
            const float dx = c.x - sx, dy = c.y - sy, dz = c.z - sz;
            r = fmaxf(r, sqrtf(dx * dx + dy * dy + dz * dz) + c.w);
        }
    for (int off = 16; off; off >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, off));
    __shared__ float wr[32];
    if ((threadIdx.x & 31) == 0) wr[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) m = fmaxf(m, wr[k]);
        tiles[t] = make_float4(sx, sy, sz, m * 1.0001f + 1e-6f);
    }
}

// One thread per sample, the samples taken in Morton order (sorder) so that a
// block's samples are close together; the block starts at the tile of
// primitives whose Morton codes follow its first sample's and alternates
// outwards (t0, t0 + 1, t0 - 1, ...), so the best distances shrink early and
// far tiles fail the ball test.
__global__ void __launch_bounds__(ENV_THREADS) k_env_dist(const double* __restrict__ samples, long long ns, double3 o,
                                                          const Prim* __restrict__ prims, long long np,
                                                          const float4* __restrict__ tiles,
                                                          const uint64_t* __restrict__ pkeys,
                                                          const uint64_t* __restrict__ skeys,
                                                          const uint32_t* __restrict__ sorder, float* __restrict__ dist,
                                                          int32_t* __restrict__ arg) {
    __shared__ Prim tile[ENV_TILE];
    __shared__ int skip;
    __shared__ long long t0s;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = q < ns;
    const long long i = live ? (long long)sorder[q] : 0;
    const float3 p = live ? make_float3((float)(samples[3 * i] - o.x), (float)(samples[3 * i + 1] - o.y),
                                        (float)(samples[3 * i + 2] - o.z))
                          : make_float3(0, 0, 0);
    float best = INFINITY;
    int bi = -1;
    const long long ntile = (np + ENV_TILE - 1) / ENV_TILE;
    if (threadIdx.x == 0) {   // first primitive whose code is >= the block's first sample's
        const uint64_t key = skeys[(long long)blockIdx.x * blockDim.x];
        long long lo = 0, hi = np;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (pkeys[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        t0s = lo < np ? lo / ENV_TILE : ntile - 1;
    }
    __syncthreads();
    const long long t0 = t0s;
    for (long long j = 0; j < 2 * ntile; j++) {
        const long long t = (j & 1) ? t0 + (j + 1) / 2 : t0 - j / 2;   // t0, t0 + 1, t0 - 1, t0 + 2, ...
        if (t < 0 || t >= ntile) continue;   // uniform over the block
        // the block skips a tile whose bounding ball is farther from every
        // live sample than that sample's best distance
        const float4 tb = tiles[t];
        const float dx = p.x - tb.x, dy = p.y - tb.y, dz = p.z - tb.z;
        const bool need = live && (sqrtf(dx * dx + dy * dy + dz * dz) - tb.w < best);
        if (threadIdx.x == 0) skip = 1;
        __syncthreads();
        if (need) skip = 0;
        __syncthreads();
        if (skip) continue;
        const long long b = t * ENV_TILE;
        const int m = (int)(np - b < ENV_TILE ? np - b : ENV_TILE);
        for (int k = threadIdx.x; k < m; k += blockDim.x) tile[k] = prims[b + k];
        __syncthreads();
        if (need)
            for (int k = 0; k < m; k++) {
                const float d = prim_d(p, tile[k]);
                if (d < best) {
                    best = d;
                    bi = (int)(b + k);
                }
            }
        __syncthreads();
    }
    if (live) {
        dist[i] = best;
        arg[i] = bi;
    }
}

__global__ void k_env_unsort(int32_t* __restrict__ arg, long long n, const uint32_t* __restrict__ order) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && arg[i] >= 0) arg[i] = (int32_t)order[arg[i]];
}

}  // namespace

size_t envelope_tmp_bytes(long long np, long long nsamp) {
    const size_t a = ((size_t)np * sizeof(Prim) + 255) & ~(size_t)255;
    const size_t t = (((size_t)(np + ENV_TILE - 1) / ENV_TILE + 1) * sizeof(float4) + 255) & ~(size_t)255;
    const size_t k = ((size_t)(np + 1) * 8 + 255) & ~(size_t)255, v = ((size_t)(np + 1) * 4 + 255) & ~(size_t)255;
    const size_t ks = ((size_t)(nsamp + 1) * 8 + 255) & ~(size_t)255, vs = ((size_t)(nsamp + 1) * 4 + 255) & ~(size_t)255;
    return 2 * a + t + 2 * k + 2 * v + 2 * ks + 2 * vs + radix_tmp_bytes(np > nsamp ? np : nsamp);
}

// Primitive table sorted by the Morton code of the primitive's mean centre,
// its tile bounds, then the distance of every sample (FP32, relative to o).
// prim_id: index into the unsorted table (spheres, then cones, then slabs).
void launch_envelope(const int32_t* k1, long long n1, const int32_t* k2, long long n2, const int32_t* k3, long long n3,
                     const int32_t* Ci, const long long* W, double unit, const double* o3, const double* samples,
                     long long nsamp, float* dist, int32_t* prim_id, void* tmp, int* d_err, cudaStream_t s) {
    const long long np = n1 + n2 + n3;
    if (np <= 0 || nsamp <= 0) return;
    const size_t a = ((size_t)np * sizeof(Prim) + 255) & ~(size_t)255;
    const size_t t = (((size_t)(np + ENV_TILE - 1) / ENV_TILE + 1) * sizeof(float4) + 255) & ~(size_t)255;
    const size_t k = ((size_t)(np + 1) * 8 + 255) & ~(size_t)255, v = ((size_t)(np + 1) * 4 + 255) & ~(size_t)255;
    char* p = (char*)tmp;
    Prim* raw = (Prim*)p;
    p += a;
    Prim* sorted = (Prim*)p;
    p += a;
    float4* tiles = (float4*)p;
    p += t;
    uint64_t* m0 = (uint64_t*)p;
    p += k;
    uint64_t* m1 = (uint64_t*)p;
    p += k;
    uint32_t* i0 = (uint32_t*)p;
    p += v;
    uint32_t* i1 = (uint32_t*)p;
    p += v;
    const size_t ks = ((size_t)(nsamp + 1) * 8 + 255) & ~(size_t)255, vs = ((size_t)(nsamp + 1) * 4 + 255) & ~(size_t)255;
    uint64_t* sk0 = (uint64_t*)p;
    p += ks;
    uint64_t* sk1 = (uint64_t*)p;
    p += ks;
    uint32_t* so0 = (uint32_t*)p;
    p += vs;
    uint32_t* so1 = (uint32_t*)p;
    p += vs;
    const double3 o = make_double3(o3[0], o3[1], o3[2]);
    // grid coordinates are in (-2^21, 2^21): shifted by 2^21 and halved they fit 21 bits
    const int g0 = -(1 << 21);
    k_env_prims<<<nblk(np, 256), 256, 0, s>>>(k1, n1, k2, n2, k3, n3, Ci, W, unit, o, raw, m0, i0,
                                               make_int3(g0, g0, g0), 1);
    note_launch();
    radix_sort_pairs(m0, i0, m1, i1, np, 63, p, d_err, s);
    k_env_gather<<<nblk(np, 256), 256, 0, s>>>(raw, i1, np, sorted);
    note_launch();
    const long long ntile = (np + ENV_TILE - 1) / ENV_TILE;
    k_env_tiles<<<(unsigned)ntile, 128, 0, s>>>(sorted, np, tiles);
    note_launch();
    k_env_sample_keys<<<nblk(nsamp, 256), 256, 0, s>>>(samples, nsamp, 1.0 / unit, make_int3(g0, g0, g0), 1, sk0, so0);
    note_launch();
    radix_sort_pairs(sk0, so0, sk1, so1, nsamp, 63, p, d_err, s);
    k_env_dist<<<nblk(nsamp, ENV_THREADS), ENV_THREADS, 0, s>>>(samples, nsamp, o, sorted, np, tiles, m1, sk1, so1, dist,
                                                                  prim_id);
    note_launch();
    k_env_unsort<<<nblk(nsamp, 256), 256, 0, s>>>(prim_id, nsamp, i1);   // sorted positions -> table rows
    note_launch();
}

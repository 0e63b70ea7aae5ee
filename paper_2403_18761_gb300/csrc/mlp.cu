// Learned sphere proposer: a small MLP (3 hidden layers of 128, BF16 weights
// and activations, FP32 accumulation) trained and evaluated on the GPU with
// the library's own kernels.  The paper has no counterpart: it grows every
// sphere by sphere shrinking (Sec. 5.1); here the network proposes the
// radius of the sphere a pin will grow into, the shrinking starts from that
// proposal instead of from a radius above the mesh's extent, and the
// shrinking itself (and the exact RPD check after the insertion) decides.
//
// The dense layers are tile GEMMs on the 5th-generation tensor cores:
// D[128 x N] (TMEM, FP32) += A[128 x K] B[N x K]^T with both operands BF16 in
// shared memory, issued by one thread as tcgen05.mma kind::f16 (M = 128,
// K = 16 per instruction), completion signalled through an mbarrier by
// tcgen05.commit, the accumulator read back by tcgen05.ld for a fused
// epilogue (bias + ReLU, ReLU mask, or FP32 atomic accumulation).  The
// operands are staged by the CTA's threads (transposed where the layer needs
// it) into the canonical no-swizzle K-major layout: 8 rows x 16 bytes per
// core matrix, core matrices consecutive along K (leading byte offset 128)
// and rows of core matrices K * 2 bytes x 8 apart (stride byte offset).
#include <cuda_runtime.h>
#include <math.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "prim.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int TM = 128;                 // rows of a tile (tcgen05 M)
constexpr int MLP_THREADS = 128;        // 4 warps: one per 32 TMEM lanes
constexpr long long MBAR_SPIN_LIMIT = 1ll << 24;

// ----------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: no swizzle, K-major.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);            // start address, bits 0-13
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;        // leading byte offset, bits 16-29
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;        // stride byte offset, bits 32-45
    d |= (uint64_t)1 << 46;                              // descriptor version 1
    return d;                                            // base offset 0, layout SWIZZLE_NONE (0)
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major.
__device__ __forceinline__ uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for phase `phase` of the barrier; false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < MBAR_SPIN_LIMIT; it++) {
        uint32_t done = 0;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; k++) v[k] = __uint_as_float(r[k]);
}

// Byte offset of element (row, k) in a no-swizzle K-major tile of kdim
// columns: core matrix (row / 8, k / 8) at ((row / 8) * (kdim / 8) + k / 8)
// * 128, row % 8 at 16-byte steps, k % 8 at 2-byte steps.
__device__ __forceinline__ uint32_t tile_off(int row, int k, int kdim) {
    return (uint32_t)((((row >> 3) * (kdim >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

// -------------------------------------------------------------- tile GEMM
// Shared memory of one tile: A (128 x K), B (N x K), the barrier and the
// TMEM base address.  K, N <= 128.
struct TileSmem {
    __nv_bfloat16 a[TM * 128];
    __nv_bfloat16 b[128 * 128];
    uint64_t bar;
    uint32_t tmem;
    int err;
};

// Issue the K / 16 MMAs of the staged tile from one thread and wait for
// their completion (every thread waits).  False if the bounded wait ran out.
__device__ __forceinline__ bool tile_mma(TileSmem& S, int K, int N, uint32_t phase) {
    fence_proxy_async();   // staged operands visible to the tensor cores
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (threadIdx.x == 0) {
        const uint32_t idesc = instr_desc(TM, N);
        const uint32_t a0 = smem_u32(S.a), b0 = smem_u32(S.b);
        for (int j = 0; j < K / 16; j++)
            mma_bf16(S.tmem, smem_desc(a0 + 256u * j, 128u, 16u * K), smem_desc(b0 + 256u * j, 128u, 16u * K),
                     idesc, j > 0);
        mma_commit(&S.bar);
    }
    const bool ok = mbar_wait(&S.bar, phase);
    fence_after_sync();
    return ok;
}

__device__ __forceinline__ void tile_begin(TileSmem& S, int ncols) {
    if (threadIdx.x < 32) tmem_alloc(&S.tmem, ncols);
    if (threadIdx.x == 0) {
        mbar_init(&S.bar, 1);
        S.err = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

__device__ __forceinline__ void tile_end(TileSmem& S, int ncols, bool ok, int* err) {
    if (!ok && threadIdx.x == 0) atomicCAS(err, 0, (int)RPD_E_TIMEOUT);
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(S.tmem, ncols);
}

// Stage rows [r0, r0 + 128) x [0, K) of a row-major bf16 matrix (ld columns)
// as an A or B operand (K-major); rows past nrows are zero.
__device__ __forceinline__ void stage_rows(__nv_bfloat16* dst, const __nv_bfloat16* __restrict__ src, long long r0,
                                           long long nrows, int nr, int K, int ld) {
    const int chunks = nr * (K / 8);
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
        const int row = c / (K / 8), kc = (c % (K / 8)) * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (r0 + row < nrows) v = *reinterpret_cast<const uint4*>(src + (r0 + row) * ld + kc);
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(dst) + tile_off(row, kc, K)) = v;
    }
}

// Stage the transpose: operand row i, column j = src[(c0 + j) * ld + i] for
// i < nr (operand rows) and j < K (src rows c0.., zero past nsrc).
__device__ __forceinline__ void stage_cols(__nv_bfloat16* dst, const __nv_bfloat16* __restrict__ src, long long c0,
                                           long long nsrc, int nr, int K, int ld) {
    const int chunks = nr * (K / 8);
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
        const int row = c % nr, kc = (c / nr) * 8;
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const long long sr = c0 + kc + q;
            v[q] = sr < nsrc ? src[sr * ld + row] : __float2bfloat16(0.0f);
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(dst) + tile_off(row, kc, K)) = *reinterpret_cast<uint4*>(v);
    }
}

// Forward: Y[m][n] = relu(sum_k X[m][k] W[n][k] + b[n]) for the CTA's 128 rows.
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_fwd(const __nv_bfloat16* __restrict__ X, long long M, int K,
                                                         const __nv_bfloat16* __restrict__ W,
                                                         const float* __restrict__ bias, int N,
                                                         __nv_bfloat16* __restrict__ Y, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
    const long long m0 = (long long)blockIdx.x * TM;
    tile_begin(S, 128);
    stage_rows(S.a, X, m0, M, TM, K, K);
    stage_rows(S.b, W, 0, N, N, K, K);
    const bool ok = tile_mma(S, K, N, 0);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long m = m0 + 32 * w + lane;
    for (int c0 = 0; c0 < N; c0 += 32) {
        float v[32];
        tmem_ld32(S.tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
        if (ok && m < M) {
            __align__(16) __nv_bfloat16 o[32];
#pragma unroll
            for (int k = 0; k < 32; k++) o[k] = __float2bfloat16(fmaxf(v[k] + bias[c0 + k], 0.0f));
#pragma unroll
            for (int q = 0; q < 4; q++)
                reinterpret_cast<uint4*>(Y + m * N + c0)[q] = reinterpret_cast<const uint4*>(o)[q];
        }
    }
    tile_end(S, 128, ok, err);
}

// Input gradient: dZprev[m][k] = (sum_n dZ[m][n] W[n][k]) * (H[m][k] > 0).
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_dx(const __nv_bfloat16* __restrict__ dZ, long long M, int N,
                                                        const __nv_bfloat16* __restrict__ W, int K,
                                                        const __nv_bfloat16* __restrict__ H,
                                                        __nv_bfloat16* __restrict__ dZprev, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
    const long long m0 = (long long)blockIdx.x * TM;
    tile_begin(S, 128);
    stage_rows(S.a, dZ, m0, M, TM, N, N);    // A: 128 x N (reduction over n)
    stage_cols(S.b, W, 0, N, K, N, K);       // B: K rows x N (B[k][n] = W[n][k])
    const bool ok = tile_mma(S, N, K, 0);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long m = m0 + 32 * w + lane;
    for (int c0 = 0; c0 < K; c0 += 32) {
        float v[32];
        tmem_ld32(S.tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
        if (ok && m < M) {
            __align__(16) __nv_bfloat16 h[32], o[32];
#pragma unroll
            for (int q = 0; q < 4; q++) reinterpret_cast<uint4*>(h)[q] = reinterpret_cast<const uint4*>(H + m * K + c0)[q];
#pragma unroll
            for (int k = 0; k < 32; k++) o[k] = __float2bfloat16(__bfloat162float(h[k]) > 0.0f ? v[k] : 0.0f);
#pragma unroll
            for (int q = 0; q < 4; q++)
                reinterpret_cast<uint4*>(dZprev + m * K + c0)[q] = reinterpret_cast<const uint4*>(o)[q];
        }
    }
    tile_end(S, 128, ok, err);
}

// Weight gradient of the CTA's 128 rows: dW[n][k] += sum_m dZ[m][n] H[m][k].
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_dw(const __nv_bfloat16* __restrict__ dZ, long long M, int N,
                                                        const __nv_bfloat16* __restrict__ H, int K,
                                                        float* __restrict__ dW, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(smem_raw);
    const long long m0 = (long long)blockIdx.x * TM;
    tile_begin(S, 128);
    stage_cols(S.a, dZ, m0, M, N, TM, N);    // A: N rows (n) x 128 (m)
    stage_cols(S.b, H, m0, M, K, TM, K);     // B: K rows (k) x 128 (m)
    const bool ok = tile_mma(S, TM, K, 0);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = 32 * w + lane;
    for (int c0 = 0; c0 < K; c0 += 32) {
        float v[32];
        tmem_ld32(S.tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
        if (ok && n < N)
#pragma unroll
            for (int k = 0; k < 32; k++) atomicAdd(&dW[n * K + c0 + k], v[k]);
    }
    tile_end(S, 128, ok, err);
}

}  // namespace

// ------------------------------------------------------- CUDA-core parts
namespace {

constexpr int HID = 128;   // hidden width
constexpr int NIN = 32;    // padded input width
// parameter offsets in the FP32 master vector
constexpr long long OW0 = 0, OB0 = OW0 + HID * NIN, OW1 = OB0 + HID, OB1 = OW1 + HID * HID, OW2 = OB1 + HID,
                    OB2 = OW2 + HID * HID, OW3 = OB2 + HID, OB3 = OW3 + HID, NPARAM = OB3 + 1;

// fp32 rows [n][n_in] -> bf16 rows [cap][NIN], zero padded.
__global__ void k_to_bf16(const float* __restrict__ x, long long n, int n_in, long long cap,
                          __nv_bfloat16* __restrict__ X) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap * NIN) return;
    const long long r = i / NIN;
    const int c = (int)(i % NIN);
    X[i] = __float2bfloat16(r < n && c < n_in ? x[r * n_in + c] : 0.0f);
}

// Training batch: row r of the batch is row (cur[0] + r) mod n_total of the
// data (cur on the device, so every step is the same launch sequence).
__global__ void k_to_bf16_batch(const float* __restrict__ x, long long n_total, int n_in, long long b, long long cap,
                                const long long* __restrict__ cur, __nv_bfloat16* __restrict__ X) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap * NIN) return;
    const long long r = i / NIN;
    const int c = (int)(i % NIN);
    const long long src = (cur[0] + r) % n_total;
    X[i] = __float2bfloat16(r < b && c < n_in ? x[src * n_in + c] : 0.0f);
}

// After a step: the next batch starts b rows later; one more Adam step.
__global__ void k_cursor_advance(long long* cur, long long b, long long n_total) {
    cur[0] = (cur[0] + b) % n_total;
    cur[1] += 1;
}

__global__ void k_cast_weights(const float* __restrict__ p, __nv_bfloat16* __restrict__ W0,
                               __nv_bfloat16* __restrict__ W1, __nv_bfloat16* __restrict__ W2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < HID * NIN) W0[i] = __float2bfloat16(p[OW0 + i]);
    if (i < HID * HID) {
        W1[i] = __float2bfloat16(p[OW1 + i]);
        W2[i] = __float2bfloat16(p[OW2 + i]);
    }
}

// Output layer on the CUDA cores (one warp per row): y = H2 . w3 + b3; with
// targets, also the mean-squared-error gradient: dy = 2 (y - t) / n,
// dZ2 = bf16(dy w3 (H2 > 0)), and the head's weight and bias gradients.
__global__ void k_head(const __nv_bfloat16* __restrict__ H2, long long n, const float* __restrict__ p,
                       float* __restrict__ y, const float* __restrict__ t, __nv_bfloat16* __restrict__ dZ2,
                       float* __restrict__ g, float* __restrict__ loss, const long long* __restrict__ cur,
                       long long n_total) {
    __shared__ float sw[HID + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = threadIdx.x; k <= HID; k += blockDim.x) sw[k] = 0.0f;
    __syncthreads();
    float w3[4], h[4];
    for (int q = 0; q < 4; q++) w3[q] = p[OW3 + 4 * lane + q];
    const float b3 = p[OB3];
    float lsum = 0.0f;
    for (long long r = (long long)blockIdx.x * nw + warp; r < n; r += (long long)gridDim.x * nw) {
        float s = 0.0f;
        for (int q = 0; q < 4; q++) {
            h[q] = __bfloat162float(H2[r * HID + 4 * lane + q]);
            s += h[q] * w3[q];
        }
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        const float yr = s + b3;
        if (lane == 0 && y) y[r] = yr;
        if (!t) continue;
        const float e = yr - t[cur ? (cur[0] + r) % n_total : r];
        const float dy = 2.0f * e / (float)n;
        if (lane == 0) {
            lsum += e * e;
            atomicAdd(&sw[HID], dy);
        }
        for (int q = 0; q < 4; q++) {
            dZ2[r * HID + 4 * lane + q] = __float2bfloat16(h[q] > 0.0f ? dy * w3[q] : 0.0f);
            atomicAdd(&sw[4 * lane + q], dy * h[q]);
        }
    }
    __syncthreads();
    if (!t) return;
    for (int k = threadIdx.x; k < HID; k += blockDim.x) atomicAdd(&g[OW3 + k], sw[k]);
    if (threadIdx.x == 0) atomicAdd(&g[OB3], sw[HID]);
    if (lane == 0 && lsum != 0.0f) atomicAdd(loss, lsum / (float)n);
}

// Bias gradient: column sums of dZ [n][HID] into g[off .. off + HID).
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dZ, long long n, float* __restrict__ g, long long off) {
    const int c = threadIdx.x;   // blockDim.x == HID
    float s = 0.0f;
    for (long long r = blockIdx.x; r < n; r += gridDim.x) s += __bfloat162float(dZ[r * HID + c]);
    atomicAdd(&g[off + c], s);
}

// Adam step on the FP32 master parameters; step number cur[1] + 1 (bias
// corrections 1 - b^step).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, const long long* __restrict__ cur) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float step = (float)(cur[1] + 1);
    const float c1 = 1.0f - powf(b1, step), c2 = 1.0f - powf(b2, step);
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

// ------------------------------------------------------------ host side
#define TRY_M(expr)                  \
    do {                             \
        rpd_status _s = (expr);      \
        if (_s != RPD_OK) return _s; \
    } while (0)

struct rpd_mlp {
    cudaStream_t stream = nullptr;
    int n_in = 0;
    float* p = nullptr;   // FP32 master parameters
    float* g = nullptr;   // gradient
    float* m = nullptr;   // Adam moments
    float* v = nullptr;
    __nv_bfloat16* Wb = nullptr;   // BF16 copies of the three hidden layers
    int* err = nullptr;
    float* loss = nullptr;
    long long step = 0;
    long long* cur = nullptr;          // device: [next batch row, Adam steps taken]
    cudaStream_t tstream = nullptr;    // private stream the training steps are captured on
    cudaEvent_t tev[2] = {nullptr, nullptr};
    long long cap = 0;    // rows of the activation buffers (multiple of 128)
    __nv_bfloat16 *X = nullptr, *H0 = nullptr, *H1 = nullptr, *H2 = nullptr, *D2 = nullptr, *D1 = nullptr,
                  *D0 = nullptr;
    __nv_bfloat16* W0() const { return Wb; }
    __nv_bfloat16* W1() const { return Wb + HID * NIN; }
    __nv_bfloat16* W2() const { return Wb + HID * NIN + HID * HID; }
};

namespace {

size_t tile_smem() { return sizeof(TileSmem) + 1024; }

void free_acts(rpd_mlp* q) {
    for (__nv_bfloat16* b : {q->X, q->H0, q->H1, q->H2, q->D2, q->D1, q->D0})
        if (b) cudaFree(b);
    q->X = q->H0 = q->H1 = q->H2 = q->D2 = q->D1 = q->D0 = nullptr;
    q->cap = 0;
}

rpd_status ensure_acts(rpd_mlp* q, long long n) {
    const long long need = ((n + TM - 1) / TM) * TM;
    if (need <= q->cap) return RPD_OK;
    free_acts(q);
    __nv_bfloat16** bufs[7] = {&q->X, &q->H0, &q->H1, &q->H2, &q->D2, &q->D1, &q->D0};
    for (int k = 0; k < 7; k++)
        if (cudaMalloc(bufs[k], sizeof(__nv_bfloat16) * need * (k == 0 ? NIN : HID)) != cudaSuccess) {
            cudaGetLastError();
            free_acts(q);
            return RPD_E_OOM;
        }
    q->cap = need;
    return RPD_OK;
}

rpd_status launch_check(rpd_mlp* q) {
    if (cudaGetLastError() != cudaSuccess) return RPD_E_CUDA;
    int e = 0;
    if (cudaMemcpyAsync(&e, q->err, sizeof(int), cudaMemcpyDeviceToHost, q->stream) != cudaSuccess ||
        cudaStreamSynchronize(q->stream) != cudaSuccess) {
        cudaGetLastError();
        return RPD_E_CUDA;
    }
    return e ? (rpd_status)e : RPD_OK;
}

// Forward through the three hidden layers (tensor cores) and the head.  With
// n_total > 0 the n rows are the training batch that starts at the device
// cursor's row of the n_total data rows (x and t are the whole data).
void forward(rpd_mlp* q, const float* x, long long n, float* y, const float* t, long long n_total = 0) {
    cudaStream_t s = q->stream;
    const unsigned tiles = (unsigned)((n + TM - 1) / TM);
    const size_t sm = tile_smem();
    if (n_total > 0)
        k_to_bf16_batch<<<nblk(q->cap * NIN, 256), 256, 0, s>>>(x, n_total, q->n_in, n, q->cap, q->cur, q->X);
    else
        k_to_bf16<<<nblk(q->cap * NIN, 256), 256, 0, s>>>(x, n, q->n_in, q->cap, q->X);
    note_launch();
    k_mlp_fwd<<<tiles, MLP_THREADS, sm, s>>>(q->X, n, NIN, q->W0(), q->p + OB0, HID, q->H0, q->err);
    k_mlp_fwd<<<tiles, MLP_THREADS, sm, s>>>(q->H0, n, HID, q->W1(), q->p + OB1, HID, q->H1, q->err);
    k_mlp_fwd<<<tiles, MLP_THREADS, sm, s>>>(q->H1, n, HID, q->W2(), q->p + OB2, HID, q->H2, q->err);
    for (int k = 0; k < 3; k++) note_launch();
    if (t) {
        cudaMemsetAsync(q->g, 0, sizeof(float) * NPARAM, s);
        cudaMemsetAsync(q->loss, 0, sizeof(float), s);
    }
    k_head<<<152 * 4, 256, 0, s>>>(q->H2, n, q->p, y, t, q->D2, q->g, q->loss, n_total > 0 ? q->cur : nullptr,
                                   n_total);
    note_launch();
}

// Backward from dZ2 (written by the head): every gradient into q->g.
void backward(rpd_mlp* q, long long n) {
    cudaStream_t s = q->stream;
    const unsigned tiles = (unsigned)((n + TM - 1) / TM);
    const size_t sm = tile_smem();
    const unsigned bg = (unsigned)std::min<long long>(n, 152 * 8);
    k_mlp_dw<<<tiles, MLP_THREADS, sm, s>>>(q->D2, n, HID, q->H1, HID, q->g + OW2, q->err);
    k_bias_grad<<<bg, HID, 0, s>>>(q->D2, n, q->g, OB2);
    k_mlp_dx<<<tiles, MLP_THREADS, sm, s>>>(q->D2, n, HID, q->W2(), HID, q->H1, q->D1, q->err);
    k_mlp_dw<<<tiles, MLP_THREADS, sm, s>>>(q->D1, n, HID, q->H0, HID, q->g + OW1, q->err);
    k_bias_grad<<<bg, HID, 0, s>>>(q->D1, n, q->g, OB1);
    k_mlp_dx<<<tiles, MLP_THREADS, sm, s>>>(q->D1, n, HID, q->W1(), HID, q->H0, q->D0, q->err);
    k_mlp_dw<<<tiles, MLP_THREADS, sm, s>>>(q->D0, n, HID, q->X, NIN, q->g + OW0, q->err);
    k_bias_grad<<<bg, HID, 0, s>>>(q->D0, n, q->g, OB0);
    for (int k = 0; k < 8; k++) note_launch();
}

void cast_weights(rpd_mlp* q) {
    k_cast_weights<<<nblk(HID * HID, 256), 256, 0, q->stream>>>(q->p, q->W0(), q->W1(), q->W2());
    note_launch();
}

}  // namespace

extern "C" {

rpd_status rpd_mlp_create(int32_t n_in, uint64_t seed, void* cuda_stream, rpd_mlp** out) {
    if (!out) return RPD_E_INVALID;
    *out = nullptr;
    if (n_in < 1 || n_in > NIN) return RPD_E_INVALID;
    rpd_mlp* q = new rpd_mlp();
    q->stream = (cudaStream_t)cuda_stream;
    q->n_in = n_in;
    const size_t sm = tile_smem();
    bool ok = cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess &&
              cudaFuncSetAttribute(k_mlp_dx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess &&
              cudaFuncSetAttribute(k_mlp_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess;
    ok = ok && cudaMalloc(&q->p, sizeof(float) * NPARAM) == cudaSuccess &&
         cudaMalloc(&q->g, sizeof(float) * NPARAM) == cudaSuccess &&
         cudaMalloc(&q->m, sizeof(float) * NPARAM) == cudaSuccess &&
         cudaMalloc(&q->v, sizeof(float) * NPARAM) == cudaSuccess &&
         cudaMalloc(&q->Wb, sizeof(__nv_bfloat16) * (HID * NIN + 2 * HID * HID)) == cudaSuccess &&
         cudaMalloc(&q->err, sizeof(int)) == cudaSuccess && cudaMalloc(&q->loss, sizeof(float)) == cudaSuccess &&
         cudaMalloc(&q->cur, 2 * sizeof(long long)) == cudaSuccess &&
         cudaStreamCreateWithFlags(&q->tstream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&q->tev[0], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&q->tev[1], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        rpd_mlp_destroy(q);
        return RPD_E_OOM;
    }
    // He-uniform weights from a 64-bit xorshift stream of the seed; zero biases
    std::vector<float> h(NPARAM, 0.0f);
    unsigned long long st = seed * 0x9E3779B97F4A7C15ull + 0xD1B54A32D192ED03ull;
    auto uni = [&]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return (float)((st >> 11) * 0x1.0p-53) * 2.0f - 1.0f;
    };
    const float a0 = sqrtf(6.0f / (float)n_in), a1 = sqrtf(6.0f / HID);
    for (int r = 0; r < HID; r++)
        for (int c = 0; c < NIN; c++) h[OW0 + r * NIN + c] = c < n_in ? a0 * uni() : 0.0f;
    for (long long i = 0; i < HID * HID; i++) h[OW1 + i] = a1 * uni();
    for (long long i = 0; i < HID * HID; i++) h[OW2 + i] = a1 * uni();
    for (int k = 0; k < HID; k++) h[OW3 + k] = 0.1f * a1 * uni();
    cudaMemcpyAsync(q->p, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice, q->stream);
    cudaMemsetAsync(q->m, 0, sizeof(float) * NPARAM, q->stream);
    cudaMemsetAsync(q->v, 0, sizeof(float) * NPARAM, q->stream);
    cudaMemsetAsync(q->err, 0, sizeof(int), q->stream);
    cast_weights(q);
    const rpd_status s = launch_check(q);
    if (s != RPD_OK) {
        rpd_mlp_destroy(q);
        return s;
    }
    *out = q;
    return RPD_OK;
}

rpd_status rpd_mlp_params(rpd_mlp* q, float* d_out, int64_t cap, int64_t* n) {
    if (!q) return RPD_E_INVALID;
    if (n) *n = NPARAM;
    if (!d_out) return RPD_OK;
    if (cap < NPARAM) return RPD_E_INVALID;
    cudaMemcpyAsync(d_out, q->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, q->stream);
    return launch_check(q);
}

rpd_status rpd_mlp_set_params(rpd_mlp* q, const float* d_in, int64_t n) {
    if (!q || !d_in || n != NPARAM) return RPD_E_INVALID;
    cudaMemcpyAsync(q->p, d_in, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, q->stream);
    cast_weights(q);
    return launch_check(q);
}

rpd_status rpd_mlp_forward(rpd_mlp* q, const float* d_x, int64_t n, float* d_y) {
    if (!q || n < 0 || (n > 0 && (!d_x || !d_y))) return RPD_E_INVALID;
    if (n == 0) return RPD_OK;
    TRY_M(ensure_acts(q, n));
    forward(q, d_x, n, d_y, nullptr);
    return launch_check(q);
}

rpd_status rpd_mlp_grad(rpd_mlp* q, const float* d_x, const float* d_t, int64_t n, float* d_grad, float* h_loss) {
    if (!q || n < 1 || !d_x || !d_t) return RPD_E_INVALID;
    TRY_M(ensure_acts(q, n));
    forward(q, d_x, n, nullptr, d_t);
    backward(q, n);
    if (d_grad) cudaMemcpyAsync(d_grad, q->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, q->stream);
    if (h_loss) cudaMemcpyAsync(h_loss, q->loss, sizeof(float), cudaMemcpyDeviceToHost, q->stream);
    return launch_check(q);
}

rpd_status rpd_mlp_train(rpd_mlp* q, const float* d_x, const float* d_t, int64_t n, int32_t steps, int32_t batch,
                         float lr, float* h_loss) {
    if (!q || n < 1 || !d_x || !d_t || steps < 0 || batch < 1 || !(lr > 0)) return RPD_E_INVALID;
    const long long b = std::min<long long>(batch, n);
    TRY_M(ensure_acts(q, b));
    if (steps > 0) {
        // consecutive batches of the (caller-shuffled) data, wrapping around:
        // batch rows chosen on the device from the cursor, so one step's
        // launches are captured once as a CUDA graph and replayed
        const long long c0[2] = {0, q->step};
        cudaMemcpyAsync(q->cur, c0, sizeof(c0), cudaMemcpyHostToDevice, q->stream);
        cudaEventRecord(q->tev[0], q->stream);
        cudaStreamWaitEvent(q->tstream, q->tev[0], 0);
        cudaStream_t user = q->stream;
        q->stream = q->tstream;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const long long l0 = rpd_launch_count();
        bool ok = cudaStreamBeginCapture(q->tstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            forward(q, d_x, b, nullptr, d_t, n);
            backward(q, b);
            k_adam<<<nblk(NPARAM, 256), 256, 0, q->tstream>>>(q->p, q->g, q->m, q->v, NPARAM, lr, 0.9f, 0.999f, 1e-8f,
                                                               q->cur);
            note_launch();
            cast_weights(q);
            k_cursor_advance<<<1, 1, 0, q->tstream>>>(q->cur, b, n);
            note_launch();
            ok = cudaStreamEndCapture(q->tstream, &graph) == cudaSuccess && graph;
        }
        const long long per_step = rpd_launch_count() - l0;
        ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        for (int it = 0; ok && it < steps; it++) ok = cudaGraphLaunch(exec, q->tstream) == cudaSuccess;
        if (ok)   // the captured launches ran `steps` times, not once
            for (long long k = 0; k < per_step * (steps - 1); k++) note_launch();
        cudaEventRecord(q->tev[1], q->tstream);
        q->stream = user;
        cudaStreamWaitEvent(q->stream, q->tev[1], 0);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (!ok) {
            cudaGetLastError();
            cudaStreamSynchronize(q->tstream);
            return RPD_E_CUDA;
        }
        q->step += steps;
    }
    if (h_loss) cudaMemcpyAsync(h_loss, q->loss, sizeof(float), cudaMemcpyDeviceToHost, q->stream);
    return launch_check(q);
}

void rpd_mlp_destroy(rpd_mlp* q) {
    if (!q) return;
    if (q->stream) cudaStreamSynchronize(q->stream);
    free_acts(q);
    if (q->tstream) cudaStreamSynchronize(q->tstream);
    for (void* b : {(void*)q->p, (void*)q->g, (void*)q->m, (void*)q->v, (void*)q->Wb, (void*)q->err, (void*)q->loss,
                    (void*)q->cur})
        if (b) cudaFree(b);
    for (cudaEvent_t e : q->tev)
        if (e) cudaEventDestroy(e);
    if (q->tstream) cudaStreamDestroy(q->tstream);
    cudaGetLastError();
    delete q;
}

}  // extern "C"

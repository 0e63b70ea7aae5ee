// CUDA-core peak microbenchmarks: the denominators of the FP32 and FP64
// roofline fractions of the clip and volume kernels.
//
// Each thread runs CHAINS independent fused multiply-add chains x <- x * a + b
// for `iters` rounds; with enough warps per SM and CHAINS-way instruction-level
// parallelism the FMA pipes stay full, so flop / time is the sustained
// throughput of the pipe (2 flop per FMA).  a slightly below 1 and b small keep
// every value normal and bounded; the chains' sum is stored only when it equals
// a sentinel it never reaches, so the compiler cannot drop the loop.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "prim.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int PEAK_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_chain(long long iters, T a, T b, T* sink) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += x[c];
    if (s == (T)-12345.0) sink[blockIdx.x] = s;
}

template <typename T>
rpd_status run_peak(long long iters, cudaStream_t s, double* tflops, double* ms_out) {
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chain<T>, PEAK_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        return RPD_E_CUDA;
    }
    const long long blocks = (long long)nsm * (per_sm > 0 ? per_sm : 1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return RPD_E_CUDA;
    }
    const T a = (T)0.9999, b = (T)1e-4;
    // warm-up launch (clocks up, code loaded), then the timed one
    k_fma_chain<T><<<(unsigned)blocks, PEAK_THREADS, 0, s>>>(iters / 8 + 1, a, b, (T*)nullptr);
    note_launch();
    cudaEventRecord(e0, s);
    k_fma_chain<T><<<(unsigned)blocks, PEAK_THREADS, 0, s>>>(iters, a, b, (T*)nullptr);
    note_launch();
    cudaEventRecord(e1, s);
    float ms = 0;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || ms <= 0) {
        cudaGetLastError();
        return RPD_E_CUDA;
    }
    const double flop = 2.0 * CHAINS * (double)iters * (double)blocks * PEAK_THREADS;
    *tflops = flop / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return RPD_OK;
}

}  // namespace

extern "C" rpd_status rpd_peak_fma(int32_t precision, int64_t iters, void* cuda_stream, double* tflops,
                                   double* ms) {
    if (!tflops || iters < 1 || iters > (1ll << 40)) return RPD_E_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (precision == RPD_FP32_FILTERED) return run_peak<float>(iters, s, tflops, ms);
    if (precision == RPD_FP64) return run_peak<double>(iters, s, tflops, ms);
    return RPD_E_INVALID;
}

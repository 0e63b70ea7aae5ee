// Device primitives: scan, radix sort, segmented warp-shuffle reduction.
#include "prim.cuh"

#include <cuda_runtime.h>
#include <stdint.h>

namespace {

inline unsigned div_up_ll(long long a, int b) { return (unsigned)((a + b - 1) / b); }

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ long long warp_incl_scan(long long v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        long long o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* total) {
    __shared__ long long wsum[SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long x = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
        long long xi = warp_incl_scan(x);
        if (lane < SCAN_THREADS / 32) wsum[lane] = xi - x;
        if (lane == SCAN_THREADS / 32 - 1) *total = xi;
    }
    __syncthreads();
    long long r = inc - v + wsum[w];
    __syncthreads();
    return r;
}

template <typename T>
__global__ void scan_tiles(const T* __restrict__ in, int64_t* __restrict__ out, long long n,
                           int64_t* __restrict__ tile_sum) {
    __shared__ long long tot;
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        long long i = base + k;
        v[k] = i < n ? (long long)in[i] : 0;
        s += v[k];
    }
    long long pre = block_excl_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        long long i = base + k;
        if (i < n) out[i] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void scan_add(int64_t* __restrict__ out, long long n, const int64_t* __restrict__ tile_off) {
    long long base = (long long)blockIdx.x * SCAN_TILE;
    long long add = tile_off[blockIdx.x];
    for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_THREADS) {
        long long i = base + k;
        if (i < n) out[i] += add;
    }
}

__global__ void scan_total(int64_t* out, long long n, const int64_t* tile_off, long long ntiles) {
    out[n] = tile_off[ntiles];
}

long long n_tiles(long long n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

size_t scan_tmp_rec(long long n) {
    long long t = n_tiles(n);
    if (n <= 0) return 0;
    size_t here = sizeof(int64_t) * (2 * (size_t)t + 2);
    if (t <= 1) return here;
    return here + scan_tmp_rec(t);
}

template <typename T>
void scan_impl(const T* in, int64_t* out, long long n, void* tmp, cudaStream_t s) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int64_t), s);
        return;
    }
    long long t = n_tiles(n);
    int64_t* tsum = (int64_t*)tmp;
    int64_t* toff = tsum + t + 1;
    void* rest = toff + t + 1;
    scan_tiles<T><<<(unsigned)t, SCAN_THREADS, 0, s>>>(in, out, n, tsum);
    note_launch();
    if (t == 1) {
        cudaMemsetAsync(toff, 0, sizeof(int64_t), s);
        cudaMemcpyAsync(toff + 1, tsum, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    } else {
        scan_impl<int64_t>(tsum, toff, t, rest, s);
        scan_add<<<(unsigned)t, SCAN_THREADS, 0, s>>>(out, n, toff);
        note_launch();
    }
    scan_total<<<1, 1, 0, s>>>(out, n, toff, t);
    note_launch();
}

// ------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 4096 keys per block

__global__ void rs_hist(const uint64_t* __restrict__ keys, long long n, int shift, uint32_t* __restrict__ hist,
                        int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * RS_TILE;
    for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
        long long i = base + k;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[(long long)blockIdx.x * 256 + threadIdx.x] = h[threadIdx.x];
}

// Global offsets per (block, digit): digit-major exclusive scan of the
// block-major histogram, one thread per digit (256 threads, one block).
__global__ void rs_scan_hist(const uint32_t* __restrict__ hist, int nblocks, int64_t* __restrict__ hoff) {
    __shared__ long long base[256];
    const int d = threadIdx.x;
    long long s = 0;
    for (int b = 0; b < nblocks; b++) s += hist[(long long)b * 256 + d];
    base[d] = s;
    __syncthreads();
    if (d < 32) {
        // exclusive scan of the 256 digit totals by one warp (8 per lane)
        long long v[8], run = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            v[k] = base[d * 8 + k];
            run += v[k];
        }
        long long inc = run;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            long long o = __shfl_up_sync(0xffffffffu, inc, off);
            if (d >= off) inc += o;
        }
        long long pre = inc - run;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            base[d * 8 + k] = pre;
            pre += v[k];
        }
    }
    __syncthreads();
    s = base[d];
    for (int b = 0; b < nblocks; b++) {
        hoff[(long long)b * 256 + d] = s;
        s += hist[(long long)b * 256 + d];
    }
}

__global__ void rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                           uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, long long n, int shift,
                           const int64_t* __restrict__ hoff, int nblocks) {
    __shared__ uint32_t wh[RS_WARPS][256];
    __shared__ int64_t goff[256];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < RS_WARPS * 256; k += RS_THREADS) (&wh[0][0])[k] = 0;
    goff[threadIdx.x] = hoff[(long long)blockIdx.x * 256 + threadIdx.x];
    __syncthreads();
    long long base = (long long)blockIdx.x * RS_TILE + (long long)w * (RS_TILE / RS_WARPS);
    uint64_t key[RS_ROUNDS];
    uint32_t val[RS_ROUNDS];
    uint32_t pos[RS_ROUNDS];
    int dig[RS_ROUNDS];
    unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        long long i = base + r * 32 + lane;
        bool ok = i < n;
        key[r] = ok ? kin[i] : 0;
        val[r] = ok ? vin[i] : 0;
        dig[r] = ok ? (int)((key[r] >> shift) & 255) : 256;
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        int d = dig[r];
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && d < 256) old = wh[w][d];
        old = __shfl_sync(0xffffffffu, old, leader);
        pos[r] = old + __popc(peers & lt);
        if (lane == leader && d < 256) wh[w][d] = old + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        int d = threadIdx.x;   // 256 threads = 256 digits
        uint32_t run = 0;
        for (int q = 0; q < RS_WARPS; q++) {
            uint32_t t = wh[q][d];
            wh[q][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        int d = dig[r];
        if (d < 256) {
            long long dst = goff[d] + wh[w][d] + pos[r];
            kout[dst] = key[r];
            vout[dst] = val[r];
        }
    }
}

// -------------------------------------------------------- segmented reduce
__global__ void seg_heads(const uint64_t* __restrict__ keys, long long n, uint64_t sentinel,
                          uint8_t* __restrict__ head) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = keys[i];
    head[i] = (k != sentinel) && (i == 0 || keys[i - 1] != k);
}

__global__ void seg_reduce(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ pay, long long n,
                           uint64_t sentinel, const uint8_t* __restrict__ head, const int64_t* __restrict__ excl,
                           uint64_t* __restrict__ ukey, int32_t* __restrict__ chi, int32_t* __restrict__ beta) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    bool valid = i < n && keys[i] != sentinel;
    long long seg = -1;
    int c = 0, b = 0;
    if (valid) {
        seg = excl[i] + head[i] - 1;
        uint32_t p = pay[i];
        c = (int)(int16_t)(p & 0xffffu);
        b = (int)((p >> 16) & 1u);
        if (head[i]) ukey[seg] = keys[i];
    }
    // segmented inclusive scan across the warp (segments are contiguous runs)
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        long long s2 = __shfl_up_sync(0xffffffffu, seg, off);
        int c2 = __shfl_up_sync(0xffffffffu, c, off);
        int b2 = __shfl_up_sync(0xffffffffu, b, off);
        if (lane >= off && s2 == seg) {
            c += c2;
            b += b2;
        }
    }
    long long nxt = __shfl_down_sync(0xffffffffu, seg, 1);
    bool last = (lane == 31) || (nxt != seg);
    if (valid && last) {
        atomicAdd(&chi[seg], c);
        atomicAdd(&beta[seg], b);
    }
}

__global__ void seg_count(const int64_t* excl, long long n, int64_t* d_nseg) { *d_nseg = excl[n]; }

}  // namespace

size_t scan_tmp_bytes(long long n) { return scan_tmp_rec(n) + 64; }

void scan_excl(const int32_t* in, int64_t* out, long long n, void* tmp, cudaStream_t s) {
    scan_impl<int32_t>(in, out, n, tmp, s);
}
void scan_excl(const uint8_t* in, int64_t* out, long long n, void* tmp, cudaStream_t s) {
    scan_impl<uint8_t>(in, out, n, tmp, s);
}
void scan_excl(const int64_t* in, int64_t* out, long long n, void* tmp, cudaStream_t s) {
    scan_impl<int64_t>(in, out, n, tmp, s);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t radix_tmp_bytes(long long n) {
    long long nb = (n + RS_TILE - 1) / RS_TILE;
    if (nb < 1) nb = 1;
    long long nh = 256 * nb;
    return 2 * align256(sizeof(uint64_t) * (size_t)n) + 2 * align256(sizeof(uint32_t) * (size_t)n) +
           align256(sizeof(uint32_t) * (size_t)nh) + align256(sizeof(int64_t) * (size_t)(nh + 1)) +
           align256(scan_tmp_bytes(nh));
}

void radix_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                      long long n, int bits, void* tmp, cudaStream_t s) {
    if (n <= 0) return;
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    long long nb = (n + RS_TILE - 1) / RS_TILE;
    long long nh = 256 * nb;
    char* p = (char*)tmp;
    uint64_t* ka = (uint64_t*)p; p += align256(sizeof(uint64_t) * n);
    uint64_t* kb = (uint64_t*)p; p += align256(sizeof(uint64_t) * n);
    uint32_t* va = (uint32_t*)p; p += align256(sizeof(uint32_t) * n);
    uint32_t* vb = (uint32_t*)p; p += align256(sizeof(uint32_t) * n);
    uint32_t* hist = (uint32_t*)p; p += align256(sizeof(uint32_t) * nh);
    int64_t* hoff = (int64_t*)p; p += align256(sizeof(int64_t) * (nh + 1));
    const uint64_t* ksrc = keys_in;
    const uint32_t* vsrc = vals_in;
    for (int q = 0; q < passes; q++) {
        bool lastp = (q == passes - 1);
        uint64_t* kdst = lastp ? keys_out : ((q & 1) ? kb : ka);
        uint32_t* vdst = lastp ? vals_out : ((q & 1) ? vb : va);
        int shift = 8 * q;
        rs_hist<<<(unsigned)nb, RS_THREADS, 0, s>>>(ksrc, n, shift, hist, (int)nb);
        note_launch();
        rs_scan_hist<<<1, 256, 0, s>>>(hist, (int)nb, hoff);
        note_launch();
        rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(ksrc, vsrc, kdst, vdst, n, shift, hoff, (int)nb);
        note_launch();
        ksrc = kdst;
        vsrc = vdst;
    }
}

size_t segreduce_tmp_bytes(long long n) {
    return align256((size_t)(n > 0 ? n : 1)) + align256(sizeof(int64_t) * (size_t)(n + 1)) +
           align256(scan_tmp_bytes(n));
}

void segmented_reduce(const uint64_t* keys, const uint32_t* pay, long long n, uint64_t sentinel, uint64_t* ukey,
                      int32_t* chi, int32_t* beta0, int64_t* d_nseg, void* tmp, cudaStream_t s) {
    if (n <= 0) {
        cudaMemsetAsync(d_nseg, 0, sizeof(int64_t), s);
        return;
    }
    char* p = (char*)tmp;
    uint8_t* head = (uint8_t*)p; p += align256((size_t)n);
    int64_t* excl = (int64_t*)p; p += align256(sizeof(int64_t) * (n + 1));
    void* stmp = p;
    const int T = 256;
    seg_heads<<<div_up_ll(n, T), T, 0, s>>>(keys, n, sentinel, head);
    note_launch();
    scan_impl<uint8_t>(head, excl, n, stmp, s);
    cudaMemsetAsync(chi, 0, sizeof(int32_t) * n, s);
    cudaMemsetAsync(beta0, 0, sizeof(int32_t) * n, s);
    seg_reduce<<<div_up_ll(n, T), T, 0, s>>>(keys, pay, n, sentinel, head, excl, ukey, chi, beta0);
    note_launch();
    seg_count<<<1, 1, 0, s>>>(excl, n, d_nseg);
    note_launch();
}

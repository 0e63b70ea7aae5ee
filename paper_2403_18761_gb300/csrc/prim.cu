// Device primitives: exclusive scan and onesweep radix sort.
#include "prim.cuh"

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>

#include "rpd.h"

namespace {

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
// Onesweep LSD radix sort (8-bit digits): one kernel builds the digit
// histograms of every pass, one scans them, then one kernel per pass ranks
// and scatters a tile of 4096 keys.  Tiles take their index from an atomic
// counter in launch order, publish their digit counts, and obtain their
// global offsets by decoupled look-back over the preceding tiles (a waiting
// tile only ever waits for a tile that is already running).  Every wait is
// bounded; on timeout the pass records RPD_E_TIMEOUT and drops the writes it
// cannot place.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 4096 keys per tile
constexpr int RS_MAXPASS = 8;
constexpr uint32_t LB_AGG = 1u << 30, LB_PRE = 2u << 30, LB_VAL = (1u << 30) - 1;
constexpr int LB_SPIN_LIMIT = 1 << 22;

__device__ __forceinline__ long long rs_count(const long long* d_n, long long n) { return d_n ? *d_n : n; }

__global__ void rs_hist_all(const uint64_t* __restrict__ keys, const long long* __restrict__ d_n, long long n_host,
                            int passes, uint32_t* __restrict__ ghist) {
    __shared__ uint32_t h[RS_MAXPASS][256];
    for (int k = threadIdx.x; k < RS_MAXPASS * 256; k += RS_THREADS) (&h[0][0])[k] = 0;
    __syncthreads();
    const long long n = rs_count(d_n, n_host);
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * RS_TILE; base < n; base += (long long)gridDim.x * RS_TILE) {
        for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
            const long long i = base + k;
            const bool ok = i < n;
            const uint64_t key = ok ? keys[i] : 0;
            for (int q = 0; q < passes; q++) {
                const int d = ok ? (int)((key >> (8 * q)) & 255) : 256;
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                if (d < 256 && lane == __ffs(peers) - 1) atomicAdd(&h[q][d], (uint32_t)__popc(peers));
            }
        }
    }
    __syncthreads();
    for (int q = 0; q < passes; q++) {
        const uint32_t v = h[q][threadIdx.x];
        if (v) atomicAdd(&ghist[q * 256 + threadIdx.x], v);
    }
}

// Exclusive scan over the 256 digits of every pass (one block).
__global__ void rs_scan_all(const uint32_t* __restrict__ ghist, int passes, uint32_t* __restrict__ gbase) {
    __shared__ uint32_t wsum[RS_WARPS];
    const int d = threadIdx.x, lane = d & 31, w = d >> 5;
    for (int q = 0; q < passes; q++) {
        const uint32_t v = ghist[q * 256 + d];
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t off = 0;
        for (int k = 0; k < w; k++) off += wsum[k];
        gbase[q * 256 + d] = off + inc - v;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(RS_THREADS) rs_pass(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                     uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                     const long long* __restrict__ d_n, long long n_host, int shift,
                                                     const uint32_t* __restrict__ gbase, uint32_t* look,
                                                     uint32_t* tcnt, int* err, int spin_limit,
                                                     const uint32_t* stall_row) {
    __shared__ uint32_t wh[RS_WARPS][256];
    __shared__ uint32_t dbase[256];
    __shared__ int tile_s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) tile_s = (int)atomicAdd(tcnt, 1u);
    for (int k = threadIdx.x; k < RS_WARPS * 256; k += RS_THREADS) (&wh[0][0])[k] = 0;
    __syncthreads();
    const long long n = rs_count(d_n, n_host);
    const long long tile = tile_s;
    if (tile * RS_TILE >= n) return;   // block-uniform
    const long long base = tile * RS_TILE + (long long)w * (RS_TILE / RS_WARPS);
    uint64_t key[RS_ROUNDS];
    uint32_t val[RS_ROUNDS];
    uint32_t pos[RS_ROUNDS];
    int dig[RS_ROUNDS];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        const long long i = base + r * 32 + lane;
        const bool ok = i < n;
        key[r] = ok ? kin[i] : 0;
        val[r] = ok ? vin[i] : 0;
        dig[r] = ok ? (int)((key[r] >> shift) & 255) : 256;
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        const int d = dig[r];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && d < 256) old = wh[w][d];
        old = __shfl_sync(0xffffffffu, old, leader);
        pos[r] = old + __popc(peers & lt);
        if (lane == leader && d < 256) wh[w][d] = old + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;   // 256 threads = 256 digits
        uint32_t run = 0;
        for (int q = 0; q < RS_WARPS; q++) {
            const uint32_t t = wh[q][d];
            wh[q][d] = run;
            run += t;
        }
        // publish this tile's count, then look back for its offset
        volatile uint32_t* L = look;
        uint32_t excl = 0;
        if (tile == 0) {
            atomicExch(&look[d], LB_PRE | run);
        } else {
            atomicExch(&look[tile * 256 + d], LB_AGG | run);
            long long t = tile - 1;
            int spins = 0;
            // test hook: tile 1 waits on a row that no tile publishes, so its
            // bounded wait runs out
            volatile const uint32_t* stall = (stall_row && tile == 1) ? stall_row : nullptr;
            while (true) {
                const uint32_t v = stall ? stall[d] : L[t * 256 + d];
                if (v & LB_PRE) {
                    excl += v & LB_VAL;
                    break;
                }
                if (v & LB_AGG) {
                    excl += v & LB_VAL;
                    t--;
                    continue;
                }
                if (++spins > spin_limit) {
                    atomicCAS(err, 0, (int)RPD_E_TIMEOUT);
                    excl = 0x80000000u;   // marks the digit as unplaceable
                    break;
                }
            }
            if (excl != 0x80000000u) atomicExch(&look[tile * 256 + d], LB_PRE | (excl + run));
        }
        dbase[d] = excl == 0x80000000u ? 0xffffffffu : gbase[d] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        const int d = dig[r];
        if (d < 256 && dbase[d] != 0xffffffffu) {
            const long long dst = (long long)dbase[d] + wh[w][d] + pos[r];
            if (dst < n) {
                kout[dst] = key[r];
                vout[dst] = val[r];
            }
        }
    }
}

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

static long long rs_tiles(long long n) { return n > 0 ? (n + RS_TILE - 1) / RS_TILE : 1; }

size_t radix_tmp_bytes(long long n) {
    const long long nt = rs_tiles(n);
    return 2 * align256(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1)) +
           2 * align256(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)) +
           align256(sizeof(uint32_t) * (size_t)(2 * RS_MAXPASS * 256 + RS_MAXPASS)) +
           align256(sizeof(uint32_t) * (size_t)(RS_MAXPASS * nt * 256 + 256));
}

// Test hook, read at every sort: RPD_TEST_LOOKBACK_STALL=N makes tile 1 of
// every radix pass look back at a row that is never published, with a spin
// bound of N, so that its wait runs out and the pass reports RPD_E_TIMEOUT.
static int lookback_stall_limit() {
    const char* e = getenv("RPD_TEST_LOOKBACK_STALL");
    return e ? atoi(e) : 0;
}

static void radix_sort_impl(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                            const long long* d_n, long long nmax, int bits, void* tmp, int* d_err, cudaStream_t s) {
    if (nmax <= 0) return;
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    if (passes > RS_MAXPASS) passes = RS_MAXPASS;
    const long long nt = rs_tiles(nmax);
    char* p = (char*)tmp;
    uint64_t* ka = (uint64_t*)p; p += align256(sizeof(uint64_t) * nmax);
    uint64_t* kb = (uint64_t*)p; p += align256(sizeof(uint64_t) * nmax);
    uint32_t* va = (uint32_t*)p; p += align256(sizeof(uint32_t) * nmax);
    uint32_t* vb = (uint32_t*)p; p += align256(sizeof(uint32_t) * nmax);
    uint32_t* ctl = (uint32_t*)p; p += align256(sizeof(uint32_t) * (2 * RS_MAXPASS * 256 + RS_MAXPASS));
    uint32_t* look = (uint32_t*)p;
    uint32_t* ghist = ctl;
    uint32_t* gbase = ctl + RS_MAXPASS * 256;
    uint32_t* tcnt = ctl + 2 * RS_MAXPASS * 256;
    // histograms, tile counters and look-back words start at zero
    cudaMemsetAsync(ctl, 0, sizeof(uint32_t) * (2 * RS_MAXPASS * 256 + RS_MAXPASS), s);
    cudaMemsetAsync(look, 0, sizeof(uint32_t) * (size_t)(passes * nt * 256 + 256), s);
    const int stall = lookback_stall_limit();
    const uint32_t* stall_row = stall > 0 ? look + (size_t)passes * nt * 256 : nullptr;
    const int spin_limit = stall > 0 ? stall : LB_SPIN_LIMIT;
    const unsigned hb = (unsigned)std::min<long long>(nt, 152LL * 8);
    rs_hist_all<<<hb, RS_THREADS, 0, s>>>(keys_in, d_n, nmax, passes, ghist);
    note_launch();
    rs_scan_all<<<1, 256, 0, s>>>(ghist, passes, gbase);
    note_launch();
    const uint64_t* ksrc = keys_in;
    const uint32_t* vsrc = vals_in;
    for (int q = 0; q < passes; q++) {
        const bool lastp = (q == passes - 1);
        uint64_t* kdst = lastp ? keys_out : ((q & 1) ? kb : ka);
        uint32_t* vdst = lastp ? vals_out : ((q & 1) ? vb : va);
        rs_pass<<<(unsigned)nt, RS_THREADS, 0, s>>>(ksrc, vsrc, kdst, vdst, d_n, nmax, 8 * q, gbase + q * 256,
                                                     look + (size_t)q * nt * 256, tcnt + q, d_err, spin_limit,
                                                     stall_row);
        note_launch();
        ksrc = kdst;
        vsrc = vdst;
    }
}

void radix_sort_pairs(const uint64_t* keys_in, const uint32_t* vals_in, uint64_t* keys_out, uint32_t* vals_out,
                      long long n, int bits, void* tmp, int* d_err, cudaStream_t s) {
    radix_sort_impl(keys_in, vals_in, keys_out, vals_out, nullptr, n, bits, tmp, d_err, s);
}

// A5-A7 helpers: union-find over element pieces, key unpacking, flags.
//
// Components (Sec. 4.1.1): the pieces of one restricted element in two
// face-adjacent tets belong to the same component when the element crosses
// their shared face (the piece has a face on it for an RPC, an edge on it for
// an RPF, an end point on it for an RPE).  Union-find hooks the larger root
// under the smaller with atomicCAS, so parent pointers only decrease and no
// cycle can form; every loop is bounded and reports RPD_E_TIMEOUT if the bound
// is hit.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int UF_LIMIT = 1 << 22;

__device__ __forceinline__ int uf_find(int32_t* parent, int x) {
    volatile int32_t* P = parent;
    for (int it = 0; it < UF_LIMIT; it++) {
        int px = P[x];
        if (px == x) return x;
        int gx = P[px];
        if (gx != px) P[x] = gx;   // path halving (benign race: gx is an ancestor)
        x = gx;
    }
    return -1;
}

__device__ __forceinline__ void uf_union(int32_t* parent, int a, int b, DevState* st) {
    for (int it = 0; it < UF_LIMIT; it++) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a < 0 || b < 0) break;
        if (a == b) return;
        if (a < b) {
            int t = a;
            a = b;
            b = t;
        }
        int old = atomicCAS(&parent[a], a, b);
        if (old == a) return;
    }
    dev_fail(st, RPD_E_TIMEOUT, CNT_UF_LIMIT);
}

__global__ void k_iota(int32_t* p, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

// slot of sphere `sph` among the (sorted) candidates of tet t, or -1
__device__ __forceinline__ int find_slot(const ClipArgs& A, long long t, int sph) {
    int n = A.cand_cnt[t];
    const int32_t* c = A.cand + t * RPD_MAXC;
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = c[mid];
        if (v == sph) return mid;
        if (v < sph) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__global__ void k_link_cells(ClipArgs A, long long npairs, int32_t* __restrict__ parent) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs || A.pflag[p] != 1) return;
    unsigned lk = A.c_link[p];
    if (!lk) return;
    long long t = A.pair_tet[p];
    int i = A.cand[t * RPD_MAXC + (p - A.pair_off[t])];
    for (int f = 0; f < 4; f++) {
        if (!((lk >> f) & 1)) continue;
        long long t2 = A.adj[4 * t + f];
        if (t2 <= t) continue;    // each shared face once, from its lower tet
        int s2 = find_slot(A, t2, i);
        long long p2 = s2 < 0 ? -1 : A.pair_off[t2] + s2;
        if (p2 < 0 || A.pflag[p2] != 1) {
            dev_fail(A.st, RPD_E_DEGENERATE, CNT_LINK_MISSING);
            continue;
        }
        uf_union(parent, (int)p, (int)p2, A.st);
    }
}

__global__ void k_link_records(ClipArgs A, int which, long long nrec, int32_t* __restrict__ parent) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    unsigned lk = A.rlink[which][r];
    if (!lk) return;
    long long t = A.rtet[which][r];
    uint64_t key = A.rkey[which][r];
    int shift = (which + 1) * A.key_bits;
    int i = (int)(key >> shift);
    const int32_t* off = which == 0 ? A.f_off : A.e_off;
    const uint8_t* cnt = which == 0 ? A.f_cnt : A.e_cnt;
    for (int f = 0; f < 4; f++) {
        if (!((lk >> f) & 1)) continue;
        long long t2 = A.adj[4 * t + f];
        if (t2 <= t) continue;
        int s2 = find_slot(A, t2, i);
        long long r2 = -1;
        if (s2 >= 0) {
            long long p2 = A.pair_off[t2] + s2;
            if (A.pflag[p2] == 1) {
                long long b0 = off[p2], b1 = b0 + cnt[p2];
                for (long long z = b0; z < b1; z++)
                    if (A.rkey[which][z] == key) {
                        r2 = z;
                        break;
                    }
            }
        }
        if (r2 < 0) {
            dev_fail(A.st, RPD_E_DEGENERATE, CNT_LINK_MISSING);
            continue;
        }
        uf_union(parent, (int)r, (int)r2, A.st);
    }
}

__global__ void k_cell_payload(ClipArgs A, long long npairs, int32_t* __restrict__ parent, uint32_t* __restrict__ pay,
                               uint64_t* __restrict__ keys, uint64_t sentinel) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    if (A.pflag[p] != 1) {
        keys[p] = sentinel;
        pay[p] = 0;
        return;
    }
    long long t = A.pair_tet[p];
    int i = A.cand[t * RPD_MAXC + (p - A.pair_off[t])];
    int root = uf_find(parent, (int)p) == (int)p;
    keys[p] = (uint64_t)i;
    pay[p] = ((uint32_t)(uint16_t)(int16_t)A.c_val[p]) | ((uint32_t)root << 16);
}

__global__ void k_record_payload(ClipArgs A, int which, long long nrec, int32_t* __restrict__ parent,
                                 uint32_t* __restrict__ pay) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrec) return;
    int root = parent ? (uf_find(parent, (int)r) == (int)r) : 1;
    pay[r] = ((uint32_t)(uint16_t)A.rval[which][r]) | ((uint32_t)root << 16);
}

__global__ void k_unpack(const uint64_t* __restrict__ ukey, long long n, int kind, int b, int32_t* __restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = ukey[i];
    uint64_t mask = (b >= 64) ? ~0ull : ((1ull << b) - 1);
    for (int j = 0; j < kind; j++) out[i * kind + j] = (int32_t)((k >> (b * (kind - 1 - j))) & mask);
}

__global__ void k_flags(const int32_t* __restrict__ chi, const int32_t* __restrict__ beta, long long n,
                        uint8_t* __restrict__ flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (beta[i] == 1 && chi[i] == 1) ? 1 : 0;
}

__global__ void k_compact_pieces(ClipArgs A, long long npairs, const int64_t* __restrict__ off, int32_t* d_tet,
                                 int32_t* d_sphere, double* d_vol, double* d_mom) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs || A.pflag[p] != 1) return;
    long long o = off[p];
    long long t = A.pair_tet[p];
    if (d_tet) d_tet[o] = (int32_t)t;
    if (d_sphere) d_sphere[o] = A.cand[t * RPD_MAXC + (p - A.pair_off[t])];
    if (d_vol) d_vol[o] = A.p_vol[p];
    if (d_mom)
        for (int k = 0; k < 3; k++) d_mom[3 * o + k] = A.p_mom[3 * p + k];
}

}  // namespace

void launch_components_cells(const ClipArgs& a, long long npairs, int32_t* parent, uint32_t* pay, uint64_t* keys,
                             int key_bits, uint64_t sentinel, cudaStream_t s) {
    (void)key_bits;
    if (npairs <= 0) return;
    k_iota<<<nblk(npairs, 256), 256, 0, s>>>(parent, npairs);
    note_launch();
    k_link_cells<<<nblk(npairs, 256), 256, 0, s>>>(a, npairs, parent);
    note_launch();
    k_cell_payload<<<nblk(npairs, 256), 256, 0, s>>>(a, npairs, parent, pay, keys, sentinel);
    note_launch();
}

void launch_components_records(const ClipArgs& a, int which, long long nrec, int32_t* parent, uint32_t* pay,
                               cudaStream_t s) {
    if (nrec <= 0) return;
    if (which < 2) {
        k_iota<<<nblk(nrec, 256), 256, 0, s>>>(parent, nrec);
        note_launch();
        k_link_records<<<nblk(nrec, 256), 256, 0, s>>>(a, which, nrec, parent);
        note_launch();
        k_record_payload<<<nblk(nrec, 256), 256, 0, s>>>(a, which, nrec, parent, pay);
        note_launch();
    } else {
        k_record_payload<<<nblk(nrec, 256), 256, 0, s>>>(a, which, nrec, nullptr, pay);
        note_launch();
    }
}

void launch_unpack_keys(const uint64_t* ukey, long long n, int kind, int key_bits, int32_t* out, cudaStream_t s) {
    if (n <= 0) return;
    k_unpack<<<nblk(n, 256), 256, 0, s>>>(ukey, n, kind, key_bits, out);
    note_launch();
}

void launch_flags(const int32_t* chi, const int32_t* beta0, long long n, uint8_t* flag, cudaStream_t s) {
    if (n <= 0) return;
    k_flags<<<nblk(n, 256), 256, 0, s>>>(chi, beta0, n, flag);
    note_launch();
}

void launch_compact_pieces(const ClipArgs& a, long long npairs, const int64_t* off, int32_t* d_tet, int32_t* d_sphere,
                           double* d_vol, double* d_mom, cudaStream_t s) {
    if (npairs <= 0) return;
    k_compact_pieces<<<nblk(npairs, 256), 256, 0, s>>>(a, npairs, off, d_tet, d_sphere, d_vol, d_mom);
    note_launch();
}

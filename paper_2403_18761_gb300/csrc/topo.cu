// A5-A7: union-find over element pieces, chi and roots summed per key,
// sorted key rows, flags.
//
// Components (Sec. 4.1.1): the pieces of one restricted element in two
// face-adjacent tets belong to the same component when the element crosses
// their shared face (the piece has a face on it for an RPC, an edge on it for
// an RPF, an end point on it for an RPE).  Union-find hooks the larger root
// under the smaller with atomicCAS, so parent pointers only decrease and no
// cycle can form; a negative parent marks a root, so a memset initialises the
// forest.  Every loop is bounded and reports RPD_E_TIMEOUT if the bound is hit.
//
// chi and beta0 per key (Sec. 4.1.2, Sec. 4.1.1): every piece or record adds
// its contribution and, if it is a root, one component to its key's slot of a
// hash table (per sphere for cells).  The keys are then put in order by a
// bucket pass on their first sphere index (the keys of one sphere are few)
// and a rank inside each bucket.
#include <cuda_runtime.h>
#include <stdint.h>

#include <stdlib.h>

#include <algorithm>

#include "internal.cuh"
#include "prim.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Iteration bound of the union-find loops (ClipArgs::uf_limit); the library
// uses UF_LIMIT, a test hook may lower it to make the bound run out.
constexpr int UF_LIMIT = 1 << 22;

__device__ __forceinline__ int uf_find(int32_t* parent, int x, int limit) {
    volatile int32_t* P = parent;
    for (int it = 0; it < limit; it++) {
        const int px = P[x];
        if (px < 0) return x;
        const int gx = P[px];
        if (gx < 0) return px;
        P[x] = gx;   // path halving (benign race: gx is an ancestor)
        x = gx;
    }
    return -1;
}

__device__ __forceinline__ void uf_union(int32_t* parent, int a, int b, DevState* st, int limit) {
    for (int it = 0; it < limit; it++) {
        a = uf_find(parent, a, limit);
        b = uf_find(parent, b, limit);
        if (a < 0 || b < 0) break;
        if (a == b) return;
        if (a < b) {
            int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(&parent[a], -1, b) == -1) return;
    }
    dev_fail(st, RPD_E_TIMEOUT, CNT_UF_LIMIT);
}

// Slot of sphere `sph` among the candidates of tet t, or -1.  A candidate row
// is 32 ints (128-byte aligned): its used part is read with independent
// 16-byte loads and searched in registers (one memory round trip).
__device__ __forceinline__ int find_slot(const ClipArgs& A, long long t, int sph) {
    const int n = A.cand_cnt[t];
    const int4* c4 = reinterpret_cast<const int4*>(A.cand + t * RPD_MAXC);
    int found = -1;
    for (int k = 0; 4 * k < n; k++) {
        const int4 v = c4[k];
        if (v.x == sph && 4 * k < n) found = 4 * k;
        if (v.y == sph && 4 * k + 1 < n) found = 4 * k + 1;
        if (v.z == sph && 4 * k + 2 < n) found = 4 * k + 2;
        if (v.w == sph && 4 * k + 3 < n) found = 4 * k + 3;
    }
    return found;
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
        uf_union(parent, (int)p, (int)p2, A.st, A.uf_limit);
    }
}

// Record count of one kind: read on the device (written by the clip), capped.
__device__ __forceinline__ long long rec_count(const ClipArgs& A, int which, long long nmax) {
    const long long n = (long long)A.rcount[which];
    return n < nmax ? n : nmax;
}

__global__ void k_link_records(ClipArgs A, int which, long long nmax, int32_t* __restrict__ parent) {
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nrec = rec_count(A, which, nmax);   // records past it were never written
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
                long long b0 = off[p2], b1 = min(b0 + (long long)cnt[p2], nrec);
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
        uf_union(parent, (int)r, (int)r2, A.st, A.uf_limit);
    }
}

// ------------------------------------------------------ aggregation (A5-A7)
// Cells: chi and root counts summed straight into per-sphere slots.
__global__ void k_cell_agg(ClipArgs A, long long npairs, int32_t* __restrict__ parent, int32_t* __restrict__ cchi,
                           int32_t* __restrict__ cbeta, uint8_t* __restrict__ cpres) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = p < npairs && A.pflag[p] == 1;
    int i = -1, c = 0, r = 0;
    if (live) {
        const long long t = A.pair_tet[p];
        i = A.cand[t * RPD_MAXC + (p - A.pair_off[t])];
        c = (int)A.c_val[p];
        r = parent[p] < 0;
    }
    // the pairs of a warp come from a few neighbouring tets and share spheres:
    // one atomic per distinct sphere of the warp
    const unsigned peers = __match_any_sync(0xffffffffu, i);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    int sc = 0, sr = 0;
    for (unsigned m = peers; m; m &= m - 1) {
        const int k = __ffs(m) - 1;
        sc += __shfl_sync(peers, c, k);
        sr += __shfl_sync(peers, r, k);
    }
    if (!live || lane != leader) return;
    if (sc) atomicAdd(&cchi[i], sc);
    if (sr) atomicAdd(&cbeta[i], sr);
    cpres[i] = 1;
}

__global__ void k_cell_emit(long long ns, const uint8_t* __restrict__ cpres, const int64_t* __restrict__ pos,
                            const int32_t* __restrict__ cchi, const int32_t* __restrict__ cbeta,
                            int32_t* __restrict__ keys, int32_t* __restrict__ chi, int32_t* __restrict__ beta,
                            uint8_t* __restrict__ flag, long long* __restrict__ count) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *count = pos[ns];
    if (i >= ns || !cpres[i]) return;
    const long long q = pos[i];
    const int c = cchi[i], b = cbeta[i];
    keys[q] = (int32_t)i;
    chi[q] = c;
    beta[q] = b;
    flag[q] = (b == 1 && c == 1) ? 1 : 0;
}

// Faces, edges, vertices: records hashed by key; chi and root counts summed
// into the key's slot.
__global__ void k_rec_agg(ClipArgs A, int which, long long nmax, int32_t* __restrict__ parent, uint64_t* __restrict__ tk,
                          int32_t* __restrict__ tchi, int32_t* __restrict__ tbeta, unsigned long long mask,
                          int shift) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rec_count(A, which, nmax)) return;
    const uint64_t key = A.rkey[which][r];
    const bool root = parent ? parent[r] < 0 : true;
    const long long h = table_insert(tk, mask, shift, key);
    if (h < 0) {   // cannot happen: capacity >= 2 * records
        dev_fail(A.st, RPD_E_OVERFLOW, CNT_CAPACITY);
        return;
    }
    atomicAdd(&tchi[h], (int)A.rval[which][r]);
    if (root) atomicAdd(&tbeta[h], 1);
}

// Occupied slots appended (warp-aggregated) to (key, slot) lists; each key
// counted in the bucket of its first sphere.
__global__ void k_table_compact(const uint64_t* __restrict__ tk, long long cap, int shift, uint64_t* __restrict__ ck,
                                uint32_t* __restrict__ cs, unsigned long long* __restrict__ count,
                                int32_t* __restrict__ bcount) {
    const long long h = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const uint64_t key = h < cap ? tk[h] : HEMPTY;
    const bool occ = key != HEMPTY;
    const unsigned m = __ballot_sync(0xffffffffu, occ);
    if (!m) return;
    unsigned long long base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (occ) {
        const unsigned long long q = base + __popc(m & ((1u << lane) - 1u));
        ck[q] = key;
        cs[q] = (uint32_t)h;
        atomicAdd(&bcount[key >> shift], 1);
    }
}

// (key, slot) into the bucket of the key's first sphere (any order inside).
__global__ void k_bucket_fill(const uint64_t* __restrict__ ck, const uint32_t* __restrict__ cs,
                              const unsigned long long* __restrict__ count, long long nmax, int shift,
                              const int64_t* __restrict__ bstart, int32_t* __restrict__ bfill,
                              uint64_t* __restrict__ bk, uint32_t* __restrict__ bs) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)*count || i >= nmax) return;
    const uint64_t key = ck[i];
    const long long b = (long long)(key >> shift);
    const long long q = bstart[b] + atomicAdd(&bfill[b], 1);
    bk[q] = key;
    bs[q] = cs[i];
}

// Rank inside the bucket, then the output row: sorted key, chi, beta0, flag.
__global__ void k_bucket_emit(const uint64_t* __restrict__ bk, const uint32_t* __restrict__ bs,
                              const unsigned long long* __restrict__ count, long long nmax, int kind, int b,
                              const int64_t* __restrict__ bstart, const int32_t* __restrict__ tchi,
                              const int32_t* __restrict__ tbeta, int32_t* __restrict__ keys,
                              int32_t* __restrict__ chi, int32_t* __restrict__ beta, uint8_t* __restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)*count || i >= nmax) return;
    const uint64_t k = bk[i];
    const long long bu = (long long)(k >> ((kind - 1) * b));
    const long long b0 = bstart[bu], b1 = bstart[bu + 1];
    long long q = b0;
    for (long long j = b0; j < b1; j++) q += bk[j] < k;
    const uint64_t mask = (b >= 64) ? ~0ull : ((1ull << b) - 1);
    for (int j = 0; j < kind; j++) keys[q * kind + j] = (int32_t)((k >> (b * (kind - 1 - j))) & mask);
    const uint32_t h = bs[i];
    const int c = tchi[h], bb = tbeta[h];
    chi[q] = c;
    beta[q] = bb;
    flag[q] = (bb == 1 && c == 1) ? 1 : 0;
}

__global__ void k_copy_rows(const int32_t* __restrict__ keys, int32_t* __restrict__ d_keys, long long nk,
                            const void* __restrict__ vals, void* __restrict__ d_vals, long long n, int elem) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nk + n; i += stride) {
        if (i < nk) {
            if (keys) d_keys[i] = keys[i];
        } else if (vals) {
            const long long j = i - nk;
            if (elem == 4) ((int32_t*)d_vals)[j] = ((const int32_t*)vals)[j];
            else ((uint8_t*)d_vals)[j] = ((const uint8_t*)vals)[j];
        }
    }
}

// Fill byte ranges (blockIdx.y selects the range): 16-byte stores over the
// aligned middle, single bytes at the ends.
__global__ void k_clear(ClearList C) {
    char* p = (char*)C.p[blockIdx.y];
    const long long n = C.bytes[blockIdx.y];
    const unsigned char v = (unsigned char)C.value[blockIdx.y];
    const long long a = (long long)((16 - ((uintptr_t)p & 15)) & 15);
    const long long head = n < a ? n : a;
    const long long n16 = (n - head) / 16;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned w = 0x01010101u * v;
    uint4* q = (uint4*)(p + head);
    for (long long i = tid; i < n16; i += stride) q[i] = make_uint4(w, w, w, w);
    const long long tail0 = head + 16 * n16;
    if (tid < head) p[tid] = (char)v;
    if (tid < n - tail0) p[tail0 + tid] = (char)v;
}

// blockIdx.y selects the segment
__global__ void k_export(ExportArgs a) {
    const ExportSeg g = a.seg[blockIdx.y];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
        if (g.elem == 4) ((int32_t*)g.dst)[i] = ((const int32_t*)g.src)[i];
        else ((uint8_t*)g.dst)[i] = ((const uint8_t*)g.src)[i];
    }
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

// Test hook, read at every build: RPD_TEST_UF_LIMIT=N bounds every
// union-find loop by N iterations instead of UF_LIMIT (N = 0 makes every
// union give up, so the build reports RPD_E_TIMEOUT).
int uf_iteration_limit() {
    const char* e = getenv("RPD_TEST_UF_LIMIT");
    return e ? atoi(e) : UF_LIMIT;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static int table_bits(long long n) {
    int b = 4;
    while ((1ll << b) < n + 1) b++;
    return b;
}

// Scratch layout of one kind: the 0xff-filled part first (parents, table
// keys), then the zero-filled part, then the rest.
namespace {
struct Layout {
    size_t ff_bytes, zero_bytes, total;
    size_t o_tk, o_tchi, o_cnt, o_bcount, o_bfill, o_cchi, o_cpres, o_ck, o_cs, o_bstart, o_bk, o_bs, o_scan;
};
Layout layout(int kind, long long ncap, long long ns) {
    Layout L{};
    const size_t m = (size_t)(ncap > 0 ? ncap : 1);
    const size_t cap = kind == 1 ? 0 : ((size_t)1 << table_bits(ncap));
    size_t p = al256(sizeof(int32_t) * m);   // parents
    L.o_tk = p;
    p += al256(sizeof(uint64_t) * cap);
    L.ff_bytes = p;
    L.o_tchi = p;                            // tchi, tbeta
    p += al256(sizeof(int32_t) * 2 * cap);
    L.o_cnt = p;
    p += al256(sizeof(unsigned long long));
    L.o_bcount = p;
    p += al256(sizeof(int32_t) * (ns + 1));
    L.o_bfill = p;
    p += al256(sizeof(int32_t) * (ns + 1));
    L.o_cchi = p;                            // cchi, cbeta
    p += al256(kind == 1 ? sizeof(int32_t) * 2 * ns : 0);
    L.o_cpres = p;
    p += al256(kind == 1 ? (size_t)ns : 0);
    L.zero_bytes = p - L.ff_bytes;
    L.o_ck = p;
    p += al256(kind == 1 ? 0 : sizeof(uint64_t) * m);
    L.o_cs = p;
    p += al256(kind == 1 ? 0 : sizeof(uint32_t) * m);
    L.o_bk = p;
    p += al256(kind == 1 ? 0 : sizeof(uint64_t) * m);
    L.o_bs = p;
    p += al256(kind == 1 ? 0 : sizeof(uint32_t) * m);
    L.o_bstart = p;
    p += al256(sizeof(int64_t) * (ns + 1));
    L.o_scan = p;
    p += al256(scan_tmp_bytes(ns + 1));
    L.total = p;
    return L;
}
}  // namespace

size_t finalize_tmp_bytes(int kind, long long ncap, long long ns) { return layout(kind, ncap, ns).total; }

void finalize_clear_list(int kind, long long ncap, long long ns, void* tmp, ClearList& C) {
    const Layout L = layout(kind, ncap, ns);
    if (C.n + 2 > 16) return;
    C.p[C.n] = tmp;
    C.bytes[C.n] = (long long)L.ff_bytes;
    C.value[C.n++] = 0xff;
    C.p[C.n] = (char*)tmp + L.ff_bytes;
    C.bytes[C.n] = (long long)L.zero_bytes;
    C.value[C.n++] = 0;
}

void launch_clear(const ClearList& C, cudaStream_t s) {
    long long nmax = 0;
    for (int i = 0; i < C.n; i++) nmax = std::max(nmax, C.bytes[i]);
    if (C.n == 0 || nmax == 0) return;
    const unsigned bx = (unsigned)std::min<long long>((nmax + 16 * 256 - 1) / (16 * 256), 152LL * 8);
    k_clear<<<dim3(bx, (unsigned)C.n), 256, 0, s>>>(C);
    note_launch();
}

void launch_finalize_clear(int kind, long long ncap, long long ns, void* tmp, cudaStream_t s) {
    ClearList C{};
    finalize_clear_list(kind, ncap, ns, tmp, C);
    launch_clear(C, s);
}

void launch_finalize(const ClipArgs& a, int kind, long long n, long long ncap, long long ns, int key_bits,
                     const FinalOut& out, void* tmp, cudaStream_t s) {
    // kind 1: n = the number of pairs; kinds 2..4: n = the record capacity,
    // the record count itself is read on the device (a.rcount)
    const Layout L = layout(kind, ncap, ns);
    char* base = (char*)tmp;
    int32_t* parent = (int32_t*)base;
    int32_t* bcount = (int32_t*)(base + L.o_bcount);
    int32_t* bfill = (int32_t*)(base + L.o_bfill);
    int64_t* bstart = (int64_t*)(base + L.o_bstart);
    void* stmp = base + L.o_scan;
    if (kind == 1) {
        int32_t* cchi = (int32_t*)(base + L.o_cchi);
        int32_t* cbeta = cchi + ns;
        uint8_t* cpres = (uint8_t*)(base + L.o_cpres);
        if (n > 0) {
            k_link_cells<<<nblk(n, 256), 256, 0, s>>>(a, n, parent);
            note_launch();
            k_cell_agg<<<nblk(n, 256), 256, 0, s>>>(a, n, parent, cchi, cbeta, cpres);
            note_launch();
        }
        scan_excl(cpres, bstart, ns, stmp, s);
        k_cell_emit<<<nblk(ns, 256), 256, 0, s>>>(ns, cpres, bstart, cchi, cbeta, out.keys, out.chi, out.beta,
                                                  out.flag, out.count);
        note_launch();
        return;
    }
    const int which = kind - 2;
    const int tb = table_bits(ncap);
    const long long cap = 1ll << tb;
    uint64_t* tk = (uint64_t*)(base + L.o_tk);
    int32_t* tchi = (int32_t*)(base + L.o_tchi);
    int32_t* tbeta = tchi + cap;
    unsigned long long* cnt = (unsigned long long*)(base + L.o_cnt);
    uint64_t* ck = (uint64_t*)(base + L.o_ck);
    uint32_t* cs = (uint32_t*)(base + L.o_cs);
    uint64_t* bk = (uint64_t*)(base + L.o_bk);
    uint32_t* bs = (uint32_t*)(base + L.o_bs);
    const int shift = (kind - 1) * key_bits;   // first sphere of a key
    if (n > 0) {
        if (which < 2) {   // faces and edges have components across tets; vertices are points
            k_link_records<<<nblk(n, 256), 256, 0, s>>>(a, which, n, parent);
            note_launch();
        }
        k_rec_agg<<<nblk(n, 256), 256, 0, s>>>(a, which, n, which < 2 ? parent : nullptr, tk, tchi, tbeta,
                                               (unsigned long long)(cap - 1), 64 - tb);
        note_launch();
    }
    k_table_compact<<<nblk(cap, 256), 256, 0, s>>>(tk, cap, shift, ck, cs, cnt, bcount);
    note_launch();
    scan_excl(bcount, bstart, ns, stmp, s);
    if (n > 0) {
        k_bucket_fill<<<nblk(n, 256), 256, 0, s>>>(ck, cs, cnt, n, shift, bstart, bfill, bk, bs);
        note_launch();
        k_bucket_emit<<<nblk(n, 256), 256, 0, s>>>(bk, bs, cnt, n, kind, key_bits, bstart, tchi, tbeta, out.keys,
                                                   out.chi, out.beta, out.flag);
        note_launch();
    }
    cudaMemcpyAsync(out.count, cnt, sizeof(long long), cudaMemcpyDeviceToDevice, s);
}

void launch_copy_rows(const int32_t* keys, int32_t* d_keys, long long n_keys, const void* vals, void* d_vals,
                      long long n, int elem, cudaStream_t s) {
    const long long total = n_keys + n;
    if (total <= 0 || (!keys && !vals)) return;
    const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 16);
    k_copy_rows<<<blocks, 256, 0, s>>>(keys, d_keys, n_keys, vals, d_vals, n, elem);
    note_launch();
}

void launch_export(const ExportArgs& a, cudaStream_t s) {
    long long nmax = 0;
    for (int i = 0; i < a.nseg; i++) nmax = std::max(nmax, a.seg[i].n);
    if (a.nseg == 0 || nmax == 0) return;
    const unsigned bx = (unsigned)std::min<long long>((nmax + 255) / 256, 152LL * 4);
    k_export<<<dim3(bx, (unsigned)a.nseg), 256, 0, s>>>(a);
    note_launch();
}

void launch_compact_pieces(const ClipArgs& a, long long npairs, const int64_t* off, int32_t* d_tet, int32_t* d_sphere,
                           double* d_vol, double* d_mom, cudaStream_t s) {
    if (npairs <= 0) return;
    k_compact_pieces<<<nblk(npairs, 256), 256, 0, s>>>(a, npairs, off, d_tet, d_sphere, d_vol, d_mom);
    note_launch();
}

// Partial update of the restricted power diagram after spheres are inserted
// (Sec. 4 intro and Sec. 5.2: only the cells related to the new spheres are
// clipped again).
//
// A piece P(t,i) = t cap cell_i depends only on the candidate spheres of its
// tet and on the order they are clipped in: P(t,i) = t cap (intersection over
// k in cand(t) of the radical half-spaces of (i, k)).  After the neighbour
// and candidate stages have run on the enlarged sphere set, every tet whose
// candidate list and clip order are unchanged keeps its pieces, their volumes
// and their fractional Euler records exactly; only the other tets are clipped
// again.  These kernels find the changed tets and carry the unchanged tets'
// per-pair outputs and element records over into the new context's arrays
// (records repacked when the number of bits per sphere index grows), so that
// the finalisation that follows sees exactly what a full build would produce.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "prim.cuh"

namespace {

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }
size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// One warp per tet: compare count, candidate ids and clip order.
__global__ void k_cand_diff(const int32_t* __restrict__ cnt_new, const int32_t* __restrict__ cand_new,
                            const uint8_t* __restrict__ ord_new, const int32_t* __restrict__ cnt_old,
                            const int32_t* __restrict__ cand_old, const uint8_t* __restrict__ ord_old, long long nt,
                            uint8_t* __restrict__ changed, unsigned long long* __restrict__ n_changed) {
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= nt) return;   // warp-uniform
    const int n = cnt_new[t];
    bool diff = n != cnt_old[t];
    if (!diff && lane < n)
        diff = cand_new[t * RPD_MAXC + lane] != cand_old[t * RPD_MAXC + lane] ||
               ord_new[t * RPD_MAXC + lane] != ord_old[t * RPD_MAXC + lane];
    diff = __any_sync(0xffffffffu, diff);
    if (lane == 0) {
        changed[t] = diff ? 1 : 0;
        if (diff) atomicAdd(n_changed, 1ull);
    }
}

// Per pair of an unchanged tet: copy its outputs from the old context's pair
// (same tet, same candidate slot) and count its face and edge records.
__global__ void k_keep_pairs(ClipArgs o, ClipArgs a, long long npairs, const uint8_t* __restrict__ changed,
                             int32_t* __restrict__ kf, int32_t* __restrict__ ke) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const long long t = a.pair_tet[p];
    if (changed[t]) {
        kf[p] = ke[p] = 0;
        return;
    }
    const long long q = o.pair_off[t] + (p - a.pair_off[t]);
    a.pflag[p] = o.pflag[q];
    a.c_val[p] = o.c_val[q];
    a.c_link[p] = o.c_link[q];
    a.p_vol[p] = o.p_vol[q];
    for (int k = 0; k < 3; k++) a.p_mom[3 * p + k] = o.p_mom[3 * q + k];
    a.f_cnt[p] = o.f_cnt[q];
    a.e_cnt[p] = o.e_cnt[q];
    kf[p] = o.f_cnt[q];
    ke[p] = o.e_cnt[q];
}

// Packed key of `arity` sphere indices, `ob` bits each, repacked to `nb` bits.
__device__ __forceinline__ uint64_t repack(uint64_t key, int arity, int ob, int nb) {
    if (ob == nb) return key;
    const uint64_t m = (1ull << ob) - 1;
    uint64_t out = 0;
    for (int k = 0; k < arity; k++) out |= ((key >> (k * ob)) & m) << (k * nb);
    return out;
}

// Face (which = 0) and edge (which = 1) records of unchanged pairs, copied
// to the offsets the scans of kf / ke gave them.
__global__ void k_keep_records(ClipArgs o, ClipArgs a, long long npairs, const uint8_t* __restrict__ changed,
                               const int64_t* __restrict__ off_f, const int64_t* __restrict__ off_e, int ob, int nb) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const long long t = a.pair_tet[p];
    if (changed[t]) return;
    const long long q = o.pair_off[t] + (p - a.pair_off[t]);
    for (int which = 0; which < 2; which++) {
        const int32_t* so = which == 0 ? o.f_off : o.e_off;
        const uint8_t* sc = which == 0 ? o.f_cnt : o.e_cnt;
        const long long dst0 = which == 0 ? off_f[p] : off_e[p];
        const long long src0 = so[q];
        const int n = sc[q];
        if (which == 0) a.f_off[p] = (int32_t)dst0;
        else a.e_off[p] = (int32_t)dst0;
        for (int z = 0; z < n; z++) {
            const long long d = dst0 + z, r = src0 + z;
            if (d >= a.rcap[which]) break;   // the count reports the overflow; the build retries larger
            a.rkey[which][d] = repack(o.rkey[which][r], which + 2, ob, nb);
            a.rtet[which][d] = o.rtet[which][r];
            a.rval[which][d] = o.rval[which][r];
            a.rlink[which][d] = o.rlink[which][r];
            if (which == 1 && a.elen) a.elen[d] = o.elen ? o.elen[r] : 0;
        }
    }
}

__global__ void k_keep_flag_rpv(ClipArgs o, long long n_old, const uint8_t* __restrict__ changed,
                                uint8_t* __restrict__ keep) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_old) return;
    keep[r] = changed[o.rtet[2][r]] ? 0 : 1;
}

__global__ void k_keep_rpv(ClipArgs o, ClipArgs a, long long n_old, const uint8_t* __restrict__ keep,
                           const int64_t* __restrict__ pos, int ob, int nb) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_old || !keep[r]) return;
    const long long d = pos[r];
    if (d >= a.rcap[2]) return;
    a.rkey[2][d] = repack(o.rkey[2][r], 4, ob, nb);
    a.rtet[2][d] = o.rtet[2][r];
    a.rval[2][d] = o.rval[2][r];
    a.rlink[2][d] = o.rlink[2][r];
}

__global__ void k_set_counts(unsigned long long* __restrict__ rcount, const int64_t* __restrict__ off_f,
                             const int64_t* __restrict__ off_e, const int64_t* __restrict__ pos_v, long long npairs,
                             long long n_old_v) {
    rcount[0] = (unsigned long long)off_f[npairs];
    rcount[1] = (unsigned long long)off_e[npairs];
    rcount[2] = (unsigned long long)pos_v[n_old_v];
}

}  // namespace

void launch_cand_diff(const int32_t* cnt_new, const int32_t* cand_new, const uint8_t* ord_new, const int32_t* cnt_old,
                      const int32_t* cand_old, const uint8_t* ord_old, long long nt, uint8_t* changed,
                      unsigned long long* n_changed, cudaStream_t s) {
    cudaMemsetAsync(n_changed, 0, sizeof(unsigned long long), s);
    if (nt == 0) return;
    k_cand_diff<<<nblk(32 * nt, 256), 256, 0, s>>>(cnt_new, cand_new, ord_new, cnt_old, cand_old, ord_old, nt,
                                                    changed, n_changed);
    note_launch();
}

size_t keep_tmp_bytes(long long npairs, long long n_old_rpv) {
    const long long n = npairs + 1, m = n_old_rpv + 1;
    return 2 * al(sizeof(int32_t) * n) + 2 * al(sizeof(int64_t) * n) + al(sizeof(uint8_t) * m) +
           al(sizeof(int64_t) * m) + al(scan_tmp_bytes(n > m ? n : m));
}

void launch_keep(const ClipArgs& o, long long n_old_rpv, const ClipArgs& a, long long npairs,
                 const uint8_t* changed, int ob, int nb, void* tmp, cudaStream_t s) {
    // with more than 16 bits per sphere index the old context wrote no vertex
    // records (only counted them): there is nothing to carry over
    if (4 * ob > 64) n_old_rpv = 0;
    char* p = (char*)tmp;
    const long long n = npairs + 1, m = n_old_rpv + 1;
    int32_t* kf = (int32_t*)p; p += al(sizeof(int32_t) * n);
    int32_t* ke = (int32_t*)p; p += al(sizeof(int32_t) * n);
    int64_t* off_f = (int64_t*)p; p += al(sizeof(int64_t) * n);
    int64_t* off_e = (int64_t*)p; p += al(sizeof(int64_t) * n);
    uint8_t* keep = (uint8_t*)p; p += al(sizeof(uint8_t) * m);
    int64_t* pos_v = (int64_t*)p; p += al(sizeof(int64_t) * m);
    void* stmp = p;
    if (npairs > 0) {
        k_keep_pairs<<<nblk(npairs, 256), 256, 0, s>>>(o, a, npairs, changed, kf, ke);
        note_launch();
    }
    scan_excl(kf, off_f, npairs, stmp, s);
    scan_excl(ke, off_e, npairs, stmp, s);
    if (npairs > 0) {
        k_keep_records<<<nblk(npairs, 256), 256, 0, s>>>(o, a, npairs, changed, off_f, off_e, ob, nb);
        note_launch();
    }
    if (n_old_rpv > 0) {
        k_keep_flag_rpv<<<nblk(n_old_rpv, 256), 256, 0, s>>>(o, n_old_rpv, changed, keep);
        note_launch();
    }
    scan_excl(keep, pos_v, n_old_rpv, stmp, s);
    if (n_old_rpv > 0 && 4 * nb <= 64) {
        k_keep_rpv<<<nblk(n_old_rpv, 256), 256, 0, s>>>(o, a, n_old_rpv, keep, pos_v, ob, nb);
        note_launch();
    }
    k_set_counts<<<1, 1, 0, s>>>(a.rcount, off_f, off_e, pos_v, npairs, n_old_rpv);
    note_launch();
}

// rpd_euler_static: the restricted power diagram and the Euler characteristic
// of one element kind, computed with no device allocation at all.
//
// Some callers cannot call cudaMalloc when they need a result: pipelines that
// fix their device-memory budget up front and may not grow it later, or code
// that runs where an allocation could fail or stall at the wrong moment (a
// memory pool shared with other work, a long-running service that must not
// fragment the device heap).  This entry point runs the same kernels as
// rpd_build and rpd_euler, but carves every workspace buffer out of one
// file-scope device
// array of RPD_STATIC_SCRATCH_BYTES (32 MiB), which every GPU that loads the
// library holds until the process exits.  Problems whose workspace does not
// fit are rejected with RPD_E_OVERFLOW before the stage that would need more.
//
// In host code `g_scratch` only names the symbol; its device address is
// looked up with cudaGetSymbolAddress at every call (a host-side lookup with
// no device work), so a module reloaded after cudaDeviceReset is seen.  The
// call synchronises its stream three times (the sizes of the later stages are
// read on the host).  All calls
// share the array and it keeps the previous call's contents, so every buffer
// that must start at zero is cleared here, and calls that overlap on the GPU
// (other streams or host threads) race with each other.
#include <cuda_runtime.h>
#include <math.h>


#include "internal.cuh"
#include "prim.cuh"
#include "rpd.h"

#define RPD_STATIC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_scratch[RPD_STATIC_SCRATCH_BYTES];

namespace {

// Device address of the scratch array on the current device.
cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Arena {
    char* base;
    size_t used;
    bool full;
    template <typename T>
    T* take(size_t count) {
        size_t bytes = (sizeof(T) * (count ? count : 1) + 255) & ~(size_t)255;
        if (full || used + bytes > RPD_STATIC_SCRATCH_BYTES) {
            full = true;
            return nullptr;
        }
        T* p = (T*)(base + used);
        used += bytes;
        return p;
    }
};

// Errors are reported by status code only (no message storage, which could
// allocate host memory).
rpd_status fail_static(rpd_status s, const char* /*why*/) { return s; }

rpd_status read_status(DevState* st, cudaStream_t s) {
    DevState h;
    if (cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return fail_static(RPD_E_CUDA, "CUDA error in rpd_euler_static");
    }
    if (h.err) return fail_static((rpd_status)h.err, "device-side error (see rpd_build for the same input)");
    return RPD_OK;
}

#define NEED_S(ptr)                                                                                         \
    do {                                                                                                    \
        if (!(ptr)) return fail_static(RPD_E_OVERFLOW, "problem exceeds the 32 MiB static scratch array"); \
    } while (0)

#define TRY_S(expr)                      \
    do {                                 \
        rpd_status _s = (expr);          \
        if (_s != RPD_OK) return _s;     \
    } while (0)

int sphere_bits(long long ns) {
    int b = 1;
    while ((1ll << b) - 1 <= ns) b++;
    return b;
}

}  // namespace

extern "C" rpd_status rpd_euler_static(const double* d_verts, int64_t nv, const int32_t* d_tets, int64_t nt,
                                       const double* d_centers, const double* d_radii, int64_t ns,
                                       const rpd_options* opt, void* cuda_stream, rpd_kind kind, int32_t* d_keys,
                                       int32_t* d_chi, int64_t cap, int64_t* n_out) {
    rpd_options o;
    rpd_default_options(&o);
    if (opt) o = *opt;
    if (nv < 4 || nv >= (1ll << 21) || nt < 1 || nt >= (1ll << 26) || ns < 1 || ns >= (1ll << 21))
        return fail_static(RPD_E_INVALID, "sizes out of range");
    if (!d_verts || !d_tets || !d_centers || !d_radii || !n_out) return fail_static(RPD_E_INVALID, "null pointer");
    if (kind < 1 || kind > 4 || o.k < 1 || o.k > RPD_MAXK || o.grid_bits < 0 || o.grid_bits > 40)
        return fail_static(RPD_E_INVALID, "bad kind or options");
    if (o.precision != RPD_FP64 && o.precision != RPD_FP32_FILTERED) return fail_static(RPD_E_INVALID, "unknown precision");
    const int b = sphere_bits(ns);
    if (kind == 4 && 4 * b > 64) return fail_static(RPD_E_OVERFLOW, "RPV keys need at most 2^16 - 1 spheres");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        cudaGetLastError();
        return fail_static(RPD_E_CUDA, "cudaGetSymbolAddress failed for the static scratch array");
    }
    Arena ar{(char*)base, 0, false};
    const int K = o.k;
    // ---- A0-A2 (same kernels as rpd_build)
    DevState* st = ar.take<DevState>(1);
    int32_t* Xi = ar.take<int32_t>(3 * nv);
    int32_t* Ci = ar.take<int32_t>(3 * ns);
    long long* W = ar.take<long long>(ns);
    int32_t* adj = ar.take<int32_t>(4 * nt);
    uint32_t* own = ar.take<uint32_t>(nt);
    int32_t* tets = ar.take<int32_t>(4 * nt);
    void* ptmp = ar.take<char>(prep_tmp_bytes(nt, nv));
    const long long ncap = 2 * ns + 64;
    GridParams* gp = ar.take<GridParams>(1);
    int64_t* cell_start = ar.take<int64_t>(ncap + 1);
    int32_t* cell_ids = ar.take<int32_t>(ns);
    int4* cell_sph = ar.take<int4>(ns);
    long long* cell_w = ar.take<long long>(ns);
    long long* cell_wmax = ar.take<long long>(2 * ncap);
    void* gtmp = ar.take<char>(grid_tmp_bytes(ns, ncap));
    int32_t* knn = ar.take<int32_t>(nv * K);
    long long* dplus = ar.take<long long>(nv);
    void* ktmp = ar.take<char>(knn_tmp_bytes(nv));
    int32_t* cand_cnt = ar.take<int32_t>(nt);
    int32_t* cand = ar.take<int32_t>(nt * RPD_MAXC);
    uint8_t* cand_ord = ar.take<uint8_t>(nt * RPD_MAXC);
    int32_t* fb_list = ar.take<int32_t>(nt);
    int32_t* fb_count = ar.take<int32_t>(1);
    int64_t* pair_off = ar.take<int64_t>(nt + 1);
    void* stmp = ar.take<char>(scan_tmp_bytes(nt + 1));
    int32_t* bin_count = ar.take<int32_t>(RPD_NBINS);
    int32_t* bin_fill = ar.take<int32_t>(RPD_NBINS);
    NEED_S(!ar.full);
    cudaMemsetAsync(st, 0, sizeof(DevState), s);
    cudaMemcpyAsync(tets, d_tets, sizeof(int32_t) * 4 * nt, cudaMemcpyDeviceToDevice, s);
    launch_snap(d_verts, nv, d_centers, d_radii, ns, o.grid_bits, Xi, Ci, W, st, s);
    launch_prep_mesh(tets, nt, nv, Xi, adj, own, ptmp, st, s);
    launch_sphere_grid(Ci, W, ns, ncap, gp, cell_start, cell_ids, cell_sph, cell_w, cell_wmax, gtmp, s);
    launch_knn(Xi, nv, ns, gp, cell_start, cell_sph, cell_w, cell_wmax, ncap, K, knn, dplus, ktmp, &st->err,
               (o.debug_checks & 4) != 0, s);
    launch_candidates(tets, nt, nv, Xi, Ci, W, knn, dplus, K, gp, cell_start, cell_ids, cell_wmax, cand_cnt, cand,
                      cand_ord, fb_list, fb_count, st, s);
    scan_excl(cand_cnt, pair_off, nt, stmp, s);
    launch_bin_count(cand_cnt, nt, bin_count, s);
    long long npairs = 0;
    int32_t hb[RPD_NBINS];
    cudaMemcpyAsync(&npairs, pair_off + nt, sizeof(long long), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(hb, bin_count, sizeof(hb), cudaMemcpyDeviceToHost, s);
    TRY_S(read_status(st, s));
    // ---- A3-A4
    ClipArgs a{};
    int32_t* pair_tet = ar.take<int32_t>(npairs);
    int32_t* bins = ar.take<int32_t>(npairs);
    unsigned long long* rcount = ar.take<unsigned long long>(3);
    unsigned long long* qcount = ar.take<unsigned long long>(RPD_NBINS);
    a.tets = tets;
    a.Xi = Xi;
    a.Ci = Ci;
    a.W = W;
    a.own = own;
    a.adj = adj;
    a.cand_cnt = cand_cnt;
    a.cand = cand;
    a.cand_ord = cand_ord;
    a.pair_off = pair_off;
    a.pair_tet = pair_tet;
    a.unit = ldexp(1.0, -o.grid_bits);
    a.pflag = ar.take<uint8_t>(npairs);
    a.c_val = ar.take<int32_t>(npairs);
    a.c_link = ar.take<uint8_t>(npairs);
    a.p_vol = ar.take<double>(npairs);
    a.p_mom = ar.take<double>(3 * npairs);
    a.f_off = ar.take<int32_t>(npairs);
    a.f_cnt = ar.take<uint8_t>(npairs);
    a.e_off = ar.take<int32_t>(npairs);
    a.e_cnt = ar.take<uint8_t>(npairs);
    a.rcount = rcount;
    a.key_bits = b;
    a.force_slow = o.debug_checks & 3;
    a.uf_limit = uf_iteration_limit();
    a.st = st;
    const long long rc[3] = {3 * npairs + 1024, 2 * npairs + 1024, npairs / 2 + 1024};
    for (int k = 0; k < 3; k++) {
        a.rcap[k] = rc[k];
        a.rkey[k] = ar.take<uint64_t>(rc[k]);
        a.rtet[k] = ar.take<int32_t>(rc[k]);
        a.rval[k] = ar.take<int16_t>(rc[k]);
        a.rlink[k] = ar.take<uint8_t>(rc[k]);
    }
    int32_t* qpair[RPD_NBINS] = {};
    uint8_t* qnv[RPD_NBINS] = {};
    uint32_t* qtrip[RPD_NBINS] = {};
    for (int bb = 1; bb < RPD_NBINS; bb++) {
        if (!hb[bb]) continue;
        qpair[bb] = ar.take<int32_t>(hb[bb]);
        qnv[bb] = ar.take<uint8_t>(hb[bb]);
        qtrip[bb] = ar.take<uint32_t>(2LL * hb[bb] * clip_vmax(bb));
    }
    NEED_S(!ar.full);
    launch_bin_pairs(cand_cnt, pair_off, nt, pair_tet, bins, bin_count, bin_fill, npairs, rcount, qcount, s);
    long long off = 0;
    for (int bb = 0; bb < RPD_NBINS; bb++) {
        const long long nb = hb[bb];
        if (bb == 0) {
            launch_whole_tets(a, bins, bin_count, nb, s);
        } else if (nb > 0) {
            ClipArgs ab = a;
            ab.qpair = qpair[bb];
            ab.qnv = qnv[bb];
            ab.qtrip = qtrip[bb];
            ab.qcap = nb;
            ab.qcount = qcount + bb;
            launch_clip(ab, bb, o.precision, bins + off, bin_count + bb, nb, s);
            launch_records(ab, bb, nb, s);
        }
        off += nb;
    }
    unsigned long long cnt[3];
    cudaMemcpyAsync(cnt, rcount, sizeof(cnt), cudaMemcpyDeviceToHost, s);
    TRY_S(read_status(st, s));
    for (int k = 0; k < 3; k++)
        if ((long long)cnt[k] > rc[k]) return fail_static(RPD_E_OVERFLOW, "element records exceed their capacity");
    // ---- A5-A7 for the requested kind
    const long long n = kind == 1 ? npairs : (long long)cnt[kind - 2];
    const long long rows = kind == 1 ? ns : n;
    FinalOut fo;
    fo.keys = ar.take<int32_t>(rows * kind);
    fo.chi = ar.take<int32_t>(rows);
    fo.beta = ar.take<int32_t>(rows);
    fo.flag = ar.take<uint8_t>(rows);
    fo.count = ar.take<long long>(1);
    void* ftmp = ar.take<char>(finalize_tmp_bytes(kind, n, ns));
    NEED_S(!ar.full);
    launch_finalize_clear(kind, n, ns, ftmp, s);
    launch_finalize(a, kind, n, n, ns, b, fo, ftmp, s);
    long long m = 0;
    cudaMemcpyAsync(&m, fo.count, sizeof(long long), cudaMemcpyDeviceToHost, s);
    TRY_S(read_status(st, s));
    *n_out = m;
    if (!d_keys && !d_chi) return RPD_OK;
    if (cap < m) return fail_static(RPD_E_INVALID, "cap is smaller than the number of elements");
    if (d_keys && m) cudaMemcpyAsync(d_keys, fo.keys, sizeof(int32_t) * m * kind, cudaMemcpyDeviceToDevice, s);
    if (d_chi && m) cudaMemcpyAsync(d_chi, fo.chi, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return fail_static(RPD_E_CUDA, "CUDA error in rpd_euler_static");
    }
    return RPD_OK;
}

// C-ABI of librpd: context lifecycle, orchestration of the stages, outputs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"
#include "prim.cuh"
#include "rpd.h"

namespace {

thread_local std::string g_build_error;

// Optional host-side allocation-failure injection for tests:
// RPD_FAIL_ALLOC_AFTER=N makes the (N+1)-th device allocation of a build fail.
long long alloc_budget() {
    static const long long budget = [] {
        const char* e = getenv("RPD_FAIL_ALLOC_AFTER");
        return e ? atoll(e) : -1ll;
    }();
    return budget;
}

std::atomic<long long> g_launches{0};

// Timing events are recycled per device: a context takes its events from the
// pool and returns them, all completed, when it is destroyed.
struct EventPool {
    std::mutex mu;
    std::vector<cudaEvent_t> free_ev[64];
};
EventPool& event_pool() {
    static EventPool p;
    return p;
}
bool acquire_events(int dev, cudaEvent_t* out, int n) {
    EventPool& P = event_pool();
    std::lock_guard<std::mutex> lock(P.mu);
    for (int k = 0; k < n; k++) {
        if (!P.free_ev[dev].empty()) {
            out[k] = P.free_ev[dev].back();
            P.free_ev[dev].pop_back();
        } else if (cudaEventCreate(&out[k]) != cudaSuccess) {
            out[k] = nullptr;
            return false;
        }
    }
    return true;
}
void release_events(int dev, cudaEvent_t* ev, int n) {
    EventPool& P = event_pool();
    std::lock_guard<std::mutex> lock(P.mu);
    for (int k = 0; k < n; k++)
        if (ev[k]) P.free_ev[dev].push_back(ev[k]);
}

// One stream-ordered memory pool per device, owned by the library, that keeps
// freed workspace cached (release threshold = max) so that repeated builds
// reuse it instead of mapping fresh memory at every synchronisation.
cudaMemPool_t library_pool() {
    static cudaMemPool_t pools[64];
    static std::atomic<bool> ready[64];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (ready[dev].load(std::memory_order_acquire)) return pools[dev];
    std::lock_guard<std::mutex> lock(mu);   // first use on this device: create it once
    if (!ready[dev].load(std::memory_order_relaxed)) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&pools[dev], &props) != cudaSuccess) return nullptr;
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &thr);
        ready[dev].store(true, std::memory_order_release);
    }
    return pools[dev];
}

}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct rpd_ctx {
    cudaStream_t stream = nullptr;
    rpd_options opt{};
    long long nv = 0, nt = 0, ns = 0, npairs = 0;
    int key_bits = 1;
    int K = 16;
    std::string last_error;
    std::vector<void*> allocs;
    long long nalloc = 0;
    bool failed_alloc = false;

    // device state
    DevState* st = nullptr;
    int32_t *Xi = nullptr, *Ci = nullptr;
    long long* W = nullptr;
    int32_t* adj = nullptr;
    uint32_t* own = nullptr;
    int32_t* tets = nullptr;
    GridParams* gp = nullptr;
    int64_t* cell_start = nullptr;
    int32_t* cell_ids = nullptr;
    long long* cell_wmax = nullptr;
    int32_t* knn = nullptr;
    long long* dplus = nullptr;
    int32_t *cand_cnt = nullptr, *cand = nullptr, *fb_list = nullptr, *fb_count = nullptr;
    uint8_t* cand_ord = nullptr;
    int64_t* pair_off = nullptr;
    int32_t *pair_tet = nullptr, *bins = nullptr, *bin_count = nullptr, *bin_fill = nullptr;
    long long hbin[RPD_NBINS] = {};
    int32_t* qpair[RPD_NBINS] = {};
    uint8_t* qnv[RPD_NBINS] = {};
    uint32_t* qtrip[RPD_NBINS] = {};
    unsigned long long* qcount = nullptr;
    ClipArgs clip{};
    unsigned long long* rcount = nullptr;
    long long nrec[3] = {0, 0, 0};
    // finalised elements per kind (index kind-1)
    long long nkeys[4] = {0, 0, 0, 0};
    bool kind_ok[4] = {true, true, true, true};
    FinalOut fout[4] = {};
    int64_t* piece_off = nullptr;
    long long npieces = 0;
    // finalisation scratch per kind (union-find parents first), kept for the
    // repair queries, and its capacity
    void* ftmp[4] = {nullptr, nullptr, nullptr, nullptr};
    long long fcap[4] = {0, 0, 0, 0};
    // partial update: tets whose candidates changed (NULL after a full build)
    uint8_t* changed = nullptr;
    unsigned long long* d_nchanged = nullptr;
    // boundary faces (4 t + f) the repair loop has grown spheres from; pins
    // skip them (carried over by partial updates)
    uint8_t* used_faces = nullptr;
    // per-RPE-key summed segment lengths (fixed point), computed on first query
    long long* edge_len = nullptr;
    // boundary triangles of the mesh for sphere shrinking (built on first use)
    double* btri = nullptr;
    int32_t* btri_face = nullptr;
    float4* btri_ball = nullptr;   // FP32 bounding balls of the boundary triangles
    long long nbtri = -1;
    // batches (rpd_build_batch): shape offsets of vertices, tets and spheres
    // (device copies and the host's), and the largest per-shape grid
    int nshapes = 1;
    long long *d_voff = nullptr, *d_toff = nullptr, *d_soff = nullptr;
    std::vector<long long> h_voff, h_toff, h_soff;
    long long max_shape_ncap = 0;
    // mesh bounding box (world units), computed on first use
    bool have_bbox = false;
    double bb_lo[3] = {0, 0, 0}, bb_hi[3] = {0, 0, 0};
    // learned radius proposer used by the repair loops (not owned) and the
    // sphere-shrinking work they did: pins, iterations, rejected proposals
    rpd_mlp* proposer = nullptr;
    double proposer_margin = 1.25;
    long long shrink_pins = 0, shrink_iters = 0, shrink_restarts = 0;
    rpd_stats stats{};
    bool timed = false;   // stats' stage times filled in
    int device = 0;
    cudaEvent_t ev[16] = {};
    // clip stage: fork, end of each bin's clip kernel, end of each bin's work
    cudaEvent_t evc[1 + 2 * RPD_NBINS] = {};

    // Optional chunk that alloc carves from before it asks the pool: one pool
    // call instead of dozens after the pair count is known.
    char* chunk = nullptr;
    size_t chunk_size = 0, chunk_off = 0;

    template <typename T>
    T* alloc(size_t count) {
        size_t bytes = sizeof(T) * (count ? count : 1);
        long long budget = alloc_budget();
        if (budget >= 0 && nalloc >= budget) {
            failed_alloc = true;
            return nullptr;
        }
        const size_t rounded = (bytes + 255) & ~(size_t)255;
        if (chunk && chunk_off + rounded <= chunk_size) {
            T* q = (T*)(chunk + chunk_off);
            chunk_off += rounded;
            nalloc++;
            return q;
        }
        void* p = nullptr;
        cudaMemPool_t pool = library_pool();
        if (!pool || cudaMallocFromPoolAsync(&p, bytes, pool, stream) != cudaSuccess) {
            cudaGetLastError();
            failed_alloc = true;
            return nullptr;
        }
        nalloc++;
        allocs.push_back(p);
        return (T*)p;
    }
    // Reserve one chunk of `bytes` for the allocations that follow.
    bool reserve(size_t bytes) {
        char* p = alloc<char>(bytes);
        if (!p) return false;
        chunk = p;
        chunk_size = bytes;
        chunk_off = 0;
        return true;
    }
    void release_all() {
        for (void* p : allocs) cudaFreeAsync(p, stream);
        allocs.clear();
        chunk = nullptr;
    }
};

namespace {

rpd_status fail(rpd_ctx* c, rpd_status s, const std::string& msg) {
    if (c) c->last_error = msg;
    return s;
}

const char* dev_reason(int code, const unsigned long long* cnt) {
    switch (code) {
        case RPD_E_INVALID: return "invalid input: coordinate or radius off the supported grid range, NaN, index out of range, or a tet that is not positively oriented";
        case RPD_E_NONMANIFOLD: return "non-manifold mesh: a triangle is shared by more than two tets";
        case RPD_E_DEGENERATE:
            return cnt[CNT_LINK_MISSING] ? "inconsistent restricted element across a shared tet face (input not in generic position)"
                                         : "input not in generic position: an exact predicate is zero (a vertex lies on a radical plane)";
        case RPD_E_OVERFLOW: return "more than 32 candidate spheres for one tet";
        case RPD_E_TIMEOUT:
            return cnt[CNT_UF_LIMIT] ? "union-find iteration bound reached"
                                     : "bounded wait ran out (radix-sort look-back)";
        default: return "device error";
    }
}

// Read the device status block; returns RPD_OK or the first device error.
// Synchronise the stream and read the device status: counters into the
// stats, and an error raised on the device as the return value (with
// raise == false the error code is only left in *code).
rpd_status check_device(rpd_ctx* c, bool raise = true, int* code = nullptr) {
    DevState h;
    if (cudaMemcpyAsync(&h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, RPD_E_CUDA, "CUDA error while reading the device status");
    }
    c->stats.pred_fast = (int64_t)h.cnt[CNT_PRED_FAST];
    c->stats.pred_fp64 = (int64_t)h.cnt[CNT_PRED_FP64];
    c->stats.pred_exact = (int64_t)h.cnt[CNT_PRED_EXACT];
    c->stats.cand_fallback = (int64_t)h.cnt[CNT_CAND_FALLBACK];
    c->stats.whole_tets = (int64_t)h.cnt[CNT_WHOLE];
    for (int k = 0; k < 3; k++) c->stats.clip_vertices[k] = (int64_t)h.cnt[CNT_NEWVERT1 + k];
    if (code) *code = h.err;
    if (raise && h.err != 0) return fail(c, (rpd_status)h.err, dev_reason(h.err, h.cnt));
    return RPD_OK;
}

rpd_status cuda_check(rpd_ctx* c, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, RPD_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return RPD_OK;
}

int bits_for(long long ns) {
    int b = 1;
    while ((1ll << b) - 1 <= ns) b++;   // index ns-1 < 2^b - 1 leaves a sentinel
    return b;
}

#define TRY(expr)                         \
    do {                                  \
        rpd_status _s = (expr);           \
        if (_s != RPD_OK) return _s;      \
    } while (0)

#define NEED(ptr)                                                             \
    do {                                                                      \
        if (!(ptr)) return fail(c, RPD_E_OOM, "device allocation failed");    \
    } while (0)

// Library-owned side streams, per device: the clip bins run side by side (the
// few heavy pairs of the high bins are latency-bound and overlap with the
// throughput-bound low bins), as do the mesh combinatorics next to the kNN and
// the four element kinds of the finalisation.  Each context orders its work on
// them with its own events.
struct BinStreams {
    bool ready = false;
    cudaStream_t s[RPD_NBINS];
    cudaStream_t util;     // high priority: clearing scratch next to the clip
    cudaStream_t fin[4];   // high priority: the element kinds, ahead of the volume pass
};

BinStreams* bin_streams() {
    static BinStreams per_dev[64];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    BinStreams& b = per_dev[dev];
    if (!b.ready) {
        for (int k = 0; k < RPD_NBINS; k++)
            if (cudaStreamCreateWithFlags(&b.s[k], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&b.util, cudaStreamNonBlocking, hi) != cudaSuccess) return nullptr;
        for (int k = 0; k < 4; k++)
            if (cudaStreamCreateWithPriority(&b.fin[k], cudaStreamNonBlocking, hi) != cudaSuccess) return nullptr;
        b.ready = true;
    }
    return &b;
}

// Make the caller's stream wait for everything this context queued on the
// side streams (an event never recorded is already complete).
void join_side_streams(rpd_ctx* c) {
    for (cudaEvent_t e : c->ev)
        if (e) cudaStreamWaitEvent(c->stream, e, 0);
    for (cudaEvent_t e : c->evc)
        if (e) cudaStreamWaitEvent(c->stream, e, 0);
}

// The record and queue counters are zeroed here when asked (the binning
// zeroes them before the first pass; a partial update sets the record
// counters to the records it kept).
rpd_status run_clip(rpd_ctx* c, bool zero_rcount, bool zero_qcount) {
    cudaStream_t s = c->stream;
    if (zero_rcount) cudaMemsetAsync(c->rcount, 0, sizeof(unsigned long long) * 3, s);
    if (zero_qcount) cudaMemsetAsync(c->qcount, 0, sizeof(unsigned long long) * RPD_NBINS, s);
    long long off[RPD_NBINS + 1];
    off[0] = 0;
    for (int b = 0; b < RPD_NBINS; b++) off[b + 1] = off[b] + c->hbin[b];
    BinStreams* bs = bin_streams();
    if (!bs) return fail(c, RPD_E_CUDA, "stream creation failed");
    cudaEventRecord(c->evc[0], s);   // fork
    // heaviest bins first
    for (int b = RPD_NBINS - 1; b >= 0; b--) {
        const long long n = c->hbin[b];
        if (n == 0) continue;
        cudaStream_t sb = bs->s[b];
        cudaStreamWaitEvent(sb, c->evc[0], 0);
        ClipArgs a = c->clip;
        if (b == 0) {
            launch_whole_tets(a, c->bins, c->bin_count, n, sb);
            cudaEventRecord(c->evc[1 + b], sb);
        } else {
            a.qpair = c->qpair[b];
            a.qnv = c->qnv[b];
            a.qtrip = c->qtrip[b];
            a.qcap = n;
            a.qcount = c->qcount + b;
            launch_clip(a, b, c->opt.precision, c->bins + off[b], c->bin_count + b, n, sb);
            launch_records(a, b, n, sb);
            cudaEventRecord(c->evc[1 + b], sb);
            // the bin's volume pass follows its records on the same stream,
            // beside the other bins' clips (latency-bound, so the SMs have
            // room), and joins at the end of the build
            launch_volume(a, b, c->opt.precision, n, sb);
        }
        cudaEventRecord(c->evc[1 + RPD_NBINS + b], sb);
        // the records (what the finalisation reads) are complete once the
        // record kernel is
        cudaStreamWaitEvent(s, c->evc[1 + b], 0);
    }
    return cuda_check(c, "clip launch");
}

// Output and scratch buffers of one kind's finalisation, for up to ncap
// pieces (kind 1) or records.
rpd_status finalize_alloc(rpd_ctx* c, int kind, long long* d_count, long long ncap, void** tmp) {
    const int b = c->key_bits;
    FinalOut& o = c->fout[kind - 1];
    o.count = d_count;
    *tmp = nullptr;
    if (kind == 4 && 4 * b > 64) {
        c->kind_ok[3] = false;
        return RPD_OK;
    }
    const long long rows = kind == 1 ? c->ns : ncap;
    o.keys = c->alloc<int32_t>(rows * kind);
    o.chi = c->alloc<int32_t>(rows);
    o.beta = c->alloc<int32_t>(rows);
    o.flag = c->alloc<uint8_t>(rows);
    *tmp = c->alloc<char>(finalize_tmp_bytes(kind, ncap, c->ns));
    NEED(o.keys && o.chi && o.beta && o.flag && *tmp);
    return RPD_OK;
}

void record(rpd_ctx* c, int k) { cudaEventRecord(c->ev[k], c->stream); }

float elapsed(rpd_ctx* c, int a, int b) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, c->ev[a], c->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return ms;
}

rpd_status build_rest(rpd_ctx* c, rpd_ctx* old);

// Device, timing events and side streams of a context; the chunk for every
// buffer sized before the pair count is known.
rpd_status begin(rpd_ctx* c) {
    const long long nv = c->nv, nt = c->nt, ns = c->ns;
    if (cudaGetDevice(&c->device) != cudaSuccess || c->device < 0 || c->device >= 64)
        return fail(c, RPD_E_CUDA, "no usable current device");
    if (!acquire_events(c->device, c->ev, 16) || !acquire_events(c->device, c->evc, 1 + 2 * RPD_NBINS))
        return fail(c, RPD_E_CUDA, "cudaEventCreate failed");
    // side streams: mesh combinatorics next to the sphere grid and kNN, the
    // clip bins, and the four element kinds of the finalisation
    if (!bin_streams()) return fail(c, RPD_E_CUDA, "stream creation failed");
    record(c, 0);
    const long long ncap = 2 * ns + 64, pcap = 4 * nt + 1024;
    const size_t est = sizeof(DevState) + 4 * 3 * (nv + ns) + 8 * ns + 4 * 4 * nt + 4 * nt + 4 * 4 * nt +
                       prep_tmp_bytes(nt, nv) + sizeof(GridParams) + 8 * (ncap + 1) + 4 * ns + 8 * 2 * ncap +
                       grid_tmp_bytes(ns, ncap) + 4 * nv * c->K + 8 * nv + 16 * ns + 8 * ns + knn_tmp_bytes(nv) +
                       4 * nt + (4 + 1) * nt * RPD_MAXC + 4 * nt + 4 + 8 * (nt + 1) + scan_tmp_bytes(nt + 1) +
                       8 * RPD_NBINS + 8 * pcap + 8 * (3 + RPD_NBINS) + nt + 8 + 42 * 256;
    NEED(c->reserve(est));
    return RPD_OK;
}

rpd_status build(rpd_ctx* c, const double* d_verts, const int32_t* d_tets, const double* d_centers,
                 const double* d_radii) {
    cudaStream_t s = c->stream;
    const long long nv = c->nv, nt = c->nt, ns = c->ns;
    TRY(begin(c));
    BinStreams* bs = bin_streams();
    c->st = c->alloc<DevState>(1);
    c->Xi = c->alloc<int32_t>(3 * nv);
    c->Ci = c->alloc<int32_t>(3 * ns);
    c->W = c->alloc<long long>(ns);
    c->adj = c->alloc<int32_t>(4 * nt);
    c->own = c->alloc<uint32_t>(nt);
    c->tets = c->alloc<int32_t>(4 * nt);
    NEED(c->st && c->Xi && c->Ci && c->W && c->adj && c->own && c->tets);
    cudaMemsetAsync(c->st, 0, sizeof(DevState), s);
    cudaMemcpyAsync(c->tets, d_tets, sizeof(int32_t) * 4 * nt, cudaMemcpyDeviceToDevice, s);
    // ---- A0
    launch_snap(d_verts, nv, d_centers, d_radii, ns, c->opt.grid_bits, c->Xi, c->Ci, c->W, c->st, s);
    size_t tmp_bytes = prep_tmp_bytes(nt, nv);
    void* tmp = c->alloc<char>(tmp_bytes);
    NEED(tmp);
    if (c->nshapes > 1) {
        // batch: shape offsets on the device, every tet inside its own shape (checked before the mesh
        // combinatorics start, so a cross-shape tet reports RPD_E_INVALID first)
        const int S = c->nshapes;
        c->d_voff = c->alloc<long long>(S + 1);
        c->d_toff = c->alloc<long long>(S + 1);
        c->d_soff = c->alloc<long long>(S + 1);
        NEED(c->d_voff && c->d_toff && c->d_soff);
        cudaMemcpyAsync(c->d_voff, c->h_voff.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(c->d_toff, c->h_toff.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(c->d_soff, c->h_soff.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice, s);
        launch_batch_check(c->tets, c->d_toff, c->d_voff, S, nt, c->st, s);
    }
    record(c, 1);
    cudaStreamWaitEvent(bs->s[0], c->ev[1], 0);
    launch_prep_mesh(c->tets, nt, nv, c->Xi, c->adj, c->own, tmp, c->st, bs->s[0]);
    cudaEventRecord(c->ev[2], bs->s[0]);
    TRY(cuda_check(c, "prep launch"));
    return build_rest(c, nullptr);
}

// A0 of a partial update: the mesh tables and the old spheres come from the
// old context, the new spheres are snapped after them.
rpd_status update(rpd_ctx* c, rpd_ctx* old, const double* d_centers, const double* d_radii, long long n_new) {
    cudaStream_t s = c->stream;
    const long long nv = c->nv, nt = c->nt, ns0 = old->ns;
    TRY(begin(c));
    c->st = c->alloc<DevState>(1);
    c->Xi = c->alloc<int32_t>(3 * nv);
    c->Ci = c->alloc<int32_t>(3 * c->ns);
    c->W = c->alloc<long long>(c->ns);
    c->adj = c->alloc<int32_t>(4 * nt);
    c->own = c->alloc<uint32_t>(nt);
    c->tets = c->alloc<int32_t>(4 * nt);
    NEED(c->st && c->Xi && c->Ci && c->W && c->adj && c->own && c->tets);
    cudaMemsetAsync(c->st, 0, sizeof(DevState), s);
    cudaMemcpyAsync(c->Xi, old->Xi, sizeof(int32_t) * 3 * nv, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->tets, old->tets, sizeof(int32_t) * 4 * nt, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->adj, old->adj, sizeof(int32_t) * 4 * nt, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->own, old->own, sizeof(uint32_t) * nt, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->Ci, old->Ci, sizeof(int32_t) * 3 * ns0, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->W, old->W, sizeof(long long) * ns0, cudaMemcpyDeviceToDevice, s);
    launch_snap(nullptr, 0, d_centers, d_radii, n_new, c->opt.grid_bits, nullptr, c->Ci + 3 * ns0, c->W + ns0, c->st,
                s);
    if (old->used_faces) {
        c->used_faces = c->alloc<uint8_t>(4 * nt);
        NEED(c->used_faces);
        cudaMemcpyAsync(c->used_faces, old->used_faces, 4 * nt, cudaMemcpyDeviceToDevice, s);
    }
    record(c, 1);
    record(c, 2);   // no mesh combinatorics to wait for
    TRY(cuda_check(c, "update launch"));
    return build_rest(c, old);
}

// A1 to A7.  With `old` (a partial update), only the tets whose candidate
// lists changed are clipped; the others' outputs are carried over.
rpd_status build_rest(rpd_ctx* c, rpd_ctx* old) {
    cudaStream_t s = c->stream;
    const long long nv = c->nv, nt = c->nt, ns = c->ns;
    BinStreams* bs = bin_streams();
    // ---- A1
    // one grid (2 ns + 64 cells), or one per shape of a batch (2 n_s + 64
    // cells and an end offset each, laid end to end)
    const bool batch = c->nshapes > 1;
    long long ncap = batch ? 2 * ns + 65ll * c->nshapes : 2 * ns + 64;
    c->gp = c->alloc<GridParams>(c->nshapes);
    c->cell_start = c->alloc<int64_t>(ncap + 1);
    c->cell_ids = c->alloc<int32_t>(ns);
    c->cell_wmax = c->alloc<long long>(2 * ncap);
    void* gtmp = c->alloc<char>(grid_tmp_bytes(ns, ncap));
    c->knn = c->alloc<int32_t>(nv * c->K);
    c->dplus = c->alloc<long long>(nv);
    NEED(c->gp && c->cell_start && c->cell_ids && c->cell_wmax && gtmp && c->knn && c->dplus);
    int4* cell_sph = c->alloc<int4>(ns);
    long long* cell_w = c->alloc<long long>(ns);
    void* ktmp = c->alloc<char>(knn_tmp_bytes(nv));
    NEED(cell_sph && cell_w && ktmp);
    // with debug bit 8 the heaviest spheres stay out of the grid and every
    // vertex scans them first (warp-form neighbour search of one shape only)
    const bool two_word = (c->opt.debug_checks & 4) != 0;
    const bool heavy = !batch && !two_word && ns <= (1 << 17) && (c->opt.debug_checks & 8) && heavy_count(ns) > 0;
    long long* wcut = nullptr;
    int4* hsph = nullptr;
    long long* hw = nullptr;
    int* nheavy = nullptr;
    if (heavy) {
        wcut = c->alloc<long long>(1);
        hsph = c->alloc<int4>(heavy_count(ns));
        hw = c->alloc<long long>(heavy_count(ns));
        nheavy = c->alloc<int>(1);
        NEED(wcut && hsph && hw && nheavy);
        launch_heavy_select(c->Ci, c->W, ns, wcut, hsph, hw, nheavy, s);
    }
    if (batch)
        launch_sphere_grid_batch(c->Ci, c->W, c->d_soff, c->nshapes, ncap, c->gp, c->cell_start, c->cell_ids, cell_sph,
                                 cell_w, c->cell_wmax, c->max_shape_ncap, s);
    else
        launch_sphere_grid(c->Ci, c->W, ns, ncap, c->gp, c->cell_start, c->cell_ids, cell_sph, cell_w, c->cell_wmax,
                           gtmp, s, wcut);
    launch_knn(c->Xi, nv, ns, c->gp, c->cell_start, cell_sph, cell_w, c->cell_wmax, ncap, c->K, c->knn, c->dplus, ktmp,
               &c->st->err, two_word, s, c->d_voff, c->nshapes, hsph, hw, nheavy);
    TRY(cuda_check(c, "knn launch"));
    record(c, 3);
    // ---- A2
    c->cand_cnt = c->alloc<int32_t>(nt);
    c->cand = c->alloc<int32_t>(nt * RPD_MAXC);
    c->cand_ord = c->alloc<uint8_t>(nt * RPD_MAXC);
    c->fb_list = c->alloc<int32_t>(nt);
    c->fb_count = c->alloc<int32_t>(1);
    c->pair_off = c->alloc<int64_t>(nt + 1);
    void* stmp = c->alloc<char>(scan_tmp_bytes(nt + 1));
    c->bin_count = c->alloc<int32_t>(RPD_NBINS);
    c->bin_fill = c->alloc<int32_t>(RPD_NBINS);
    NEED(c->cand_cnt && c->cand && c->cand_ord && c->fb_list && c->fb_count && c->pair_off && stmp && c->bin_count &&
         c->bin_fill);
    launch_candidates(c->tets, nt, nv, c->Xi, c->Ci, c->W, c->knn, c->dplus, c->K, c->gp, c->cell_start,
                      c->cell_ids, c->cell_wmax, c->cand_cnt, c->cand, c->cand_ord, c->fb_list, c->fb_count, c->st, s,
                      c->d_voff, c->nshapes, hsph, hw, nheavy);
    scan_excl(c->cand_cnt, c->pair_off, nt, stmp, s);
    if (old) {   // partial update: clip only the tets whose candidates changed
        c->changed = c->alloc<uint8_t>(nt);
        c->d_nchanged = c->alloc<unsigned long long>(1);
        NEED(c->changed && c->d_nchanged);
        launch_cand_diff(c->cand_cnt, c->cand, c->cand_ord, old->cand_cnt, old->cand, old->cand_ord, nt, c->changed,
                         c->d_nchanged, s);
    }
    launch_bin_count(c->cand_cnt, nt, c->bin_count, s, c->changed);
    TRY(cuda_check(c, "candidate launch"));
    record(c, 4);
    // the pairs are put in bin order before the pair count is read, with room
    // for 4 pairs per tet (binned again below if there are more)
    long long pcap = 4 * nt + 1024;
    if (const char* e = getenv("RPD_PAIR_CAP")) {   // test hook: a small first capacity forces the second binning
        const long long v = atoll(e);
        if (v > 0) pcap = v;
    }
    c->pair_tet = c->alloc<int32_t>(pcap);
    c->bins = c->alloc<int32_t>(pcap);
    c->rcount = c->alloc<unsigned long long>(3);
    c->qcount = c->alloc<unsigned long long>(RPD_NBINS);
    NEED(c->pair_tet && c->bins && c->rcount && c->qcount);
    launch_bin_pairs(c->cand_cnt, c->pair_off, nt, c->pair_tet, c->bins, c->bin_count, c->bin_fill, pcap, c->rcount,
                     c->qcount, s, c->changed);
    cudaStreamWaitEvent(s, c->ev[2], 0);   // mesh combinatorics done
    long long npairs = 0;
    int32_t hb[RPD_NBINS];
    unsigned long long nchanged = (unsigned long long)nt;
    cudaMemcpyAsync(&npairs, c->pair_off + nt, sizeof(long long), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(hb, c->bin_count, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (old) cudaMemcpyAsync(&nchanged, c->d_nchanged, sizeof(nchanged), cudaMemcpyDeviceToHost, s);
    TRY(check_device(c));   // synchronises: validation errors stop the build here
    c->npairs = npairs;
    c->stats.n_pairs = npairs;
    c->stats.update_tets = (int64_t)nchanged;
    for (int b = 0; b < RPD_NBINS; b++) c->stats.bin_pairs[b] = c->hbin[b] = hb[b];
    // ---- A3-A4
    {   // one chunk for the pair, queue, record and finalisation buffers
        size_t est = (size_t)npairs * 760 + ((size_t)ns * 64 + (4 << 20));
        for (int b = 1; b < RPD_NBINS; b++) est += (size_t)c->hbin[b] * (2 * clip_vmax(b) * 4 + 8);
        const long long cap0[3] = {3 * npairs + 1024, 2 * npairs + 1024, npairs / 2 + 1024};
        est += finalize_tmp_bytes(1, npairs, ns);
        for (int k = 0; k < 3; k++) est += finalize_tmp_bytes(k + 2, cap0[k], ns) + (size_t)cap0[k] * 40;
        NEED(c->reserve(est));
    }
    if (npairs > pcap) {
        c->pair_tet = c->alloc<int32_t>(npairs);
        c->bins = c->alloc<int32_t>(npairs);
        NEED(c->pair_tet && c->bins);
        launch_bin_pairs(c->cand_cnt, c->pair_off, nt, c->pair_tet, c->bins, c->bin_count, c->bin_fill, npairs,
                         c->rcount, c->qcount, s, c->changed);
    }
    for (int b = 1; b < RPD_NBINS; b++) {
        long long n = c->hbin[b];
        if (n == 0) continue;
        c->qpair[b] = c->alloc<int32_t>(n);
        c->qnv[b] = c->alloc<uint8_t>(n);
        c->qtrip[b] = c->alloc<uint32_t>(2 * n * clip_vmax(b));
        NEED(c->qpair[b] && c->qnv[b] && c->qtrip[b]);
    }
    ClipArgs& a = c->clip;
    a.tets = c->tets;
    a.Xi = c->Xi;
    a.Ci = c->Ci;
    a.W = c->W;
    a.own = c->own;
    a.adj = c->adj;
    a.cand_cnt = c->cand_cnt;
    a.cand = c->cand;
    a.cand_ord = c->cand_ord;
    a.pair_off = c->pair_off;
    a.pair_tet = c->pair_tet;
    a.unit = ldexp(1.0, -c->opt.grid_bits);
    a.pflag = c->alloc<uint8_t>(npairs);
    a.c_val = c->alloc<int32_t>(npairs);
    a.c_link = c->alloc<uint8_t>(npairs);
    a.p_vol = c->alloc<double>(npairs);
    a.p_mom = c->alloc<double>(3 * npairs);
    a.f_off = c->alloc<int32_t>(npairs);
    a.f_cnt = c->alloc<uint8_t>(npairs);
    a.e_off = c->alloc<int32_t>(npairs);
    a.e_cnt = c->alloc<uint8_t>(npairs);
    a.rcount = c->rcount;
    a.key_bits = c->key_bits;
    a.force_slow = c->opt.debug_checks & 3;
    a.uf_limit = uf_iteration_limit();
    a.st = c->st;
    NEED(a.pflag && a.c_val && a.c_link && a.p_vol && a.p_mom && a.f_off && a.f_cnt && a.e_off && a.e_cnt);
    // finalisation buffers that do not depend on the record counts
    long long* d_nseg = c->alloc<long long>(4);
    c->piece_off = c->alloc<int64_t>(npairs + 1);
    void* ptmp = c->alloc<char>(scan_tmp_bytes(npairs + 1));
    NEED(d_nseg && c->piece_off && ptmp);
    void* ftmp[4] = {nullptr, nullptr, nullptr, nullptr};
    long long fcap[4] = {npairs, 0, 0, 0};
    TRY(finalize_alloc(c, 1, d_nseg, npairs, &ftmp[0]));
    long long cap[3] = {3 * npairs + 1024, 2 * npairs + 1024, npairs / 2 + 1024};
    if (!old) {
        // A face, edge or vertex of the diagram meets a tet in one convex
        // piece, so a tet with n candidates emits at most C(n,2) RPF, C(n,3)
        // RPE and C(n,4) RPV records: per pair of a bin whose tets have at
        // most nb candidates, (nb-1)/2, (nb-1)(nb-2)/6 and (nb-1)(nb-2)(nb-3)/24.
        // The smaller of that and the default sizes the record and table
        // buffers (the records of a partial update also hold kept ones).
        static const int nbmax[RPD_NBINS] = {1, 2, 3, 4, 6, 8, 16, 32};
        double bound[3] = {0, 0, 0};
        for (int b = 0; b < RPD_NBINS; b++) {
            const double n = nbmax[b], p = (double)c->hbin[b];
            bound[0] += p * (n - 1) / 2;
            bound[1] += p * (n - 1) * (n - 2) / 6;
            bound[2] += p * (n - 1) * (n - 2) * (n - 3) / 24;
        }
        for (int k = 0; k < 3; k++) cap[k] = std::min(cap[k], (long long)ceil(bound[k]) + 1024);
    }
    if (const char* e = getenv("RPD_RECORD_CAP")) {   // test hook: small first capacities force a rebuild
        const long long v = atoll(e);
        if (v > 0)
            for (long long& x : cap) x = v;
    }
    void* ktmp2 = nullptr;
    if (old) {
        ktmp2 = c->alloc<char>(keep_tmp_bytes(npairs, old->nrec[2]));
        NEED(ktmp2);
    }
    long long h[5];
    for (int attempt = 0; attempt < 2; attempt++) {
        for (int k = 0; k < 3; k++) {
            a.rcap[k] = cap[k];
            a.rkey[k] = c->alloc<uint64_t>(cap[k]);
            a.rtet[k] = c->alloc<int32_t>(cap[k]);
            a.rval[k] = c->alloc<int16_t>(cap[k]);
            a.rlink[k] = c->alloc<uint8_t>(cap[k]);
            NEED(a.rkey[k] && a.rtet[k] && a.rval[k] && a.rlink[k]);
            if (k == 1 && c->opt.edge_lengths) {
                a.elen = c->alloc<long long>(cap[k]);
                NEED(a.elen);
            }
            fcap[k + 1] = cap[k];
            TRY(finalize_alloc(c, k + 2, d_nseg + k + 1, cap[k], &ftmp[k + 1]));
        }
        if (attempt == 1) join_side_streams(c);   // everything of the first pass is done
        // partial update: the unchanged tets' pair outputs and records, and
        // the record counters set to what was kept (before any clip kernel)
        if (old) launch_keep(old->clip, old->nrec[2], a, npairs, c->changed, old->key_bits, c->key_bits, ktmp2, s);
        // the finalisation scratch is cleared on a high-priority side stream,
        // queued before any clip block can occupy the SMs
        record(c, 11);
        cudaStreamWaitEvent(bs->util, c->ev[11], 0);
        ClearList clr{};
        for (int kind = 1; kind <= 4; kind++)
            if (ftmp[kind - 1]) finalize_clear_list(kind, fcap[kind - 1], c->ns, ftmp[kind - 1], clr);
        launch_clear(clr, bs->util);
        cudaEventRecord(c->ev[12], bs->util);
        TRY(run_clip(c, attempt > 0 && !old, attempt > 0));
        cudaStreamWaitEvent(s, c->ev[12], 0);
        record(c, 5);   // clip and record kernels done, scratch clear: the four kinds fork here
        // ---- A5-A7, the four kinds side by side on high-priority streams; the
        // record counts stay on the device (grids sized by the capacities)
        for (int kind = 1; kind <= 4; kind++) {
            cudaStream_t sk = bs->fin[kind - 1];
            cudaStreamWaitEvent(sk, c->ev[5], 0);
            if (c->kind_ok[kind - 1]) {
                launch_finalize(c->clip, kind, fcap[kind - 1], fcap[kind - 1], c->ns, c->key_bits,
                                c->fout[kind - 1], ftmp[kind - 1], sk);
            } else {
                cudaMemsetAsync(d_nseg + kind - 1, 0, sizeof(long long), sk);
            }
            cudaEventRecord(c->ev[6 + kind - 1], sk);
        }
        scan_excl(a.pflag, c->piece_off, npairs, ptmp, s);
        TRY(cuda_check(c, "finalize launch"));
        for (int kind = 1; kind <= 4; kind++) cudaStreamWaitEvent(s, c->ev[6 + kind - 1], 0);
        for (int b = 0; b < RPD_NBINS; b++)   // volume passes
            if (c->hbin[b]) cudaStreamWaitEvent(s, c->evc[1 + RPD_NBINS + b], 0);
        unsigned long long cnt[3], qc[RPD_NBINS];
        cudaMemcpyAsync(cnt, c->rcount, sizeof(cnt), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(qc, c->qcount, sizeof(qc), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(h, d_nseg, sizeof(long long) * 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(h + 4, c->piece_off + npairs, sizeof(long long), cudaMemcpyDeviceToHost, s);
        int dev_err = 0;
        TRY(check_device(c, false, &dev_err));
        for (int b = 0; b < RPD_NBINS; b++) c->stats.bin_cut[b] = (int64_t)qc[b];
        bool fits = true;
        for (int k = 0; k < 3; k++) {
            c->nrec[k] = (long long)cnt[k];
            if ((long long)cnt[k] > cap[k]) {   // records were dropped: rebuild from the clip
                fits = false;
                cap[k] = (long long)cnt[k] + 1024;
            }
        }
        if (fits) {
            if (dev_err) TRY(check_device(c));   // raises what the device reported
            break;
        }
        if (attempt == 1) return fail(c, RPD_E_OVERFLOW, "record buffers overflowed twice");
        // the finalisation ran on truncated records: its status is void; keep
        // the counters of the stages before the clip and start over
        const unsigned long long fb = (unsigned long long)c->stats.cand_fallback;
        cudaMemsetAsync(c->st, 0, sizeof(DevState), s);
        cudaMemcpyAsync(&c->st->cnt[CNT_CAND_FALLBACK], &fb, sizeof(fb), cudaMemcpyHostToDevice, s);
        TRY(check_device(c));
    }
    for (int k = 0; k < 3; k++) c->stats.n_records[k + 1] = c->nrec[k];
    for (int k = 0; k < 4; k++) {
        c->nkeys[k] = h[k];
        c->stats.n_keys[k] = h[k];
    }
    c->npieces = h[4];
    c->stats.n_pieces = h[4];
    c->stats.n_records[0] = h[4];
    for (int k = 0; k < 4; k++) {
        c->ftmp[k] = ftmp[k];
        c->fcap[k] = fcap[k];
    }
    c->timed = false;   // stage times are read from the events when the stats are asked for
    return RPD_OK;
}

// Stage times of the build from its events (all complete once it returned).
void stage_times(rpd_ctx* c) {
    if (c->timed) return;
    c->stats.ms_prep = elapsed(c, 0, 2);   // snapping + mesh combinatorics (beside the kNN)
    c->stats.ms_knn = elapsed(c, 1, 3);
    c->stats.ms_cand = elapsed(c, 3, 4);
    c->stats.ms_clip = elapsed(c, 4, 5);
    for (int b = 0; b < RPD_NBINS; b++) {
        if (c->hbin[b] == 0) continue;
        float k = 0, w = 0;
        if (cudaEventElapsedTime(&k, c->evc[0], c->evc[1 + b]) != cudaSuccess ||
            cudaEventElapsedTime(&w, c->evc[0], c->evc[1 + RPD_NBINS + b]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        c->stats.ms_clip_kernels = std::max(c->stats.ms_clip_kernels, k);
        c->stats.ms_clip_span = std::max(c->stats.ms_clip_span, w);
    }
    for (int k = 0; k < 4; k++) c->stats.ms_finalize[k] = elapsed(c, 5, 6 + k);   // the kinds run side by side
    c->timed = true;
}

rpd_status check_kind(rpd_ctx* c, int kind) {
    if (!c) return RPD_E_INVALID;
    if (kind < 1 || kind > 4) return fail(c, RPD_E_INVALID, "kind must be 1..4");
    if (!c->kind_ok[kind - 1]) return fail(c, RPD_E_OVERFLOW, "RPV keys need at most 2^16 - 1 spheres");
    return RPD_OK;
}

}  // namespace

extern "C" {

void rpd_default_options(rpd_options* opt) {
    if (!opt) return;
    opt->precision = RPD_FP32_FILTERED;
    opt->k = 16;
    opt->grid_bits = 20;
    opt->debug_checks = 0;
    opt->edge_lengths = 0;
}

rpd_status rpd_build(const double* d_verts, int64_t nv, const int32_t* d_tets, int64_t nt, const double* d_centers,
                     const double* d_radii, int64_t ns, const rpd_options* opt, void* cuda_stream, rpd_ctx** out) {
    if (!out) return RPD_E_INVALID;
    *out = nullptr;
    rpd_options o;
    rpd_default_options(&o);
    if (opt) o = *opt;
    auto reject = [](const char* m) {
        g_build_error = m;
        return RPD_E_INVALID;
    };
    if (nv < 4 || nv >= (1ll << 21)) return reject("nv must be in [4, 2^21)");
    if (nt < 1 || nt >= (1ll << 31) / RPD_MAXC) return reject("nt must be in [1, 2^26)");
    if (ns < 1 || ns >= (1ll << 21)) return reject("ns must be in [1, 2^21)");
    if (!d_verts || !d_tets || !d_centers || !d_radii) return reject("null input pointer");
    if (o.k < 1 || o.k > RPD_MAXK) return reject("k must be in [1, 32]");
    if (o.grid_bits < 0 || o.grid_bits > 40) return reject("grid_bits must be in [0, 40]");
    if (o.precision != RPD_FP64 && o.precision != RPD_FP32_FILTERED) return reject("unknown precision");
    rpd_ctx* c = new rpd_ctx();
    c->stream = (cudaStream_t)cuda_stream;
    c->opt = o;
    c->nv = nv;
    c->nt = nt;
    c->ns = ns;
    c->K = o.k;
    c->key_bits = bits_for(ns);
    rpd_status st = build(c, d_verts, d_tets, d_centers, d_radii);
    if (st != RPD_OK) {
        g_build_error = c->last_error.empty() ? "build failed" : c->last_error;
        rpd_destroy(c);
        return st;
    }
    g_build_error.clear();
    *out = c;
    return RPD_OK;
}

rpd_status rpd_build_batch(const double* d_verts, const int32_t* d_tets, const double* d_centers,
                           const double* d_radii, int32_t nshapes, const int64_t* h_vert_off,
                           const int64_t* h_tet_off, const int64_t* h_sphere_off, const rpd_options* opt,
                           void* cuda_stream, rpd_ctx** out) {
    if (!out) return RPD_E_INVALID;
    *out = nullptr;
    auto reject = [](const char* m) {
        g_build_error = m;
        return RPD_E_INVALID;
    };
    if (nshapes < 1 || nshapes > (1 << 20)) return reject("nshapes must be in [1, 2^20]");
    if (!h_vert_off || !h_tet_off || !h_sphere_off) return reject("null offset array");
    if (h_vert_off[0] != 0 || h_tet_off[0] != 0 || h_sphere_off[0] != 0) return reject("offsets must start at 0");
    long long max_ncap = 0;
    for (int s = 0; s < nshapes; s++) {
        const long long nv_s = h_vert_off[s + 1] - h_vert_off[s], nt_s = h_tet_off[s + 1] - h_tet_off[s],
                        ns_s = h_sphere_off[s + 1] - h_sphere_off[s];
        if (nv_s < 4 || nt_s < 1 || ns_s < 1) return reject("every shape needs >= 4 vertices, a tet and a sphere");
        max_ncap = std::max(max_ncap, 2 * ns_s + 64);
    }
    if (max_ncap > batch_grid_cap()) return reject("a shape of a batch has more spheres than its grid takes");
    const long long nv = h_vert_off[nshapes], nt = h_tet_off[nshapes], ns = h_sphere_off[nshapes];
    if (ns >= (1ll << 21)) return reject("a batch holds fewer than 2^21 spheres");
    rpd_options o;
    rpd_default_options(&o);
    if (opt) o = *opt;
    if (o.debug_checks & 4) return reject("the tiled neighbour search does not take batches");
    if (nshapes == 1) return rpd_build(d_verts, nv, d_tets, nt, d_centers, d_radii, ns, &o, cuda_stream, out);
    if (nv >= (1ll << 21)) return reject("nv must be < 2^21");
    if (nt >= (1ll << 31) / RPD_MAXC) return reject("nt must be < 2^26");
    if (!d_verts || !d_tets || !d_centers || !d_radii) return reject("null input pointer");
    if (o.k < 1 || o.k > RPD_MAXK) return reject("k must be in [1, 32]");
    if (o.grid_bits < 0 || o.grid_bits > 40) return reject("grid_bits must be in [0, 40]");
    if (o.precision != RPD_FP64 && o.precision != RPD_FP32_FILTERED) return reject("unknown precision");
    rpd_ctx* c = new rpd_ctx();
    c->stream = (cudaStream_t)cuda_stream;
    c->opt = o;
    c->nv = nv;
    c->nt = nt;
    c->ns = ns;
    c->K = o.k;
    c->key_bits = bits_for(ns);
    c->nshapes = nshapes;
    c->h_voff.assign(h_vert_off, h_vert_off + nshapes + 1);
    c->h_toff.assign(h_tet_off, h_tet_off + nshapes + 1);
    c->h_soff.assign(h_sphere_off, h_sphere_off + nshapes + 1);
    c->max_shape_ncap = max_ncap;
    rpd_status st = build(c, d_verts, d_tets, d_centers, d_radii);
    if (st != RPD_OK) {
        g_build_error = c->last_error.empty() ? "build failed" : c->last_error;
        rpd_destroy(c);
        return st;
    }
    g_build_error.clear();
    *out = c;
    return RPD_OK;
}

}  // extern "C"

// Time `build` (which makes and returns a context) for each k of ks, reps
// times after one warm-up, with CUDA events on the stream; keep the fastest
// median.  Every k gives the same diagram (the candidate sets are exact), so
// only the time decides.
template <typename Build>
static rpd_status autotune(const rpd_options* base, const int32_t* ks, int32_t nk, int32_t reps, void* cuda_stream,
                           Build build, rpd_options* best, float* ms_best) {
    if (!ks || nk < 1 || nk > 32 || reps < 1 || reps > 64 || !best) return RPD_E_INVALID;
    rpd_options o;
    rpd_default_options(&o);
    if (base) o = *base;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return RPD_E_CUDA;
    }
    float best_ms = INFINITY;
    int best_k = -1;
    rpd_status err = RPD_OK;
    for (int q = 0; q < nk && err == RPD_OK; q++) {
        o.k = ks[q];
        std::vector<float> t;
        for (int r = 0; r <= reps && err == RPD_OK; r++) {
            rpd_ctx* c = nullptr;
            cudaEventRecord(e0, s);
            err = build(&o, &c);
            cudaEventRecord(e1, s);
            float ms = 0;
            if (err == RPD_OK &&
                (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)) {
                cudaGetLastError();
                err = RPD_E_CUDA;
            }
            if (c) rpd_destroy(c);
            if (r > 0) t.push_back(ms);   // the first build of each k warms up
        }
        if (err != RPD_OK) break;
        std::sort(t.begin(), t.end());
        const float med = t[t.size() / 2];
        if (med < best_ms) {
            best_ms = med;
            best_k = ks[q];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != RPD_OK) return err;
    o.k = best_k;
    *best = o;
    if (ms_best) *ms_best = best_ms;
    return RPD_OK;
}

extern "C" {

rpd_status rpd_autotune(const double* d_verts, int64_t nv, const int32_t* d_tets, int64_t nt, const double* d_centers,
                        const double* d_radii, int64_t ns, const rpd_options* base, const int32_t* ks, int32_t nk,
                        int32_t reps, void* cuda_stream, rpd_options* best, float* ms_best) {
    return autotune(base, ks, nk, reps, cuda_stream,
                    [&](const rpd_options* o, rpd_ctx** c) {
                        return rpd_build(d_verts, nv, d_tets, nt, d_centers, d_radii, ns, o, cuda_stream, c);
                    },
                    best, ms_best);
}

rpd_status rpd_autotune_batch(const double* d_verts, const int32_t* d_tets, const double* d_centers,
                              const double* d_radii, int32_t nshapes, const int64_t* h_vert_off,
                              const int64_t* h_tet_off, const int64_t* h_sphere_off, const rpd_options* base,
                              const int32_t* ks, int32_t nk, int32_t reps, void* cuda_stream, rpd_options* best,
                              float* ms_best) {
    return autotune(base, ks, nk, reps, cuda_stream,
                    [&](const rpd_options* o, rpd_ctx** c) {
                        return rpd_build_batch(d_verts, d_tets, d_centers, d_radii, nshapes, h_vert_off, h_tet_off,
                                               h_sphere_off, o, cuda_stream, c);
                    },
                    best, ms_best);
}

rpd_status rpd_batch_offsets(rpd_ctx* ctx, int32_t kind, int64_t* h_off) {
    if (!ctx) return RPD_E_INVALID;
    if (!h_off) return fail(ctx, RPD_E_INVALID, "null output");
    const int S = ctx->nshapes;
    if (S == 1) {
        h_off[0] = 0;
        if (kind == 0) h_off[1] = ctx->npieces;
        else {
            TRY(check_kind(ctx, (rpd_kind)kind));
            h_off[1] = ctx->nkeys[kind - 1];
        }
        return RPD_OK;
    }
    long long* d = ctx->alloc<long long>(S + 1);
    if (!d) return fail(ctx, RPD_E_OOM, "device allocation failed");
    if (kind == 0) {
        launch_batch_cut_pieces(ctx->pair_off, ctx->piece_off, ctx->d_toff, S, d, ctx->stream);
    } else {
        TRY(check_kind(ctx, (rpd_kind)kind));
        launch_batch_cut(ctx->fout[kind - 1].keys, ctx->nkeys[kind - 1], kind, ctx->d_soff, S, d, ctx->stream);
    }
    cudaMemcpyAsync(h_off, d, sizeof(long long) * (S + 1), cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RPD_E_CUDA, "CUDA error while cutting the tables by shape");
    }
    return RPD_OK;
}

rpd_status rpd_insert(rpd_ctx* ctx, const double* d_centers, const double* d_radii, int64_t n_new) {
    if (!ctx) return RPD_E_INVALID;
    if (ctx->nshapes > 1) return fail(ctx, RPD_E_INVALID, "a batch context takes no insertions");
    if (n_new < 0 || ctx->ns + n_new >= (1ll << 21))
        return fail(ctx, RPD_E_INVALID, "n_new must be >= 0 and ns + n_new < 2^21");
    if (n_new == 0) return RPD_OK;
    if (!d_centers || !d_radii) return fail(ctx, RPD_E_INVALID, "null input pointer");
    rpd_ctx* c = new rpd_ctx();
    c->stream = ctx->stream;
    c->opt = ctx->opt;
    c->nv = ctx->nv;
    c->nt = ctx->nt;
    c->ns = ctx->ns + n_new;
    c->K = ctx->K;
    c->key_bits = bits_for(c->ns);
    rpd_status st = update(c, ctx, d_centers, d_radii, n_new);
    if (st != RPD_OK) {
        ctx->last_error = c->last_error.empty() ? "update failed" : c->last_error;
        rpd_destroy(c);
        return st;
    }
    // settings and counters that outlive a diagram (the mesh is unchanged)
    c->proposer = ctx->proposer;
    c->proposer_margin = ctx->proposer_margin;
    c->shrink_pins = ctx->shrink_pins;
    c->shrink_iters = ctx->shrink_iters;
    c->shrink_restarts = ctx->shrink_restarts;
    c->have_bbox = ctx->have_bbox;
    for (int a = 0; a < 3; a++) {
        c->bb_lo[a] = ctx->bb_lo[a];
        c->bb_hi[a] = ctx->bb_hi[a];
    }
    // the context takes the new diagram; the old one's memory goes with c
    std::swap(*ctx, *c);
    rpd_destroy(c);
    ctx->last_error.clear();
    return RPD_OK;
}

rpd_status rpd_pins(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, double* d_pins, double* d_normals, int32_t* d_faces,
                    int64_t cap, int64_t* n) {
    if (!ctx) return RPD_E_INVALID;
    if (kind < 1 || kind > 3) return fail(ctx, RPD_E_INVALID, "pins are defined for cells, faces and edges (kind 1..3)");
    TRY(check_kind(ctx, kind));
    cudaStream_t s = ctx->stream;
    const long long nk = ctx->nkeys[kind - 1];
    const FinalOut& o = ctx->fout[kind - 1];
    void* tmp = ctx->alloc<char>(pins_tmp_bytes(nk));
    if (!tmp) return fail(ctx, RPD_E_OOM, "device allocation failed");
    launch_pins_count(o.flag, nk, tmp, s);
    long long nfail = 0;
    cudaMemcpyAsync(&nfail, pins_fpos(tmp, nk) + nk, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RPD_E_CUDA, "CUDA error while counting failing elements");
    }
    if (n) *n = nfail;
    if (!d_keys && !d_pins && !d_normals && !d_faces) return RPD_OK;
    if (!d_keys || !d_pins || !d_normals || !d_faces) return fail(ctx, RPD_E_INVALID, "all four outputs are needed");
    if (cap < nfail) return fail(ctx, RPD_E_INVALID, "cap is smaller than the number of failing elements");
    const int32_t* parent = (const int32_t*)ctx->ftmp[kind - 1];
    const long long nmax = kind == 1 ? ctx->npairs : ctx->fcap[kind - 1];
    launch_pins(ctx->clip, kind, o.keys, o.beta, o.chi, o.flag, nk, nfail, parent, nmax, ctx->clip.uf_limit,
                ctx->used_faces, tmp, d_keys, d_pins, d_normals, d_faces, s);
    return cuda_check(ctx, "pin launch");
}

// Boundary triangles of the context's mesh, built on first use.
static rpd_status ensure_boundary(rpd_ctx* c, double** tri, int32_t** face_of) {
    static_assert(sizeof(long long) == sizeof(int64_t), "int64");
    if (c->nbtri < 0) {
        cudaStream_t s = c->stream;
        int64_t* pos = c->alloc<int64_t>(4 * c->nt + 1);
        void* tmp = c->alloc<char>(boundary_tmp_bytes(c->nt));
        if (!pos || !tmp) return fail(c, RPD_E_OOM, "device allocation failed");
        launch_boundary_count(c->adj, c->nt, pos, tmp, s);
        long long nb = 0;
        cudaMemcpyAsync(&nb, pos + 4 * c->nt, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, RPD_E_CUDA, "CUDA error while counting boundary triangles");
        }
        double* t = c->alloc<double>(9 * nb + 9);
        int32_t* f = c->alloc<int32_t>(nb + 1);
        float4* b = c->alloc<float4>(nb + 1);
        if (!t || !f || !b) return fail(c, RPD_E_OOM, "device allocation failed");
        launch_boundary_fill(c->tets, c->adj, c->Xi, c->nt, pos, ldexp(1.0, -c->opt.grid_bits), t, f, s);
        launch_boundary_spheres(t, nb, b, s);
        TRY(cuda_check(c, "boundary launch"));
        c->btri = t;
        c->btri_face = f;
        c->btri_ball = b;
        c->nbtri = nb;
    }
    *tri = c->btri;
    *face_of = c->btri_face;
    return RPD_OK;
}

rpd_status rpd_shrink(rpd_ctx* ctx, const double* d_pins, const double* d_normals, const int32_t* d_faces, int64_t n,
                      double* d_centers, double* d_radii, int32_t* d_iters) {
    if (!ctx) return RPD_E_INVALID;
    if (n < 0) return fail(ctx, RPD_E_INVALID, "n must be >= 0");
    if (n == 0) return RPD_OK;
    if (!d_pins || !d_normals || !d_faces || !d_centers || !d_radii || !d_iters)
        return fail(ctx, RPD_E_INVALID, "null pointer");
    if (n >= (1ll << 31)) return fail(ctx, RPD_E_INVALID, "n must be < 2^31");
    double* tri = nullptr;
    int32_t* face_of = nullptr;
    TRY(ensure_boundary(ctx, &tri, &face_of));
    // a first radius above twice any diameter the grid allows
    const double r0 = ldexp(1.0, 23 - ctx->opt.grid_bits);
    launch_shrink(tri, ctx->btri_ball, ctx->nbtri, face_of, d_pins, d_normals, d_faces, n, r0, nullptr, d_centers,
                  d_radii, d_iters, nullptr, ctx->stream);
    return cuda_check(ctx, "shrink launch");
}

rpd_status rpd_shrink_warm(rpd_ctx* ctx, const double* d_pins, const double* d_normals, const int32_t* d_faces,
                           int64_t n, const double* d_r_start, double* d_centers, double* d_radii, int32_t* d_iters,
                           int32_t* d_restarted) {
    if (!ctx) return RPD_E_INVALID;
    if (n < 0) return fail(ctx, RPD_E_INVALID, "n must be >= 0");
    if (n == 0) return RPD_OK;
    if (!d_pins || !d_normals || !d_faces || !d_r_start || !d_centers || !d_radii || !d_iters)
        return fail(ctx, RPD_E_INVALID, "null pointer");
    if (n >= (1ll << 31)) return fail(ctx, RPD_E_INVALID, "n must be < 2^31");
    double* tri = nullptr;
    int32_t* face_of = nullptr;
    TRY(ensure_boundary(ctx, &tri, &face_of));
    const double r0 = ldexp(1.0, 23 - ctx->opt.grid_bits);
    launch_shrink(tri, ctx->btri_ball, ctx->nbtri, face_of, d_pins, d_normals, d_faces, n, r0, d_r_start, d_centers,
                  d_radii, d_iters, d_restarted, ctx->stream);
    return cuda_check(ctx, "shrink launch");
}

// Mesh bounding box from the grid vertices, on first use.
static rpd_status ensure_bbox(rpd_ctx* c) {
    if (c->have_bbox) return RPD_OK;
    int* b = c->alloc<int>(6);
    if (!b) return fail(c, RPD_E_OOM, "device allocation failed");
    launch_bbox(c->Xi, c->nv, b, c->stream);
    int h[6];
    cudaMemcpyAsync(h, b, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, RPD_E_CUDA, "CUDA error while measuring the mesh");
    }
    const double unit = ldexp(1.0, -c->opt.grid_bits);
    for (int a = 0; a < 3; a++) {
        c->bb_lo[a] = h[a] * unit;
        c->bb_hi[a] = h[3 + a] * unit;
    }
    c->have_bbox = true;
    return RPD_OK;
}

static void bbox_frame(const rpd_ctx* c, double* bc, double* bh, double* diag) {
    double d2 = 0, half = 0;
    for (int a = 0; a < 3; a++) {
        const double e = c->bb_hi[a] - c->bb_lo[a];
        bc[a] = 0.5 * (c->bb_hi[a] + c->bb_lo[a]);
        half = std::max(half, 0.5 * e);
        d2 += e * e;
    }
    *bh = half > 0 ? half : 1.0;
    *diag = d2 > 0 ? sqrt(d2) : 1.0;
}

rpd_status rpd_pin_features(rpd_ctx* ctx, const double* d_pins, const double* d_normals, const double* d_radii,
                            int64_t n, float* d_x, float* d_t) {
    if (!ctx) return RPD_E_INVALID;
    if (n < 0) return fail(ctx, RPD_E_INVALID, "n must be >= 0");
    if (n == 0) return RPD_OK;
    if (!d_pins || !d_normals || !d_x || (d_radii && !d_t)) return fail(ctx, RPD_E_INVALID, "null pointer");
    TRY(ensure_bbox(ctx));
    double bc[3], bh, diag;
    bbox_frame(ctx, bc, &bh, &diag);
    launch_pin_features(d_pins, d_normals, d_radii, n, bc, bh, diag, d_x, d_t, ctx->stream);
    return cuda_check(ctx, "feature launch");
}

rpd_status rpd_propose(rpd_ctx* ctx, rpd_mlp* mlp, const double* d_pins, const double* d_normals, int64_t n,
                       double margin, double* d_r_start) {
    if (!ctx) return RPD_E_INVALID;
    if (!mlp || n < 0 || !(margin >= 1.0)) return fail(ctx, RPD_E_INVALID, "a network, n >= 0 and margin >= 1");
    if (n == 0) return RPD_OK;
    if (!d_pins || !d_normals || !d_r_start) return fail(ctx, RPD_E_INVALID, "null pointer");
    float* x = ctx->alloc<float>(n * RPD_PIN_FEATURES);
    float* y = ctx->alloc<float>(n);
    if (!x || !y) return fail(ctx, RPD_E_OOM, "device allocation failed");
    TRY(rpd_pin_features(ctx, d_pins, d_normals, nullptr, n, x, nullptr));
    // the network runs on its own stream: let the features land first
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RPD_E_CUDA, "CUDA error in the feature kernel");
    }
    const rpd_status s = rpd_mlp_forward(mlp, x, n, y);
    if (s != RPD_OK) return fail(ctx, s, "proposer network failed");
    double bc[3], bh, diag;
    bbox_frame(ctx, bc, &bh, &diag);
    launch_radius_start(y, n, diag, margin, d_r_start, ctx->stream);
    return cuda_check(ctx, "proposal launch");
}

rpd_status rpd_set_proposer(rpd_ctx* ctx, rpd_mlp* mlp, double margin) {
    if (!ctx) return RPD_E_INVALID;
    if (!(margin >= 1.0)) return fail(ctx, RPD_E_INVALID, "margin must be >= 1");
    ctx->proposer = mlp;
    ctx->proposer_margin = margin;
    return RPD_OK;
}

rpd_status rpd_shrink_counters(rpd_ctx* ctx, int64_t* pins, int64_t* iters, int64_t* restarts) {
    if (!ctx) return RPD_E_INVALID;
    if (pins) *pins = ctx->shrink_pins;
    if (iters) *iters = ctx->shrink_iters;
    if (restarts) *restarts = ctx->shrink_restarts;
    return RPD_OK;
}

// Per-key RPE lengths, summed from the records on first use (the volume pass
// that measures the segments runs beside the finalisation, so the sums are
// taken once the build has joined its streams).
static rpd_status ensure_edge_lengths(rpd_ctx* c) {
    if (c->edge_len) return RPD_OK;
    if (!c->clip.elen)
        return fail(c, RPD_E_INVALID, "edge lengths need a context built with rpd_options.edge_lengths = 1");
    long long* len = c->alloc<long long>(c->nkeys[2] + 1);
    if (!len) return fail(c, RPD_E_OOM, "device allocation failed");
    launch_edge_length_sum(c->clip, c->fcap[2], c->fout[2].keys, c->nkeys[2], len, c->stream);
    TRY(cuda_check(c, "edge length launch"));
    c->edge_len = len;
    return RPD_OK;
}

rpd_status rpd_edge_lengths(rpd_ctx* ctx, int32_t* d_keys, double* d_len, int64_t cap, int64_t* n) {
    if (!ctx) return RPD_E_INVALID;
    TRY(check_kind(ctx, 3));
    const long long m = ctx->nkeys[2];
    if (n) *n = m;
    if (!d_keys && !d_len) return RPD_OK;
    if (cap < m) return fail(ctx, RPD_E_INVALID, "cap is smaller than the number of elements");
    if (m == 0) return RPD_OK;
    const FinalOut& o = ctx->fout[2];
    if (d_keys) launch_copy_rows(o.keys, d_keys, 3 * m, nullptr, nullptr, 0, 4, ctx->stream);
    if (d_len) {
        TRY(ensure_edge_lengths(ctx));
        launch_fixed_to_world(ctx->edge_len, d_len, m, ldexp(1.0, -24 - ctx->opt.grid_bits), ctx->stream);
    }
    return cuda_check(ctx, "edge length launch");
}

rpd_status rpd_medial(rpd_ctx* ctx, double sigma, rpd_medial_info* info, int32_t* h_edges, int64_t cap_e,
                      int32_t* h_faces, int64_t cap_f) {
    if (!ctx || !info) return RPD_E_INVALID;
    if (!(sigma >= 0)) return fail(ctx, RPD_E_INVALID, "sigma must be >= 0");
    cudaStream_t s = ctx->stream;
    const long long nv = ctx->nkeys[0], ne = ctx->nkeys[1], nf = ctx->nkeys[2];
    const long long nt4 = ctx->kind_ok[3] ? ctx->nkeys[3] : 0;
    std::vector<int32_t> v(nv), e(2 * ne), f(3 * nf), t(4 * nt4);
    std::vector<long long> len(nf), w(ctx->ns);
    if (nv) cudaMemcpyAsync(v.data(), ctx->fout[0].keys, 4 * nv, cudaMemcpyDeviceToHost, s);
    if (ne) cudaMemcpyAsync(e.data(), ctx->fout[1].keys, 8 * ne, cudaMemcpyDeviceToHost, s);
    if (nf) {
        TRY(ensure_edge_lengths(ctx));
        cudaMemcpyAsync(f.data(), ctx->fout[2].keys, 12 * nf, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(len.data(), ctx->edge_len, 8 * nf, cudaMemcpyDeviceToHost, s);
    }
    if (nt4) cudaMemcpyAsync(t.data(), ctx->fout[3].keys, 16 * nt4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(w.data(), ctx->W, sizeof(long long) * ctx->ns, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RPD_E_CUDA, "CUDA error while reading the element tables");
    }
    // importance alpha = |RPE| / mean of the three diameters (both in grid units)
    std::vector<double> alpha(nf);
    for (long long q = 0; q < nf; q++) {
        double r = 0;
        for (int z = 0; z < 3; z++) r += sqrt((double)w[f[3 * q + z]]);
        const double mean_diam = 2.0 * r / 3.0;
        const double l = ldexp((double)len[q], -24);
        alpha[q] = mean_diam > 0 ? l / mean_diam : INFINITY;
    }
    std::vector<uint8_t> ea, fa, ta;
    medial_thin(e, f, alpha, t, sigma, ea, fa, ta);
    long long ne2 = 0, nf2 = 0, nt2 = 0;
    for (uint8_t x : ea) ne2 += x;
    for (uint8_t x : fa) nf2 += x;
    for (uint8_t x : ta) nt2 += x;
    info->vertices = nv;
    info->edges = ne;
    info->faces = nf;
    info->tets = nt4;
    info->edges_thin = ne2;
    info->faces_thin = nf2;
    info->tets_thin = nt2;
    info->chi = nv - ne + nf - nt4;
    info->chi_thin = nv - ne2 + nf2 - nt2;
    if (h_edges) {
        if (cap_e < ne2) return fail(ctx, RPD_E_INVALID, "cap_e is smaller than the thinned edge count");
        long long o = 0;
        for (long long q = 0; q < ne; q++)
            if (ea[q]) {
                h_edges[2 * o] = e[2 * q];
                h_edges[2 * o + 1] = e[2 * q + 1];
                o++;
            }
    }
    if (h_faces) {
        if (cap_f < nf2) return fail(ctx, RPD_E_INVALID, "cap_f is smaller than the thinned triangle count");
        long long o = 0;
        for (long long q = 0; q < nf; q++)
            if (fa[q]) {
                for (int z = 0; z < 3; z++) h_faces[3 * o + z] = f[3 * q + z];
                o++;
            }
    }
    return RPD_OK;
}

rpd_status rpd_spheres(rpd_ctx* ctx, double* d_centers, double* d_radii, int64_t cap, int64_t* n) {
    if (!ctx) return RPD_E_INVALID;
    if (n) *n = ctx->ns;
    if (!d_centers && !d_radii) return RPD_OK;
    if (!d_centers || !d_radii || cap < ctx->ns) return fail(ctx, RPD_E_INVALID, "both outputs and cap >= ns are needed");
    launch_sphere_out(ctx->Ci, ctx->W, ctx->ns, ldexp(1.0, -ctx->opt.grid_bits), d_centers, d_radii, ctx->stream);
    return cuda_check(ctx, "sphere output launch");
}

// Grow spheres from pins (host arrays: points, inward normals, boundary face
// ids): one per boundary triangle not -1, shrunk on the device, rounded to
// the grid, repeats of existing or of each other dropped, then inserted with a
// partial update.  *inserted = the number inserted (0: nothing new).
static rpd_status grow_from_pins(rpd_ctx* ctx, const std::vector<double>& hp, const std::vector<double>& hn,
                                 const std::vector<int32_t>& hf, long long* inserted, long long* tried = nullptr) {
    *inserted = 0;
    if (tried) *tried = 0;
    const double unit = ldexp(1.0, -ctx->opt.grid_bits), scale = ldexp(1.0, ctx->opt.grid_bits);
    // one pin per boundary triangle
    std::vector<int> keep;
    {
        std::vector<int32_t> seen;
        for (size_t q = 0; q < hf.size(); q++) {
            if (hf[q] < 0) continue;
            if (std::find(seen.begin(), seen.end(), hf[q]) != seen.end()) continue;
            seen.push_back(hf[q]);
            keep.push_back((int)q);
        }
    }
    if (keep.empty()) return RPD_OK;   // no boundary point to grow from
    const long long m = (long long)keep.size();
    if (tried) *tried = m;
    std::vector<double> kp(3 * m), kn(3 * m);
    std::vector<int32_t> kf(m);
    for (long long q = 0; q < m; q++) {
        for (int z = 0; z < 3; z++) {
            kp[3 * q + z] = hp[3 * keep[q] + z];
            kn[3 * q + z] = hn[3 * keep[q] + z];
        }
        kf[q] = hf[keep[q]];
    }
    double* dp = ctx->alloc<double>(3 * m);
    double* dn = ctx->alloc<double>(3 * m);
    int32_t* df = ctx->alloc<int32_t>(m);
    double* dc = ctx->alloc<double>(3 * m);
    double* dr = ctx->alloc<double>(m);
    int32_t* di = ctx->alloc<int32_t>(m);
    if (!dp || !dn || !df || !dc || !dr || !di) return fail(ctx, RPD_E_OOM, "device allocation failed");
    cudaMemcpyAsync(dp, kp.data(), sizeof(double) * 3 * m, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(dn, kn.data(), sizeof(double) * 3 * m, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(df, kf.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, ctx->stream);
    int32_t* drs = ctx->alloc<int32_t>(m);
    if (!drs) return fail(ctx, RPD_E_OOM, "device allocation failed");
    if (ctx->proposer) {
        // the network proposes where the shrinking starts; the shrinking
        // still decides the sphere
        double* rs = ctx->alloc<double>(m);
        if (!rs) return fail(ctx, RPD_E_OOM, "device allocation failed");
        TRY(rpd_propose(ctx, ctx->proposer, dp, dn, m, ctx->proposer_margin, rs));
        TRY(rpd_shrink_warm(ctx, dp, dn, df, m, rs, dc, dr, di, drs));
    } else {
        TRY(rpd_shrink(ctx, dp, dn, df, m, dc, dr, di));
        cudaMemsetAsync(drs, 0, sizeof(int32_t) * m, ctx->stream);
    }
    if (!ctx->used_faces) {
        ctx->used_faces = ctx->alloc<uint8_t>(4 * ctx->nt);
        if (!ctx->used_faces) return fail(ctx, RPD_E_OOM, "device allocation failed");
        cudaMemsetAsync(ctx->used_faces, 0, 4 * ctx->nt, ctx->stream);
    }
    launch_mark_faces(df, m, ctx->used_faces, 4 * ctx->nt, ctx->stream);
    std::vector<double> hc(3 * m), hr(m);
    std::vector<int32_t> hit(m), hrs(m);
    std::vector<int32_t> ci(3 * ctx->ns);
    std::vector<long long> cw(ctx->ns);
    cudaMemcpyAsync(hc.data(), dc, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(hr.data(), dr, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(hit.data(), di, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(hrs.data(), drs, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(ci.data(), ctx->Ci, sizeof(int32_t) * 3 * ctx->ns, cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(cw.data(), ctx->W, sizeof(long long) * ctx->ns, cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RPD_E_CUDA, "CUDA error while reading shrunk spheres");
    }
    for (long long q = 0; q < m; q++) {
        ctx->shrink_pins++;
        ctx->shrink_iters += hit[q];
        ctx->shrink_restarts += hrs[q];
    }
    // new spheres on the grid, without repeats of each other or of the
    // existing spheres (a repeat would have a radical plane with no normal)
    std::vector<unsigned long long> have;   // hashed snapped centres + weights seen
    auto pack = [](long long x, long long y, long long z, long long w) {
        unsigned long long h = 1469598103934665603ull;
        for (unsigned long long v : {(unsigned long long)x, (unsigned long long)y, (unsigned long long)z,
                                     (unsigned long long)w})
            h = (h ^ v) * 1099511628211ull;
        return h;
    };
    for (long long q = 0; q < ctx->ns; q++) have.push_back(pack(ci[3 * q], ci[3 * q + 1], ci[3 * q + 2], cw[q]));
    std::vector<double> nc, nr;
    for (long long q = 0; q < m; q++) {
        const double r = hr[q];
        if (!(r > 0) || !std::isfinite(hc[3 * q]) || !std::isfinite(hc[3 * q + 1]) || !std::isfinite(hc[3 * q + 2]))
            continue;
        long long g[3];
        bool ok = true;
        // a shrunk sphere lands on symmetric positions of flat or lattice
        // surfaces, where radical planes can run through mesh faces; a
        // deterministic -1/0/+1 grid-unit move per axis, keyed on the pin's
        // face, keeps the inserted spheres in general position
        unsigned long long hsh = (unsigned long long)kf[q] * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        for (int z = 0; z < 3; z++) {
            hsh ^= hsh >> 29;
            hsh *= 0xBF58476D1CE4E5B9ull;
            hsh ^= hsh >> 32;
            const double v = rint(hc[3 * q + z] * scale) + (double)((long long)(hsh % 3ull) - 1);
            if (!(fabs(v) <= (double)RPD_COORD_MAX)) ok = false;
            g[z] = (long long)v;
        }
        const long long rg = (long long)rint(r * scale);
        if (!ok || rg <= 0) continue;
        const unsigned long long key = pack(g[0], g[1], g[2], rg * rg);
        if (std::find(have.begin(), have.end(), key) != have.end()) continue;
        have.push_back(key);
        for (int z = 0; z < 3; z++) nc.push_back((double)g[z] * unit);
        nr.push_back((double)rg * unit);
    }
    if (nr.empty()) return RPD_OK;
    const long long k = (long long)nr.size();
    double* ic = ctx->alloc<double>(3 * k);
    double* ir = ctx->alloc<double>(k);
    if (!ic || !ir) return fail(ctx, RPD_E_OOM, "device allocation failed");
    cudaMemcpyAsync(ic, nc.data(), sizeof(double) * 3 * k, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(ir, nr.data(), sizeof(double) * k, cudaMemcpyHostToDevice, ctx->stream);
    TRY(rpd_insert(ctx, ic, ir, k));
    *inserted = k;
    return RPD_OK;
}

rpd_status rpd_surface_samples(rpd_ctx* ctx, double* d_points, double* d_normals, int32_t* d_faces, int64_t cap,
                               int64_t* n) {
    if (!ctx) return RPD_E_INVALID;
    double* tri = nullptr;
    int32_t* face_of = nullptr;
    TRY(ensure_boundary(ctx, &tri, &face_of));
    if (n) *n = ctx->nbtri;
    if (!d_points && !d_normals && !d_faces) return RPD_OK;
    if (!d_points || !d_normals || !d_faces || cap < ctx->nbtri)
        return fail(ctx, RPD_E_INVALID, "all three outputs and cap >= n are needed");
    launch_surface_samples(tri, face_of, ctx->nbtri, d_points, d_normals, d_faces, ctx->stream);
    return cuda_check(ctx, "surface sample launch");
}

rpd_status rpd_envelope_distance(rpd_ctx* ctx, const double* d_samples, int64_t n, float* d_dist, int32_t* d_prim) {
    if (!ctx) return RPD_E_INVALID;
    if (n < 0) return fail(ctx, RPD_E_INVALID, "n must be >= 0");
    if (n == 0) return RPD_OK;
    if (!d_samples || !d_dist || !d_prim) return fail(ctx, RPD_E_INVALID, "null pointer");
    const long long n1 = ctx->nkeys[0], n2 = ctx->nkeys[1], n3 = ctx->nkeys[2];
    if (n1 + n2 + n3 >= (1ll << 31)) return fail(ctx, RPD_E_OVERFLOW, "too many medial primitives");
    // coordinates relative to mesh vertex 0 keep the FP32 arithmetic local
    int32_t x0[3];
    cudaMemcpyAsync(x0, ctx->Xi, sizeof(x0), cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RPD_E_CUDA, "CUDA error while reading the mesh origin");
    }
    const double unit = ldexp(1.0, -ctx->opt.grid_bits);
    const double o[3] = {x0[0] * unit, x0[1] * unit, x0[2] * unit};
    void* tmp = ctx->alloc<char>(envelope_tmp_bytes(n1 + n2 + n3, n));
    if (!tmp) return fail(ctx, RPD_E_OOM, "device allocation failed");
    launch_envelope(ctx->fout[0].keys, n1, ctx->fout[1].keys, n2, ctx->fout[2].keys, n3, ctx->Ci, ctx->W, unit, o,
                    d_samples, n, d_dist, d_prim, tmp, &ctx->st->err, ctx->stream);
    return cuda_check(ctx, "envelope launch");
}

// Pins of every non-contractible cell, face and edge, on the host.
static rpd_status topology_pins(rpd_ctx* ctx, std::vector<double>& hp, std::vector<double>& hn,
                                std::vector<int32_t>& hf, long long* nfail) {
    long long nfail_total = 0;
    for (int kind = 1; kind <= 3; kind++) {
        if (!ctx->kind_ok[kind - 1]) continue;
        int64_t m = 0;
        TRY(rpd_pins(ctx, (rpd_kind)kind, nullptr, nullptr, nullptr, nullptr, 0, &m));
        nfail_total += m;
        if (m == 0) continue;
        int32_t* dk = ctx->alloc<int32_t>(m * kind);
        double* dp = ctx->alloc<double>(3 * m);
        double* dn = ctx->alloc<double>(3 * m);
        int32_t* df = ctx->alloc<int32_t>(m);
        if (!dk || !dp || !dn || !df) return fail(ctx, RPD_E_OOM, "device allocation failed");
        TRY(rpd_pins(ctx, (rpd_kind)kind, dk, dp, dn, df, m, &m));
        const size_t b0 = hf.size();
        hp.resize(3 * (b0 + m));
        hn.resize(3 * (b0 + m));
        hf.resize(b0 + m);
        cudaMemcpyAsync(hp.data() + 3 * b0, dp, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(hn.data() + 3 * b0, dn, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(hf.data() + b0, df, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, ctx->stream);
        // the host vectors grow for the next kind: let these copies land first
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, RPD_E_CUDA, "CUDA error while reading pins");
        }
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RPD_E_CUDA, "CUDA error while reading pins");
    }
    *nfail = nfail_total;
    return RPD_OK;
}

rpd_status rpd_repair(rpd_ctx* ctx, int32_t max_rounds, int64_t* rounds, int64_t* inserted, int64_t* failing) {
    if (!ctx) return RPD_E_INVALID;
    if (max_rounds < 0) return fail(ctx, RPD_E_INVALID, "max_rounds must be >= 0");
    long long nround = 0, nins = 0, nfail_total = 0;
    for (;;) {
        std::vector<double> hp, hn;
        std::vector<int32_t> hf;
        TRY(topology_pins(ctx, hp, hn, hf, &nfail_total));
        if (nfail_total == 0 || nround >= max_rounds) break;
        long long k = 0, tried = 0;
        TRY(grow_from_pins(ctx, hp, hn, hf, &k, &tried));
        // a round whose spheres all repeat existing ones still marks its
        // faces used, so the next round pins other faces; stop only when no
        // unused face is left to pin
        if (tried == 0) break;
        nins += k;
        nround++;
    }
    if (rounds) *rounds = nround;
    if (inserted) *inserted = nins;
    if (failing) *failing = nfail_total;
    return RPD_OK;
}

rpd_status rpd_repair_geometry(rpd_ctx* ctx, double delta, int32_t max_rounds, rpd_repair_report* rep) {
    if (!ctx || !rep) return RPD_E_INVALID;
    if (max_rounds < 0 || !(delta > 0)) return fail(ctx, RPD_E_INVALID, "max_rounds >= 0 and delta > 0 are needed");
    *rep = rpd_repair_report{};
    for (;;) {
        std::vector<double> hp, hn;
        std::vector<int32_t> hf;
        long long nfail = 0;
        TRY(topology_pins(ctx, hp, hn, hf, &nfail));
        rep->failing = nfail;
        // surface samples and their distance to the medial mesh's envelope
        int64_t nb = 0;
        TRY(rpd_surface_samples(ctx, nullptr, nullptr, nullptr, 0, &nb));
        double* sp = ctx->alloc<double>(3 * nb + 3);
        double* sn = ctx->alloc<double>(3 * nb + 3);
        int32_t* sf = ctx->alloc<int32_t>(nb + 1);
        float* sd = ctx->alloc<float>(nb + 1);
        int32_t* sa = ctx->alloc<int32_t>(nb + 1);
        if (!sp || !sn || !sf || !sd || !sa) return fail(ctx, RPD_E_OOM, "device allocation failed");
        TRY(rpd_surface_samples(ctx, sp, sn, sf, nb, &nb));
        TRY(rpd_envelope_distance(ctx, sp, nb, sd, sa));
        std::vector<double> gp(3 * nb), gn(3 * nb);
        std::vector<int32_t> gf(nb);
        std::vector<float> gd(nb);
        std::vector<uint8_t> used(ctx->used_faces ? 4 * ctx->nt : 0);
        cudaMemcpyAsync(gp.data(), sp, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(gn.data(), sn, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(gf.data(), sf, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(gd.data(), sd, sizeof(float) * nb, cudaMemcpyDeviceToHost, ctx->stream);
        if (!used.empty()) cudaMemcpyAsync(used.data(), ctx->used_faces, used.size(), cudaMemcpyDeviceToHost, ctx->stream);
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, RPD_E_CUDA, "CUDA error while reading envelope distances");
        }
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (long long q = 0; q < nb; q++)
            for (int z = 0; z < 3; z++) {
                lo[z] = std::min(lo[z], gp[3 * q + z]);
                hi[z] = std::max(hi[z], gp[3 * q + z]);
            }
        const double diag = nb ? sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                      (hi[2] - lo[2]) * (hi[2] - lo[2]))
                               : 0.0;
        std::vector<double> fp, fn;
        std::vector<int32_t> ff;
        long long nfar = 0;
        double mx = -INFINITY;
        std::vector<long long> far;
        for (long long q = 0; q < nb; q++) {
            const double ratio = diag > 0 ? (double)gd[q] / diag : 0.0;
            mx = std::max(mx, ratio);
            if (!(ratio > delta)) continue;
            nfar++;
            if (!used.empty() && used[gf[q]]) continue;
            far.push_back(q);
        }
        // farthest samples first; a sample within three of its distances of
        // one already taken this round waits for the next round (the sphere
        // grown there usually covers it, and clustered insertions of near
        // copies of one sphere only fragment the diagram)
        std::sort(far.begin(), far.end(), [&](long long a, long long b) {
            return gd[a] > gd[b] || (gd[a] == gd[b] && a < b);
        });
        for (long long q : far) {
            const double rho = 3.0 * (double)gd[q];
            bool near = false;
            for (size_t z = 0; z < ff.size() && !near; z++) {
                const double dx = gp[3 * q] - fp[3 * z], dy = gp[3 * q + 1] - fp[3 * z + 1],
                             dz = gp[3 * q + 2] - fp[3 * z + 2];
                near = dx * dx + dy * dy + dz * dz < rho * rho;
            }
            if (near) continue;
            for (int z = 0; z < 3; z++) {
                fp.push_back(gp[3 * q + z]);
                fn.push_back(gn[3 * q + z]);
            }
            ff.push_back(gf[q]);
        }
        rep->far_samples = nfar;
        rep->max_ratio = nb ? mx : 0.0;
        if ((nfail == 0 && nfar == 0) || rep->rounds >= max_rounds) break;
        // topology first (Sec. 4.1), then the geometry (Sec. 4.3)
        long long k = 0;
        if (nfail > 0) TRY(grow_from_pins(ctx, hp, hn, hf, &k));
        if (k == 0 && nfar > 0) TRY(grow_from_pins(ctx, fp, fn, ff, &k));
        if (k == 0) break;
        rep->inserted += k;
        rep->rounds++;
    }
    return RPD_OK;
}

// Copy the finalised rows of one kind: keys [m, kind] and one value array.
static rpd_status copy_rows(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, const void* src, void* d_dst,
                            size_t elem, int64_t cap, int64_t* n) {
    TRY(check_kind(ctx, kind));
    const long long m = ctx->nkeys[kind - 1];
    if (n) *n = m;
    if (!d_keys && !d_dst) return RPD_OK;
    if (cap < m) return fail(ctx, RPD_E_INVALID, "cap is smaller than the number of elements");
    if (m == 0) return RPD_OK;
    const FinalOut& o = ctx->fout[kind - 1];
    launch_copy_rows(d_keys ? o.keys : nullptr, d_keys, m * kind, d_dst ? src : nullptr, d_dst, m, (int)elem,
                     ctx->stream);
    return cuda_check(ctx, "output copy");
}

rpd_status rpd_euler(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, int32_t* d_chi, int64_t cap, int64_t* n) {
    if (!ctx) return RPD_E_INVALID;
    TRY(check_kind(ctx, kind));
    return copy_rows(ctx, kind, d_keys, ctx->fout[kind - 1].chi, d_chi, sizeof(int32_t), cap, n);
}

rpd_status rpd_components(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, int32_t* d_beta0, int64_t cap, int64_t* n) {
    if (!ctx) return RPD_E_INVALID;
    TRY(check_kind(ctx, kind));
    return copy_rows(ctx, kind, d_keys, ctx->fout[kind - 1].beta, d_beta0, sizeof(int32_t), cap, n);
}

rpd_status rpd_contractible(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, uint8_t* d_flag, int64_t cap, int64_t* n) {
    if (!ctx) return RPD_E_INVALID;
    TRY(check_kind(ctx, kind));
    return copy_rows(ctx, kind, d_keys, ctx->fout[kind - 1].flag, d_flag, sizeof(uint8_t), cap, n);
}

rpd_status rpd_export(rpd_ctx* ctx, void* d_out, int64_t cap_bytes, int64_t* bytes) {
    if (!ctx) return RPD_E_INVALID;
    ExportArgs a{};
    const auto al16 = [](long long x) { return (x + 15) & ~15ll; };
    long long off = 0;
    char* base = (char*)d_out;
    for (int k = 1; k <= 4; k++) {
        const long long m = ctx->nkeys[k - 1];
        const FinalOut& o = ctx->fout[k - 1];
        const void* src[3] = {o.keys, o.chi, o.beta};
        const long long n[3] = {m * k, m, m};
        for (int j = 0; j < 3; j++) {
            if (n[j] > 0) a.seg[a.nseg++] = ExportSeg{src[j], base + off, n[j], 4};
            off = al16(off + 4 * n[j]);
        }
    }
    for (int k = 1; k <= 4; k++) {
        const long long m = ctx->nkeys[k - 1];
        if (m > 0) a.seg[a.nseg++] = ExportSeg{ctx->fout[k - 1].flag, base + off, m, 1};
        off = al16(off + m);
    }
    if (bytes) *bytes = off;
    if (!d_out) return RPD_OK;
    if (cap_bytes < off) return fail(ctx, RPD_E_INVALID, "cap_bytes is smaller than the export size");
    if (((uintptr_t)d_out & 15) != 0) return fail(ctx, RPD_E_INVALID, "d_out must be 16-byte aligned");
    launch_export(a, ctx->stream);
    return cuda_check(ctx, "export launch");
}

rpd_status rpd_pieces(rpd_ctx* ctx, int32_t* d_tet, int32_t* d_sphere, double* d_vol, double* d_moment3, int64_t cap,
                      int64_t* n) {
    if (!ctx) return RPD_E_INVALID;
    if (n) *n = ctx->npieces;
    if (!d_tet && !d_sphere && !d_vol && !d_moment3) return RPD_OK;
    if (cap < ctx->npieces) return fail(ctx, RPD_E_INVALID, "cap is smaller than the number of pieces");
    launch_compact_pieces(ctx->clip, ctx->npairs, ctx->piece_off, d_tet, d_sphere, d_vol, d_moment3, ctx->stream);
    return cuda_check(ctx, "piece launch");
}

int64_t rpd_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

rpd_status rpd_stats_get(const rpd_ctx* ctx, rpd_stats* out) {
    if (!ctx || !out) return RPD_E_INVALID;
    stage_times(const_cast<rpd_ctx*>(ctx));
    *out = ctx->stats;
    return RPD_OK;
}

const char* rpd_last_error(const rpd_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

const char* rpd_build_error(void) { return g_build_error.c_str(); }

void rpd_destroy(rpd_ctx* ctx) {
    if (!ctx) return;
    join_side_streams(ctx);   // nothing queued on a side stream may outlive its memory
    ctx->release_all();
    cudaStreamSynchronize(ctx->stream);
    release_events(ctx->device, ctx->ev, 16);
    release_events(ctx->device, ctx->evc, 1 + 2 * RPD_NBINS);
    cudaGetLastError();
    delete ctx;
}

}  // extern "C"

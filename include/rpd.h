/*
 * librpd: volumetric restricted power diagram of a tetrahedral mesh against
 * weighted spheres, with the fractional Euler characteristic, the number of
 * connected components and the contractibility flag of every restricted power
 * cell (RPC), face (RPF), edge (RPE) and vertex (RPV).  CUDA (sm_103a).
 *
 * Definitions (MATTopo, arXiv 2403.18761):
 *   power distance   pd(x, m_i) = |x - c_i|^2 - r_i^2         Sec. 3.2, after Eq. 1
 *   power cell       {x : pd(x,m_i) <= pd(x,m_j) for all j}    Eq. 1
 *   restricted cell  RPC_i = cell_i cap shape                  Eq. 2-3
 *   RPF_ij = RPC_i cap RPC_j, RPE_ijk, RPV_ijkl               Sec. 3.2 (list)
 *   chi = V - E + F - C, fractional per tet                   Sec. 4.1, 4.1.2, Eq. 7
 *   beta0 = connected components ("simple traversal")         Sec. 4.1.1
 *   contractible  <=>  beta0 == 1 and chi == 1                 Sec. 3.3 (Eq. 5-6), Sec. 4.1
 *   Tet-Cell clipping of every (tet, sphere) pair              Sec. 5.2
 *
 * Conventions shared by every call:
 *   - Pointers named d_* are DEVICE memory owned by the caller.  Inputs are
 *     read-only and must stay valid until the work queued on the stream by
 *     the call has finished.  Outputs are written by stream-ordered kernels.
 *   - All work is ordered on the cudaStream_t passed to rpd_build (NULL = the
 *     legacy default stream); later calls on the same ctx use that stream.
 *   - Every call returns an rpd_status; rpd_last_error(ctx) gives a message.
 *   - Element keys are rows of sorted sphere indices (i < j < k < l), rows in
 *     lexicographic order.  Elements with an empty restriction are absent.
 *   - chi and beta0 are exact integers.
 *   - Generic position: a point exactly on a radical plane makes rpd_build
 *     fail with RPD_E_DEGENERATE (no symbolic perturbation).
 */
#ifndef RPD_H
#define RPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RPD_OK = 0,
    RPD_E_INVALID = 1,      /* bad argument, coordinate off the supported range,
                               non-positive tet, NaN, ns == 0                  */
    RPD_E_NONMANIFOLD = 2,  /* a triangle shared by more than two tets          */
    RPD_E_DEGENERATE = 3,   /* an exact predicate evaluated to zero             */
    RPD_E_OOM = 4,          /* device allocation failed                         */
    RPD_E_CUDA = 5,         /* a CUDA runtime call failed                       */
    RPD_E_OVERFLOW = 6,     /* more candidate spheres for one tet than the
                               library supports (32), or key space exceeded    */
    RPD_E_TIMEOUT = 7       /* a bounded device loop or wait gave up (union-find,
                               radix-sort look-back)                          */
} rpd_status;

/* Element kind = number of spheres in its key. */
typedef enum { RPD_CELL = 1, RPD_FACE = 2, RPD_EDGE = 3, RPD_VERTEX = 4 } rpd_kind;

/* Arithmetic of the clipping predicates.  Both give identical combinatorics
 * (uncertified signs fall back to FP64 and then to exact 256-bit integers).
 * Volumes and first moments are accumulated in native FP64 in RPD_FP64 and in
 * double-float arithmetic (unevaluated sums of two FP32 values, about 48
 * significant bits) in RPD_FP32_FILTERED; both stay within 1e-9 of the tet
 * volume of the exact result. */
typedef enum { RPD_FP64 = 0, RPD_FP32_FILTERED = 1 } rpd_precision;

typedef struct {
    int32_t precision;    /* rpd_precision                                        */
    int32_t k;            /* power neighbours kept per mesh vertex, 1..32          */
    int32_t grid_bits;    /* coordinates and radii are rounded to multiples of
                             2^-grid_bits; |x|*2^grid_bits must stay < 2^21       */
    int32_t debug_checks; /* test switches (0 in production): value 1 sends every
                             non-corner clip predicate past the first-stage
                             filter to the FP64 stage, value 2 straight to the
                             exact 256-bit stage; bit 4 makes the neighbour
                             search keep distance and id apart (the form used
                             above 2^17 spheres).  Results must not change.     */
} rpd_options;

typedef struct {
    int64_t n_pairs;          /* candidate (tet, sphere) pairs clipped            */
    int64_t n_pieces;         /* nonempty pieces P(t,i) = t cap cell_i            */
    int64_t n_records[4];     /* per-tet element contributions, by kind           */
    int64_t n_keys[4];        /* distinct elements by kind (after finalisation)   */
    int64_t pred_fast;        /* clip predicates decided by the first-stage filter */
    int64_t pred_fp64;        /* ... by the FP64 re-evaluation                     */
    int64_t pred_exact;       /* ... by exact 256-bit integer arithmetic          */
    int64_t cand_fallback;    /* tets whose candidate set needed the grid search  */
    int64_t whole_tets;       /* tets inside a single cell (no clipping)          */
    int64_t clip_vertices[3]; /* polytope vertices constructed by clipping, by the
                                 number of radical planes through them (1, 2, 3) */
    int64_t bin_pairs[8];     /* candidate pairs by candidate count of their tet:
                                 1, 2, 3, 4, 5-6, 7-8, 9-16, 17-32                */
    int64_t bin_cut[8];       /* nonempty pieces that were cut, per bin           */
    float ms_prep, ms_knn, ms_cand, ms_clip, ms_finalize[4];
    float ms_clip_kernels;    /* from the start of the clip launches to the end of
                                 the last clip kernel (volume pass excluded)      */
    float ms_clip_span;       /* same start to the end of the last volume kernel  */
    int64_t update_tets;      /* tets clipped by the call that produced the
                                 diagram: nt after rpd_build, the tets whose
                                 candidate spheres changed after rpd_insert     */
} rpd_stats;

typedef struct rpd_ctx rpd_ctx;   /* opaque; owns all device workspace and results */

/* Fill *opt with defaults: FP32_FILTERED, k = 16, grid_bits = 20, no debug. */
void rpd_default_options(rpd_options* opt);

/*
 * Build the restricted power diagram (Eq. 1-3) of a tet mesh and spheres and
 * the per-tet fractional Euler contributions (Sec. 4.1.2).
 *   d_verts   f64[nv*3]  vertex coordinates, row-major
 *   d_tets    i32[nt*4]  vertex indices, positively oriented (det > 0)
 *   d_centers f64[ns*3]  sphere centres c_i
 *   d_radii   f64[ns]    sphere radii r_i >= 0 (power weight r_i^2)
 *   opt       options (NULL = defaults)
 *   cuda_stream  a cudaStream_t or NULL
 *   out       receives a new context (NULL on failure)
 * Limits: nv < 2^21, ns < 2^21 (RPV keys need ns < 2^16), nt < 2^26.
 * Synchronises the stream twice: after the candidate stage (the pair count
 * sizes the clip buffers) and at the end (record and element counts size the
 * element tables); a third time only if the record buffers overflowed and the
 * clip is redone.
 */
rpd_status rpd_build(const double* d_verts, int64_t nv, const int32_t* d_tets, int64_t nt,
                     const double* d_centers, const double* d_radii, int64_t ns,
                     const rpd_options* opt, void* cuda_stream, rpd_ctx** out);

/*
 * Fractional Euler characteristic chi of every element of one kind
 * (Sec. 4.1.2: chi = sum of the per-tet contributions, Eq. 7).
 * Two-phase: with d_keys == NULL only *n is set.  Otherwise cap >= *n is
 * required; d_keys i32[n*kind] and d_chi i32[n] are written on the stream.
 */
rpd_status rpd_euler(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, int32_t* d_chi, int64_t cap,
                     int64_t* n);

/* Connected-component count beta0 of every element (Sec. 4.1.1); pieces in
 * face-adjacent tets are connected when the element crosses the shared face.
 * Same two-phase convention; d_beta0 i32[n]. */
rpd_status rpd_components(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, int32_t* d_beta0, int64_t cap,
                          int64_t* n);

/* Contractibility flag (beta0 == 1 && chi == 1; Sec. 3.3 Eq. 5-6, Sec. 4.1)
 * of every element.  Same two-phase convention; d_flag u8[n] (1 = contractible). */
rpd_status rpd_contractible(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, uint8_t* d_flag, int64_t cap,
                            int64_t* n);

/*
 * Insert n_new spheres (appended: they take indices ns .. ns + n_new - 1) and
 * update the diagram in place, clipping only what the new spheres change
 * (partial RPD update, Sec. 4 intro and Sec. 5.2).  The neighbour and
 * candidate stages run again on the enlarged sphere set; every tet whose
 * candidate spheres and clip order are unchanged keeps its pieces, volumes
 * and fractional Euler records, the others are clipped again, and the
 * element tables are finalised over everything.  The result is identical to
 * rpd_build on the concatenated spheres (rpd_stats.update_tets reports how
 * many tets were clipped).
 *   d_centers f64[n_new*3], d_radii f64[n_new]: caller-owned device memory,
 *             read on the context's stream
 * Same synchronisation as rpd_build.  On failure the context keeps the
 * previous diagram and the status says why (RPD_E_INVALID for n_new < 0 or
 * ns + n_new >= 2^21, the device errors of rpd_build otherwise).
 */
rpd_status rpd_insert(rpd_ctx* ctx, const double* d_centers, const double* d_radii, int64_t n_new);

/*
 * Pin points of the non-contractible elements of one kind (1 = RPC, 2 = RPF,
 * 3 = RPE), where the topology repair grows new spheres (Sec. 4.1.1, 4.1.2).
 * The surface is the set of boundary triangles of the mesh (tet faces without
 * a neighbour).  For an element with beta0 > 1 the pin is the centroid of the
 * boundary triangle, touched by the element, of the lowest-numbered tet in a
 * component other than the one of the element's lowest-numbered tet
 * (Sec. 4.1.1: a surface point on another component).  For an element with
 * beta0 = 1 and chi != 1 it is the centroid of the touched boundary triangle
 * furthest from the element's first sphere (Sec. 4.1.2: the furthest surface
 * triangle), ties to the lowest (tet, face).
 *   d_keys    i32[n*kind]  keys of the failing elements, in key order
 *   d_pins    f64[n*3]     pin points (NaN when the element touches no
 *                          qualifying boundary triangle)
 *   d_normals f64[n*3]     unit normals into the shape at the pins
 *   d_faces   i32[n]       boundary face 4*tet + face of the pin, or -1
 * Two-phase: with all outputs NULL only *n (the number of failing elements)
 * is set; otherwise all four and cap >= n are required (RPD_E_INVALID).
 * Synchronises the stream once (the count).
 */
rpd_status rpd_pins(rpd_ctx* ctx, rpd_kind kind, int32_t* d_keys, double* d_pins, double* d_normals,
                    int32_t* d_faces, int64_t cap, int64_t* n);

/*
 * Sphere shrinking (Sec. 5.1, the shrinking-ball algorithm of Ma et al. 2012)
 * from n pin points against the mesh's boundary triangles: starting from a
 * ball tangent at the pin p with a radius above the mesh's extent, the ball
 * is repeatedly replaced by the ball tangent at p through the surface point
 * nearest to its centre, while that point lies inside it (the pin's own
 * triangle is skipped), at most 100 times.  The result is an empty ball
 * touching the surface at p and at one more point.
 *   d_pins, d_normals f64[n*3], d_faces i32[n]: as written by rpd_pins (a
 *                     row with face -1 gives NaN)
 *   d_centers f64[n*3], d_radii f64[n], d_iters i32[n]: outputs (world units;
 *                     iterations taken)
 * Stream-ordered, no synchronisation except on the first call of a context
 * (which builds the boundary-triangle list).
 */
rpd_status rpd_shrink(rpd_ctx* ctx, const double* d_pins, const double* d_normals, const int32_t* d_faces, int64_t n,
                      double* d_centers, double* d_radii, int32_t* d_iters);

/* The context's spheres as the diagram uses them (centres and radii rounded
 * to the grid 2^-grid_bits), those of rpd_build followed by every inserted
 * one: d_centers f64[n*3], d_radii f64[n].  Two-phase like rpd_euler. */
rpd_status rpd_spheres(rpd_ctx* ctx, double* d_centers, double* d_radii, int64_t cap, int64_t* n);

/*
 * Topology repair loop (Sec. 4, 4.1): while some RPC, RPF or RPE is not
 * contractible and fewer than max_rounds rounds have run, take the pins of all
 * failing elements (rpd_pins), one per boundary triangle, grow a sphere from
 * each (rpd_shrink), round it to the grid, drop repeats of existing spheres,
 * and insert them with a partial update (rpd_insert).  The loop also stops
 * when no failing element has a pin or no new sphere remains.
 *   rounds, inserted, failing: host pointers (may be NULL) receiving the rounds
 *   run, the spheres inserted and the failing elements left (0 = every RPC,
 *   RPF and RPE contractible).
 * Synchronises the stream several times per round.
 */
rpd_status rpd_repair(rpd_ctx* ctx, int32_t max_rounds, int64_t* rounds, int64_t* inserted, int64_t* failing);

/* Every element table of rpd_euler, rpd_components and rpd_contractible, for
 * all four kinds, in one launch into one caller-owned device buffer (for
 * bindings that serve many queries).  Layout, in bytes from d_out, every part
 * starting on a multiple of 16 bytes: for kind = 1..4 in order, keys
 * i32[n_k*kind], chi i32[n_k], beta0 i32[n_k]; then for kind = 1..4, flag
 * u8[n_k]; n_k = rpd_stats.n_keys[kind-1].  Two-phase: with d_out == NULL
 * only *bytes is set; otherwise cap_bytes >= *bytes and a 16-byte aligned
 * d_out are required (RPD_E_INVALID).  Written on the build's stream. */
rpd_status rpd_export(rpd_ctx* ctx, void* d_out, int64_t cap_bytes, int64_t* bytes);

/* Nonempty pieces P(t,i) = t cap cell_i (Tet-Cell, Sec. 5.2) sorted by (t, i):
 * d_tet i32[n], d_sphere i32[n], d_vol f64[n], d_moment3 f64[n*3] (integral
 * of x over the piece).  Any output pointer may be NULL.  Same two-phase
 * convention. */
rpd_status rpd_pieces(rpd_ctx* ctx, int32_t* d_tet, int32_t* d_sphere, double* d_vol, double* d_moment3,
                      int64_t cap, int64_t* n);

/* Counters and per-stage device times (CUDA events) of the last build. */
rpd_status rpd_stats_get(const rpd_ctx* ctx, rpd_stats* out);

/* Message for the last non-OK status of this ctx ("" if none). */
const char* rpd_last_error(const rpd_ctx* ctx);

/* Message for the last failed rpd_build (no ctx is returned then). */
const char* rpd_build_error(void);

/* Release the context and all its device memory (synchronises its stream). */
void rpd_destroy(rpd_ctx* ctx);

/* Number of kernel launches the library has issued in this process so far
 * (all contexts, all devices; a host-side counter, no synchronisation).  The
 * difference around a call counts that call's launches. */
int64_t rpd_launch_count(void);

/*
 * rpd_build + rpd_euler in one call that allocates no device memory.  The
 * paper has no counterpart; this is a convenience of the library.
 *
 * For callers that cannot call cudaMalloc when they need the result:
 * pipelines that fix their device-memory budget up front, or services that
 * must not allocate (or fragment the device heap) while they run.  All workspace
 * comes from one file-scope device array of 32 MiB that every GPU loading the
 * library holds until the process exits (enough for roughly 30k tets; larger
 * problems are rejected with RPD_E_OVERFLOW before the stage that would need
 * more).  No cudaMalloc, cudaFree or other allocating routine is called.
 *   inputs  as rpd_build (caller-owned device memory; opt may be NULL)
 *   kind    element kind whose chi is returned
 *   d_keys  i32[n*kind], d_chi i32[n]: caller-owned outputs, cap >= n; both
 *           NULL only sets *n
 *   n       host pointer, receives the number of elements
 * The first call on a device looks up the array's device address and caches
 * it for the rest of the process: make that first call before any stream
 * capture, and do not use the entry point again on a device after
 * cudaDeviceReset there.  Every call reuses the same array (it is cleared as
 * needed), so calls that overlap on the GPU race: serialise them.
 * Synchronises the stream three times (sizes of the later stages are read on
 * the host).  Errors are reported by status only (RPD_E_INVALID for bad
 * arguments or cap < n; RPD_E_OVERFLOW when the problem needs more than the
 * array holds; RPD_E_CUDA; the device errors of rpd_build).
 */
rpd_status rpd_euler_static(const double* d_verts, int64_t nv, const int32_t* d_tets, int64_t nt,
                            const double* d_centers, const double* d_radii, int64_t ns, const rpd_options* opt,
                            void* cuda_stream, rpd_kind kind, int32_t* d_keys, int32_t* d_chi, int64_t cap,
                            int64_t* n);

/*
 * CUDA-core peak of one precision, measured on the current device: every SM
 * runs fully occupied blocks of threads, each with eight independent fused
 * multiply-add chains of `iters` rounds (2 flop per FMA), timed with CUDA
 * events after one shorter warm-up launch.  The paper has no counterpart; it
 * is the denominator of the FP32 and FP64 roofline fractions.
 *   precision  RPD_FP32_FILTERED (FP32 FMA) or RPD_FP64 (FP64 FMA)
 *   iters      rounds per chain, 1..2^40
 *   tflops     host pointer, receives the measured TFLOP/s
 *   ms         host pointer or NULL, receives the timed launch's duration
 * Synchronises the stream.  RPD_E_INVALID for bad arguments, RPD_E_CUDA if a
 * launch or the timing fails.
 */
rpd_status rpd_peak_fma(int32_t precision, int64_t iters, void* cuda_stream, double* tflops, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* RPD_H */

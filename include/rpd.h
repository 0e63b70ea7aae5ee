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
    RPD_E_TIMEOUT = 7       /* a bounded device loop gave up (union-find)       */
} rpd_status;

/* Element kind = number of spheres in its key. */
typedef enum { RPD_CELL = 1, RPD_FACE = 2, RPD_EDGE = 3, RPD_VERTEX = 4 } rpd_kind;

/* Arithmetic of the clipping predicates.  Both give identical combinatorics
 * (uncertified signs fall back to FP64 and then to exact 256-bit integers);
 * volumes and moments are accumulated in FP64 in both. */
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
 * Limits: nv < 2^21, ns <= 2^21 (RPV keys need ns <= 2^16), nt < 2^31.
 * Synchronises the stream once at the end (to size the element tables).
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
 * For callers that cannot call cudaMalloc when they need the result: work
 * recorded into a CUDA graph (allocation is illegal during stream capture),
 * or pipelines that fix their device-memory budget up front.  All workspace
 * comes from one file-scope device array of 32 MiB that every GPU loading the
 * library holds until the process exits (enough for roughly 30k tets; larger
 * problems are rejected with RPD_E_OVERFLOW before the stage that would need
 * more).  No cudaMalloc, cudaFree or other allocating routine is called.
 *   inputs  as rpd_build (caller-owned device memory; opt may be NULL)
 *   kind    element kind whose chi is returned
 *   d_keys  i32[n*kind], d_chi i32[n]: caller-owned outputs, cap >= n; both
 *           NULL only sets *n
 *   n       host pointer, receives the number of elements
 * The first call on a device looks up the array's device address: make it
 * before any stream capture.  Every call reuses the same array (it is
 * cleared as needed), so calls that overlap on the GPU race: serialise them.
 * Synchronises the stream.  Errors are reported by status only.
 */
rpd_status rpd_euler_static(const double* d_verts, int64_t nv, const int32_t* d_tets, int64_t nt,
                            const double* d_centers, const double* d_radii, int64_t ns, const rpd_options* opt,
                            void* cuda_stream, rpd_kind kind, int32_t* d_keys, int32_t* d_chi, int64_t cap,
                            int64_t* n);

#ifdef __cplusplus
}
#endif

#endif /* RPD_H */

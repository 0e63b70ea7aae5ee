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
                             above 2^17 spheres); bit 8 keeps the heaviest
                             spheres out of the neighbour grid and scans them
                             first (a tuning choice, off by default: slower on
                             the organic blob).  Results must not change.       */
    int32_t edge_lengths; /* 1: the volume pass also measures every restricted
                             power edge segment (rpd_edge_lengths and rpd_medial
                             need it, and partial updates keep it); 0: skipped  */
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

/* Fill *opt with defaults: FP32_FILTERED, k = 16, grid_bits = 20, no debug,
 * no edge lengths. */
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
 * Batched build (not in the paper, which builds one shape at a time): nshapes
 * independent problems in one context.  Their arrays are concatenated, shape
 * s owning vertices [h_vert_off[s], h_vert_off[s+1]), tets [h_tet_off[s],
 * ...) and spheres [h_sphere_off[s], ...) (HOST i64[nshapes + 1] prefix
 * offsets from 0); tets hold GLOBAL vertex indices, each inside its own shape
 * (RPD_E_INVALID otherwise).  Every stage runs once over the union: the
 * neighbour search walks one sphere grid per shape, so a tet sees only its
 * own shape's spheres, and the pairs of all shapes are binned together by
 * candidate count, so shapes of uneven size share the launches.  Results use
 * global tet and sphere ids; shape s's rows of every table are contiguous
 * (rpd_batch_offsets) and equal those of rpd_build on shape s alone with its
 * ids shifted by its offsets.
 * Limits: fewer than 2^21 spheres in all (RPV keys, as for rpd_build, need
 * fewer than 2^16), at most 5600 per shape (one grid of 2 n_s + 64 cells in
 * shared memory), shapes of >= 4 vertices, 1 tet and 1 sphere; no
 * rpd_insert (and so no repair loop) on a batch context.
 * Synchronises like rpd_build.
 */
rpd_status rpd_build_batch(const double* d_verts, const int32_t* d_tets, const double* d_centers,
                           const double* d_radii, int32_t nshapes, const int64_t* h_vert_off,
                           const int64_t* h_tet_off, const int64_t* h_sphere_off, const rpd_options* opt,
                           void* cuda_stream, rpd_ctx** out);
/* Per-shape row ranges of a batch's tables: h_off (HOST i64[nshapes + 1])
 * receives the first row of each shape and the total, for kind 1..4 (the
 * rows of rpd_euler / rpd_components / rpd_contractible) or 0 (the pieces
 * of rpd_pieces).  Synchronises the stream. */
rpd_status rpd_batch_offsets(rpd_ctx* ctx, int32_t kind, int64_t* h_off);

/*
 * Autotuner (not in the paper): builds the problem (or batch) with each
 * neighbour count k in ks[0..nk) (nk <= 32), reps timed builds after one
 * warm-up per k (reps <= 64), CUDA events on the stream, and returns in
 * *best the base options (NULL = defaults) with the k of the fastest median
 * build, and that median in *ms_best (may be NULL).  The diagram does not
 * depend on k (the candidate sets are exact), only the time does.  The clip's
 * tiles follow each tet's candidate count and need no tuning.  Errors of a
 * build are returned as they are.
 */
rpd_status rpd_autotune(const double* d_verts, int64_t nv, const int32_t* d_tets, int64_t nt, const double* d_centers,
                        const double* d_radii, int64_t ns, const rpd_options* base, const int32_t* ks, int32_t nk,
                        int32_t reps, void* cuda_stream, rpd_options* best, float* ms_best);
rpd_status rpd_autotune_batch(const double* d_verts, const int32_t* d_tets, const double* d_centers,
                              const double* d_radii, int32_t nshapes, const int64_t* h_vert_off,
                              const int64_t* h_tet_off, const int64_t* h_sphere_off, const rpd_options* base,
                              const int32_t* ks, int32_t nk, int32_t reps, void* cuda_stream, rpd_options* best,
                              float* ms_best);

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
 * triangle), ties to the lowest (tet, face).  Boundary triangles that the
 * repair loop (rpd_repair) of this context has already grown a sphere from are
 * skipped, so that a failing element gets a new place to grow from.
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

/*
 * Sphere shrinking from a proposed first radius (the learned proposer below;
 * not in the paper).  d_r_start f64[n]: the first ball's radius per pin, 0 for
 * the plain start.  The balls tangent at p are nested, so a first ball that
 * holds a surface point lies above the fixed point and the shrinking reaches
 * the same sphere as from the plain start; a first ball that holds none may
 * lie below it, and that pin starts over from the plain radius (d_restarted
 * i32[n], may be NULL, gets 1 there).  d_iters counts the rejected test too.
 * Otherwise as rpd_shrink.
 */
rpd_status rpd_shrink_warm(rpd_ctx* ctx, const double* d_pins, const double* d_normals, const int32_t* d_faces,
                           int64_t n, const double* d_r_start, double* d_centers, double* d_radii, int32_t* d_iters,
                           int32_t* d_restarted);

/*
 * Proposer inputs (not in the paper): for each pin p with inward normal n,
 * RPD_PIN_FEATURES floats: u = (p - box centre) / (half the box's longest
 * side) (3), n (3), and sin(pi 2^o u_a), cos(pi 2^o u_a) for o = 0..3 and
 * a = x, y, z in that order (24); the box is the mesh's bounding box.
 * d_x f32[n * RPD_PIN_FEATURES]; with d_radii f64[n] (may be NULL) also the
 * regression targets d_t f32[n] = log2(r / box diagonal).  Stream-ordered
 * (the first call of a context synchronises once to measure the box).
 */
#define RPD_PIN_FEATURES 30
rpd_status rpd_pin_features(rpd_ctx* ctx, const double* d_pins, const double* d_normals, const double* d_radii,
                            int64_t n, float* d_x, float* d_t);

/* Length of every restricted power edge RPE_ijk (the total length of its
 * segments), with its key; the dual triangle's importance in the thinning
 * (Sec. 5.3).  d_keys i32[n*3], d_len f64[n] (world units); two-phase like
 * rpd_euler.  Lengths are summed per key in 64-bit fixed point (2^-24 grid
 * units), so they do not depend on the order of the segments.  The context
 * must be built with rpd_options.edge_lengths = 1 (RPD_E_INVALID otherwise);
 * so must rpd_medial's. */
rpd_status rpd_edge_lengths(rpd_ctx* ctx, int32_t* d_keys, double* d_len, int64_t cap, int64_t* n);

typedef struct {
    int64_t vertices, edges, faces, tets;    /* medial mesh: RPC, RPF, RPE, RPV keys */
    int64_t edges_thin, faces_thin, tets_thin; /* after thinning (vertices stay)     */
    int64_t chi, chi_thin;                   /* V - E + F - T before and after       */
} rpd_medial_info;

/*
 * Dual medial mesh (Sec. 3.2: a vertex per RPC, an edge per RPF, a triangle
 * per RPE, a tetrahedron per RPV) and its geometry-guided thinning (Sec. 5.3):
 * tet-triangle simple pairs are removed in ascending importance
 * alpha_ijk = |RPE_ijk| / mean(2 r_i, 2 r_j, 2 r_k) until no tetrahedron is
 * left, then triangle-edge simple pairs whose triangle belonged to an original
 * tetrahedron while alpha < sigma (0.3 for CAD-like, 0.1 for organic shapes in
 * the paper).  Ties go to the smaller triangle key, and a triangle with several
 * free edges gives up the edge with the smallest key.  The pruning runs on the
 * host (a sequential priority process); the tables and lengths come from the
 * device.
 *   info     host pointer, receives the counts and Euler characteristics
 *   h_edges  HOST i32[cap_e*2] or NULL: the thinned mesh's edges, sorted keys
 *   h_faces  HOST i32[cap_f*3] or NULL: its triangles
 * Synchronises the stream.  RPD_E_INVALID for sigma < 0 or a cap below the
 * thinned count (info is filled first).
 */
rpd_status rpd_medial(rpd_ctx* ctx, double sigma, rpd_medial_info* info, int32_t* h_edges, int64_t cap_e,
                      int32_t* h_faces, int64_t cap_f);

/* The context's spheres as the diagram uses them (centres and radii rounded
 * to the grid 2^-grid_bits), those of rpd_build followed by every inserted
 * one: d_centers f64[n*3], d_radii f64[n].  Two-phase like rpd_euler. */
rpd_status rpd_spheres(rpd_ctx* ctx, double* d_centers, double* d_radii, int64_t cap, int64_t* n);

/*
 * Topology repair loop (Sec. 4, 4.1): while some RPC, RPF or RPE is not
 * contractible and fewer than max_rounds rounds have run, take the pins of all
 * failing elements (rpd_pins), one per boundary triangle, grow a sphere from
 * each (rpd_shrink), round it to the grid, drop repeats of existing spheres,
 * and insert them with a partial update (rpd_insert).  A pin's boundary
 * triangle is marked used once a sphere has been grown from it, whether or not
 * the sphere was new, and pins skip used triangles; the loop also stops when
 * no failing element has an unused triangle to pin.
 *   rounds, inserted, failing: host pointers (may be NULL) receiving the rounds
 *   run, the spheres inserted and the failing elements left (0 = every RPC,
 *   RPF and RPE contractible).
 * Synchronises the stream several times per round.
 */
rpd_status rpd_repair(rpd_ctx* ctx, int32_t max_rounds, int64_t* rounds, int64_t* inserted, int64_t* failing);

/* Surface samples of the shape: the centroid of every boundary triangle of
 * the mesh (tet faces without a neighbour), its unit normal into the shape
 * and its face id 4*tet + face.  d_points, d_normals f64[n*3], d_faces i32[n];
 * two-phase like rpd_euler.  Synchronises the stream on its first call. */
rpd_status rpd_surface_samples(rpd_ctx* ctx, double* d_points, double* d_normals, int32_t* d_faces, int64_t cap,
                               int64_t* n);

/*
 * Geometric preservation (Sec. 4.3): signed distance from each sample point to
 * the enveloping volume of the medial mesh, the union of its spheres (RPC
 * vertices), medial cones (RPF edges: spheres interpolated linearly between
 * two) and medial slabs (RPE triangles: between three); negative inside.
 * Each primitive's distance min |s - c(l)| - r(l) over its interpolated
 * spheres is taken from its interior stationary point in closed form (the
 * primitive's boundary is made of the lower primitives), in FP32 on
 * coordinates relative to mesh vertex 0; the primitives are sorted by the
 * Morton code of their centre and tiles farther than a sample's best distance
 * are skipped.
 *   d_samples f64[n*3]  points (world units), caller-owned device memory
 *   d_dist    f32[n]    distances (world units)
 *   d_prim    i32[n]    nearest primitive: row of the RPC table, then n_RPC +
 *                       row of the RPF table, then n_RPC + n_RPF + row of the
 *                       RPE table; -1 when there is none
 * Synchronises the stream once (the mesh origin).
 */
rpd_status rpd_envelope_distance(rpd_ctx* ctx, const double* d_samples, int64_t n, float* d_dist, int32_t* d_prim);

typedef struct {
    int64_t rounds;       /* rounds that inserted spheres                             */
    int64_t inserted;     /* spheres inserted                                         */
    int64_t failing;      /* non-contractible RPC/RPF/RPE left                        */
    int64_t far_samples;  /* surface samples farther than delta x diagonal left       */
    double max_ratio;     /* largest sample distance / bounding-box diagonal left     */
} rpd_repair_report;

/*
 * The repair loop with geometric preservation (Sec. 4.1, 4.3): each round
 * grows spheres from the pins of the failing elements (as rpd_repair) or, once
 * every RPC, RPF and RPE is contractible, from the surface samples whose
 * distance to the envelope exceeds delta times the samples' bounding-box
 * diagonal (Sec. 4.3's threshold), and inserts them with a partial update.
 * Far samples are taken farthest first, skipping any within three times its
 * own distance of a sample already taken in the round (a reading: the paper
 * inserts a sphere per far sample without saying how many per round).  It
 * stops when both are satisfied, when max_rounds rounds have run, or when a
 * round has nothing new to insert.
 *   rep  host pointer, receives the report (always filled on RPD_OK)
 */
rpd_status rpd_repair_geometry(rpd_ctx* ctx, double delta, int32_t max_rounds, rpd_repair_report* rep);

/*
 * Learned sphere proposer (the paper has no counterpart: it grows every sphere
 * by sphere shrinking, Sec. 5.1).  A multilayer perceptron with n_in <= 32
 * inputs, three hidden layers of 128 ReLU units and one linear output,
 * trained on pairs (features of a pin -> radius the plain sphere shrinking
 * grows from it); its prediction only sets where the shrinking starts
 * (rpd_shrink_warm), so the grown sphere stays the plain method's and the
 * exact RPD check stays the judge.  Hidden layers run on the tensor cores
 * (tcgen05, BF16 operands, FP32 accumulation in tensor memory) in the
 * library's own forward and backward kernels; weights are kept in FP32 and
 * cast to BF16 for each step; Adam (beta 0.9 / 0.999, eps 1e-8).
 * The network's buffers are its own device allocations (cudaMalloc).
 * Parameter vector layout (FP32, 37377 values): W0[128][32], b0[128],
 * W1[128][128], b1[128], W2[128][128], b2[128], w3[128], b3; W0's columns
 * past n_in are zero.  Inputs: d_x f32[n][n_in] row-major, d_t f32[n].
 * Every call synchronises the network's stream and returns RPD_E_TIMEOUT if
 * a tensor-core completion wait ran out, RPD_E_CUDA / RPD_E_OOM otherwise.
 */
typedef struct rpd_mlp rpd_mlp;
rpd_status rpd_mlp_create(int32_t n_in, uint64_t seed, void* cuda_stream, rpd_mlp** out);
/* Copy the parameters out (d_out f32[cap], cap >= 37377) or in. */
rpd_status rpd_mlp_params(rpd_mlp* mlp, float* d_out, int64_t cap, int64_t* n);
rpd_status rpd_mlp_set_params(rpd_mlp* mlp, const float* d_in, int64_t n);
/* Predictions d_y f32[n]. */
rpd_status rpd_mlp_forward(rpd_mlp* mlp, const float* d_x, int64_t n, float* d_y);
/* Gradient (d_grad f32[37377], may be NULL) of the mean squared error
 * mean((y - t)^2) over the n rows, and the loss on the host; no update. */
rpd_status rpd_mlp_grad(rpd_mlp* mlp, const float* d_x, const float* d_t, int64_t n, float* d_grad, float* h_loss);
/* `steps` Adam steps with learning rate lr on consecutive batches of `batch`
 * rows (row r of a batch is row (start + r) mod n, each batch starting where
 * the last ended; shuffle the rows beforehand); *h_loss = the last step's
 * loss.  The batch rows are chosen on the device, so one step's launches are
 * captured once as a CUDA graph on the network's private stream and replayed
 * `steps` times. */
rpd_status rpd_mlp_train(rpd_mlp* mlp, const float* d_x, const float* d_t, int64_t n, int32_t steps, int32_t batch,
                         float lr, float* h_loss);
void rpd_mlp_destroy(rpd_mlp* mlp);

/* First radii proposed by a network for n pins: d_r_start f64[n] =
 * margin * diag * 2^y with y the network's output on rpd_pin_features
 * (margin >= 1 aims above the fixed point).  Synchronises both streams. */
rpd_status rpd_propose(rpd_ctx* ctx, rpd_mlp* mlp, const double* d_pins, const double* d_normals, int64_t n,
                       double margin, double* d_r_start);
/* Make rpd_repair and rpd_repair_geometry start each shrinking from the
 * network's proposal (rpd_propose + rpd_shrink_warm); NULL restores the
 * plain start.  The context does not own the network. */
rpd_status rpd_set_proposer(rpd_ctx* ctx, rpd_mlp* mlp, double margin);
/* Sphere-shrinking work of the context's repair loops so far: pins shrunk,
 * iterations summed over them, proposals rejected. */
rpd_status rpd_shrink_counters(rpd_ctx* ctx, int64_t* pins, int64_t* iters, int64_t* restarts);

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
 * Every call looks up the array's device address on the current device
 * (host-side, no device work), so a context re-created after
 * cudaDeviceReset is served too.  Every call reuses the same array (it is
 * cleared as needed), so calls that overlap on the GPU race: serialise them.
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

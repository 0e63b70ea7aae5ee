// Host-side launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

// Uniform grid over the sphere centres (computed on the device).
struct GridParams {
    int3 org;          // minimum corner (grid units)
    int cell;          // cell edge length (grid units)
    int3 dim;          // cells per axis
    int ncell;
    long long wmax;    // largest power weight r^2
    long long cbase;   // offset of this grid's cells in the cell arrays (batches: one grid per shape)
    long long sbase;   // id of the grid's first sphere (its slots hold ids relative to it)
};

// ---------------------------------------------------------------- prep.cu
// Round coordinates and radii to the integer grid and validate them.
void launch_snap(const double* d_verts, long long nv, const double* d_centers, const double* d_radii,
                 long long ns, int grid_bits, int32_t* Xi, int32_t* Ci, long long* W, DevState* st,
                 cudaStream_t s);
// Validate tets (index range, exact orientation) and build adjacency and the
// 14 ownership bits per tet (4 corners, 6 edges, 4 faces: bit set when this
// tet is the lowest-numbered tet containing that mesh face).
size_t prep_tmp_bytes(long long nt, long long nv);
void launch_prep_mesh(const int32_t* d_tets, long long nt, long long nv, const int32_t* Xi, int32_t* adj,
                      uint32_t* own, void* tmp, DevState* st, cudaStream_t s);

// ----------------------------------------------------------------- knn.cu
size_t grid_tmp_bytes(long long ns, long long ncap);
// Counting sort of the spheres into grid cells: cell_start (ncap + 1
// offsets), and per sorted slot the sphere id, (centre, id) and weight;
// cell_wmax (2 ncap entries) gets the largest weight r^2 of each cell, then
// of each row of cells along x (index z * dim.y + y).
void launch_sphere_grid(const int32_t* Ci, const long long* W, long long ns, long long ncap, GridParams* gp,
                        int64_t* cell_start, int32_t* cell_ids, int4* cell_sph, long long* cell_w,
                        long long* cell_wmax, void* tmp, cudaStream_t s, const long long* wcut = nullptr);
// Heavy spheres (the up to min(128, ns / 128) largest weights): *wcut = the
// largest weight left in the grid (spheres above it are heavy), hsph/hw
// their (centre, id) and weights in id order, *nheavy their count.  Pass
// wcut to launch_sphere_grid and the rest to launch_knn / launch_candidates.
int heavy_count(long long ns);
void launch_heavy_select(const int32_t* Ci, const long long* W, long long ns, long long* wcut, int4* hsph,
                         long long* hw, int* nheavy, cudaStream_t s);
// k nearest spheres in power distance of every mesh vertex, with D+ = a lower
// bound of the power distance of every sphere left out of the list.
// tmp must hold knn_tmp_bytes(nv); ncap bounds the number of grid cells.
size_t knn_tmp_bytes(long long nv);
void launch_knn(const int32_t* Xi, long long nv, long long ns, const GridParams* gp, const int64_t* cell_start,
                const int4* cell_sph, const long long* cell_w, const long long* cell_wmax, long long ncap, int K,
                int32_t* knn, long long* dplus, void* tmp, int* d_err, bool two_word, cudaStream_t s,
                const long long* voff = nullptr, int nshapes = 1, const int4* hsph = nullptr,
                const long long* hw = nullptr, const int* nheavy = nullptr);
// Batches: one grid per shape, all built by one launch (a block per shape).
// Shape s owns spheres [soff[s], soff[s + 1]) (device array) and cells
// [2 soff[s] + 65 s, 2 soff[s + 1] + 65 (s + 1)) of cell_start (its
// 2 n_s + 64 cells and one end offset) and of both halves of cell_wmax
// (cell maxima, then row maxima at + ncap_total).  Every shape needs
// 2 n_s + 64 <= batch_grid_cap() cells.
long long batch_grid_cap();
void launch_sphere_grid_batch(const int32_t* Ci, const long long* W, const long long* soff, int nshapes,
                              long long ncap_total, GridParams* gp, int64_t* cell_start, int32_t* cell_ids,
                              int4* cell_sph, long long* cell_w, long long* cell_wmax, long long max_shape_ncap,
                              cudaStream_t s);
// Candidate spheres of every tet (superset of the spheres whose cell meets
// the tet with positive volume), sorted by index, at most RPD_MAXC.
void launch_candidates(const int32_t* d_tets, long long nt, long long nv, const int32_t* Xi, const int32_t* Ci,
                       const long long* W, const int32_t* knn, const long long* dplus, int K,
                       const GridParams* gp, const int64_t* cell_start, const int32_t* cell_ids,
                       const long long* cell_wmax, int32_t* cand_cnt, int32_t* cand, uint8_t* cand_ord,
                       int32_t* fb_list, int32_t* fb_count, DevState* st, cudaStream_t s,
                       const long long* voff = nullptr, int nshapes = 1, const int4* hsph = nullptr,
                       const long long* hw = nullptr, const int* nheavy = nullptr);

// ---------------------------------------------------------------- clip.cu
struct ClipArgs {
    const int32_t* tets;
    const int32_t* Xi;
    const int32_t* Ci;
    const long long* W;
    const uint32_t* own;
    const int32_t* adj;
    const int32_t* cand_cnt;   // [nt]
    const int32_t* cand;       // [nt * RPD_MAXC], sorted by sphere index
    const uint8_t* cand_ord;   // [nt * RPD_MAXC], slots in clip order
    const int64_t* pair_off;   // [nt + 1]
    const int32_t* pair_tet;   // [npairs]
    double unit;               // 2^-grid_bits
    // per-pair outputs
    uint8_t* pflag;            // 1 = nonempty piece
    int32_t* c_val;            // RPC contribution (owner rule)
    uint8_t* c_link;           // bits 0-3: shared tet faces the piece crosses
                               // (component links); bits 4-7: tet faces on
                               // which it has a face (boundary touches)
    double* p_vol;
    double* p_mom;             // [npairs * 3]
    int32_t* f_off;
    uint8_t* f_cnt;
    int32_t* e_off;
    uint8_t* e_cnt;
    // element records (RPF, RPE, RPV): key, tet, contribution, links
    uint64_t* rkey[3];
    int32_t* rtet[3];
    int16_t* rval[3];
    uint8_t* rlink[3];            // bits 0-3 links across shared tet faces,
                                  // bits 4-7 tet faces the element touches
    long long rcap[3];
    long long* elen;              // per RPE record: length of its segment in
                                  // grid units x 2^24 (fixed point), or NULL
    unsigned long long* rcount;   // [3] device counters
    int key_bits;                 // bits per sphere index in packed keys
    int force_slow;               // 0; 1 = skip the first-stage filter; 2 = exact only
    int uf_limit;                 // iteration bound of the union-find loops
    DevState* st;
    // volume queue of the bin being launched (cut pieces)
    int32_t* qpair;               // [qcap] pair ids
    uint8_t* qnv;                 // [qcap] vertex counts
    uint32_t* qtrip;              // [vmax * qcap] triplets, vertex-major
    long long qcap;
    unsigned long long* qcount;   // device counter
};
// Pairs are grouped into bins by the candidate count n of their tet
// (0: n = 1, whole tet; 1..3: n = 2..4; 4: 5-6; 5: 7-8; 6: 9-16; 7: 17-32).
#define RPD_NBINS 8
int clip_vmax(int bin);
// `only` (NULL = every tet) restricts the binning to the tets it marks.
void launch_bin_count(const int32_t* cand_cnt, long long nt, int32_t* bin_count, cudaStream_t s,
                      const uint8_t* only = nullptr);
// bins: one array of npairs pair ids, bin b starting at sum of earlier counts.
// Pairs grouped by bin (pair_tet and bins hold cap entries; writes past cap
// are dropped); also zeroes the record and queue counters when given.
// pair_tet is filled for every pair, the bins only for the tets `only` marks.
void launch_bin_pairs(const int32_t* cand_cnt, const int64_t* pair_off, long long nt, int32_t* pair_tet,
                      int32_t* bins, const int32_t* bin_count, int32_t* bin_fill, long long cap,
                      unsigned long long* rcount, unsigned long long* qcount, cudaStream_t s,
                      const uint8_t* only = nullptr);
// Pair counts are read on the device (d_n); n/nmax only size the grid.
void launch_whole_tets(const ClipArgs& a, const int32_t* pairs, const int32_t* d_n, long long nmax, cudaStream_t s);
void launch_clip(const ClipArgs& a, int bin, int precision, const int32_t* pairs, const int32_t* d_n, long long n,
                 cudaStream_t s);
// Fractional Euler records of the cut pieces queued by bin `bin` (at most n).
void launch_records(const ClipArgs& a, int bin, long long n, cudaStream_t s);
// Volume and first moment of the cut pieces queued by bin `bin` (at most n).
void launch_volume(const ClipArgs& a, int bin, int precision, long long n, cudaStream_t s);

// -------------------------------------------------------------- update.cu
// changed[t] = 1 where tet t's candidate count, candidates or clip order
// differ between the new and the old context; *n_changed counts them.
void launch_cand_diff(const int32_t* cnt_new, const int32_t* cand_new, const uint8_t* ord_new, const int32_t* cnt_old,
                      const int32_t* cand_old, const uint8_t* ord_old, long long nt, uint8_t* changed,
                      unsigned long long* n_changed, cudaStream_t s);
size_t keep_tmp_bytes(long long npairs, long long n_old_rpv);
// Per-pair outputs and element records of the unchanged tets copied from the
// old context (o) into the new one (a), packed keys repacked from ob to nb
// bits per sphere index; a.rcount receives the kept record counts.
void launch_keep(const ClipArgs& o, long long n_old_rpv, const ClipArgs& a, long long npairs, const uint8_t* changed,
                 int ob, int nb, void* tmp, cudaStream_t s);

// -------------------------------------------------------------- repair.cu
// Boundary triangles of the mesh (tet faces without a neighbour):
// pos[4 nt] (exclusive scan of the boundary flags) gives their number.
size_t boundary_tmp_bytes(long long nt);
void launch_boundary_count(const int32_t* adj, long long nt, int64_t* pos, void* tmp, cudaStream_t s);
void launch_boundary_fill(const int32_t* tets, const int32_t* adj, const int32_t* Xi, long long nt, const int64_t* pos,
                          double unit, double* tri, int32_t* face_of, cudaStream_t s);
// Pin points of the non-contractible elements of one kind (1..3): count
// (pins_fpos(tmp)[nkeys] = number of failing elements), then the pins.
size_t pins_tmp_bytes(long long nkeys);
void launch_pins_count(const uint8_t* flag, long long nkeys, void* tmp, cudaStream_t s);
const int64_t* pins_fpos(const void* tmp, long long nkeys);
void launch_pins(const ClipArgs& a, int kind, const int32_t* keys, const int32_t* beta, const int32_t* chi,
                 const uint8_t* flag, long long nkeys, long long nfail, const int32_t* parent, long long nmax,
                 int uf_limit, const uint8_t* used, void* tmp, int32_t* out_keys, double* pins, double* normals,
                 int32_t* faces, cudaStream_t s);
// Centroids, inward unit normals and face ids of the nb boundary triangles.
void launch_surface_samples(const double* tri, const int32_t* face_of, long long nb, double* pts, double* nrm,
                            int32_t* faces, cudaStream_t s);
// used[faces[i]] = 1 for the n face ids given (those outside [0, n4) skipped).
void launch_mark_faces(const int32_t* faces, long long n, uint8_t* used, long long n4, cudaStream_t s);
// Per-key sums of the RPE records' fixed-point segment lengths (a.elen) into
// len[nkeys] (zeroed here), the records' keys found in the sorted kind-3 rows.
void launch_edge_length_sum(const ClipArgs& a, long long nmax, const int32_t* keys, long long nkeys, long long* len,
                            cudaStream_t s);
// out[i] = (double)in[i] * scale (fixed-point lengths to world units).
void launch_fixed_to_world(const long long* in, double* out, long long n, double scale, cudaStream_t s);
// ----------------------------------------------------------- envelope.cu
// Signed distance (FP32) of samples to the medial mesh's spheres (k1 rows),
// cones (k2 rows) and slabs (k3 rows), coordinates taken relative to o3;
// prim_id receives the nearest primitive (row in spheres, cones, slabs order)
// or -1.  tmp holds envelope_tmp_bytes(n1 + n2 + n3, nsamp).
size_t envelope_tmp_bytes(long long np, long long nsamp);
void launch_envelope(const int32_t* k1, long long n1, const int32_t* k2, long long n2, const int32_t* k3, long long n3,
                     const int32_t* Ci, const long long* W, double unit, const double* o3, const double* samples,
                     long long nsamp, float* dist, int32_t* prim_id, void* tmp, int* d_err, cudaStream_t s);
// ------------------------------------------------------------- medial.cu
// Thinning of the medial mesh (host): alive flags of the edges, triangles
// and tetrahedra (sorted key rows) after removing simple pairs.
#include <vector>
int medial_thin(const std::vector<int32_t>& edges, const std::vector<int32_t>& faces,
                const std::vector<double>& alpha, const std::vector<int32_t>& tets, double sigma,
                std::vector<uint8_t>& edge_alive, std::vector<uint8_t>& face_alive, std::vector<uint8_t>& tet_alive);
// The context's spheres after grid rounding, in world units.
void launch_sphere_out(const int32_t* Ci, const long long* W, long long ns, double unit, double* c, double* r,
                       cudaStream_t s);
// --------------------------------------------------------------- batch.cu
// Device offsets voff/toff (nshapes + 1 entries).  A tet with a corner of
// another shape raises RPD_E_INVALID on the status word.
void launch_batch_check(const int32_t* tets, const long long* toff, const long long* voff, int nshapes,
                        long long nt, DevState* st, cudaStream_t s);
// out[0..nshapes]: first row of each shape in a table sorted by its leading
// column (row stride `stride` int32), by the leading-column bounds `bound`.
void launch_batch_cut(const int32_t* lead, long long rows, int stride, const long long* bound, int nshapes,
                      long long* out, cudaStream_t s);
void launch_batch_cut_pieces(const int64_t* pair_off, const int64_t* piece_off, const long long* toff, int nshapes,
                             long long* out, cudaStream_t s);

// Sphere shrinking from n pins against the boundary triangles; r_start
// (NULL or per pin, 0 = plain) proposes the first radius, restarted (NULL or
// per pin) flags proposals that were rejected.
// FP32 bounding balls (centre, radius) of the boundary triangles, for the
// shrinking's cull.
void launch_boundary_spheres(const double* tri, long long n, float4* bs, cudaStream_t s);
void launch_shrink(const double* tri, const float4* bs, long long ntri, const int32_t* face_of, const double* pins,
                   const double* normals, const int32_t* faces, long long n, double r0, const double* r_start,
                   double* centres, double* radii, int32_t* iters, int32_t* restarted, cudaStream_t s);
// Learned proposer glue: pin features (and log2(r / diag) targets), the
// decoded first radius, and the grid vertices' bounding box (int[6]).
void launch_pin_features(const double* pins, const double* normals, const double* radii, long long n,
                         const double* bc, double bh, double diag, float* x, float* t, cudaStream_t s);
void launch_radius_start(const float* y, long long n, double diag, double margin, double* rs, cudaStream_t s);
void launch_bbox(const int32_t* X, long long nv, int* b, cudaStream_t s);

// ---------------------------------------------------------------- topo.cu
// Iteration bound for ClipArgs::uf_limit (a test hook may lower it).
int uf_iteration_limit();
// Union-find over the nodes of one element kind; writes root flags into the
// payload (bit 16) next to the 16-bit contribution.
// A5-A7 for one element kind (1 = cells from the pieces, 2..4 = records):
// union-find components, chi and beta0 per key, sorted unique keys unpacked
// to int32 rows, contractibility flags.  Outputs hold up to n (kind 1: ns)
// rows; *count (device) receives the number of keys.
struct FinalOut {
    int32_t* keys = nullptr;    // [count, kind]
    int32_t* chi = nullptr;
    int32_t* beta = nullptr;
    uint8_t* flag = nullptr;
    long long* count = nullptr;
};
// Scratch for up to ncap pieces (kind 1) or records (kinds 2..4); it must be
// cleared by launch_finalize_clear before launch_finalize (n <= ncap) runs.
size_t finalize_tmp_bytes(int kind, long long ncap, long long ns);
void launch_finalize_clear(int kind, long long ncap, long long ns, void* tmp, cudaStream_t s);
// Byte ranges to fill, cleared by one launch.
struct ClearList {
    void* p[16];
    long long bytes[16];
    int value[16];
    int n;
};
void finalize_clear_list(int kind, long long ncap, long long ns, void* tmp, ClearList& L);
void launch_clear(const ClearList& L, cudaStream_t s);
void launch_finalize(const ClipArgs& a, int kind, long long n, long long ncap, long long ns, int key_bits,
                     const FinalOut& out, void* tmp, cudaStream_t s);
// One launch copying n_keys int32 key entries and n values of elem (1 or 4)
// bytes; a NULL source skips that part.
void launch_copy_rows(const int32_t* keys, int32_t* d_keys, long long n_keys, const void* vals, void* d_vals,
                      long long n, int elem, cudaStream_t s);
// One launch copying up to 16 segments (n elements of elem = 1 or 4 bytes
// each, source to destination).
struct ExportSeg {
    const void* src;
    void* dst;
    long long n;
    int elem;
};
struct ExportArgs {
    ExportSeg seg[16];
    int nseg;
};
void launch_export(const ExportArgs& a, cudaStream_t s);
void launch_compact_pieces(const ClipArgs& a, long long npairs, const int64_t* off, int32_t* d_tet,
                           int32_t* d_sphere, double* d_vol, double* d_mom, cudaStream_t s);

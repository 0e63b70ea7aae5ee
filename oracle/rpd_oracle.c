/*
 * Brute-force CPU oracle for the volumetric restricted power diagram
 * (TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline leg load this; the library never does).
 *
 * Follows the paper's definitions:
 *   - power distance pd(x,m_i) = |x - c_i|^2 - r_i^2 (Sec. 3.2, after Eq. 1);
 *   - power cell (Eq. 1), restricted cell RPC_i = cell_i cap shape (Eq. 2-3);
 *   - Tet-Cell strategy (Sec. 5.2): every (tet, sphere) pair is clipped on its
 *     own by the radical half-spaces {pd(x,i) <= pd(x,k)} (Sec. 4.1.2).  Here
 *     each tet is clipped against ALL other spheres (brute force);
 *   - restricted elements RPC/RPF/RPE/RPV (Sec. 3.2 list);
 *   - fractional Euler characteristic with inheritance of the weight of the
 *     carrying mesh face (Sec. 4.1.2, Eq. 7), reported both as 1/n weights
 *     (double) and with each shared mesh face owned by its lowest tet (int);
 *   - component links across shared tet faces (Sec. 4.1.1).
 *
 * Polytope representation: list of vertices, each with the three planes it
 * lies on and FP64 coordinates.  Plane ids 0..3 are the tet faces (face f is
 * opposite tet vertex f), 4+k is the radical plane of sphere k.
 *
 * Exactness: inputs are integers (grid units).  The side of a vertex w.r.t. a
 * plane h is sign(det4[P1;P2;P3;h]) * sign(det3[n1;n2;n3]) with the planes'
 * integer coefficients; it is decided in FP64 when |value| exceeds a generous
 * bound (2^-40 times the permanent) and otherwise in 256-bit integers.  Tet
 * corners are classified directly with exact 64-bit power distances.  A zero
 * sign means the input is not in generic position: the run stops with
 * ORC_DEGENERATE.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_NONMANIFOLD 2
#define ORC_DEGENERATE 3
#define ORC_OOM 4
#define ORC_OVERFLOW 6

#define MAXV 1024

typedef __int128 i128;

/* ------------------------------------------------------------ 256-bit ints */
typedef struct { uint64_t w[4]; } i256;

static i256 z_from128(i128 v) {
    i256 r;
    unsigned __int128 u = (unsigned __int128)v;
    r.w[0] = (uint64_t)u;
    r.w[1] = (uint64_t)(u >> 64);
    r.w[2] = r.w[3] = (v < 0) ? ~0ULL : 0ULL;
    return r;
}
static i256 z_add(i256 a, i256 b) {
    i256 r;
    unsigned __int128 c = 0;
    for (int k = 0; k < 4; k++) {
        c += (unsigned __int128)a.w[k] + b.w[k];
        r.w[k] = (uint64_t)c;
        c >>= 64;
    }
    return r;
}
static i256 z_neg(i256 a) {
    i256 r;
    for (int k = 0; k < 4; k++) r.w[k] = ~a.w[k];
    i256 one = {{1, 0, 0, 0}};
    return z_add(r, one);
}
static int z_sign(i256 a) {
    if (a.w[3] >> 63) return -1;
    return (a.w[0] | a.w[1] | a.w[2] | a.w[3]) ? 1 : 0;
}
static i256 z_mul(i256 a, i256 b) {
    int neg = 0;
    if (z_sign(a) < 0) { a = z_neg(a); neg ^= 1; }
    if (z_sign(b) < 0) { b = z_neg(b); neg ^= 1; }
    uint64_t r[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; i++) {
        unsigned __int128 c = 0;
        for (int j = 0; i + j < 4; j++) {
            c += (unsigned __int128)a.w[i] * b.w[j] + r[i + j];
            r[i + j] = (uint64_t)c;
            c >>= 64;
        }
    }
    i256 out = {{r[0], r[1], r[2], r[3]}};
    return neg ? z_neg(out) : out;
}
static i256 z_sub(i256 a, i256 b) { return z_add(a, z_neg(b)); }

/* ------------------------------------------------------------------ planes */
/* plane value h(x) = a.x + b in tet-local integer coordinates; a vertex is
 * kept by a clip when h < 0 there. */
typedef struct { i128 a[3]; i128 b; } plane_t;

static i256 det3_exact(const i128 m[3][3]) {
    i256 t0 = z_mul(z_from128(m[0][0]), z_from128(m[1][1] * m[2][2] - m[1][2] * m[2][1]));
    i256 t1 = z_mul(z_from128(m[0][1]), z_from128(m[1][0] * m[2][2] - m[1][2] * m[2][0]));
    i256 t2 = z_mul(z_from128(m[0][2]), z_from128(m[1][0] * m[2][1] - m[1][1] * m[2][0]));
    return z_add(z_sub(t0, t1), t2);
}

static double det3_d(const double m[3][3], double *perm) {
    double c0 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    double c1 = m[1][0] * m[2][2] - m[1][2] * m[2][0];
    double c2 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    if (perm) {
        double p0 = fabs(m[1][1] * m[2][2]) + fabs(m[1][2] * m[2][1]);
        double p1 = fabs(m[1][0] * m[2][2]) + fabs(m[1][2] * m[2][0]);
        double p2 = fabs(m[1][0] * m[2][1]) + fabs(m[1][1] * m[2][0]);
        *perm = fabs(m[0][0]) * p0 + fabs(m[0][1]) * p1 + fabs(m[0][2]) * p2;
    }
    return m[0][0] * c0 - m[0][1] * c1 + m[0][2] * c2;
}

/* sign of det3 of the normals of planes p,q,r */
static int normals_sign(const plane_t *p, const plane_t *q, const plane_t *r) {
    const plane_t *P[3] = {p, q, r};
    double md[3][3];
    i128 mi[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) { mi[i][j] = P[i]->a[j]; md[i][j] = (double)P[i]->a[j]; }
    double perm;
    double v = det3_d(md, &perm);
    double bound = perm * 0x1p-40;
    if (v > bound) return 1;
    if (v < -bound) return -1;
    return z_sign(det3_exact(mi));
}

/* sign of det4 [p; q; r; h] (rows (a, b)) */
static int det4_sign(const plane_t *p, const plane_t *q, const plane_t *r, const plane_t *h) {
    const plane_t *P[4] = {p, q, r, h};
    double v = 0, perm = 0;
    for (int skip = 0; skip < 4; skip++) {
        double md[3][3];
        int rr = 0;
        for (int i = 0; i < 4; i++) {
            if (i == skip) continue;
            for (int j = 0; j < 3; j++) md[rr][j] = (double)P[i]->a[j];
            rr++;
        }
        double pm;
        double d3 = det3_d(md, &pm);
        double bb = (double)P[skip]->b;
        double sgn = ((skip + 3) & 1) ? -1.0 : 1.0;
        v += sgn * bb * d3;
        perm += fabs(bb) * pm;
    }
    double bound = perm * 0x1p-40;
    if (v > bound) return 1;
    if (v < -bound) return -1;
    i256 acc = {{0, 0, 0, 0}};
    for (int skip = 0; skip < 4; skip++) {
        i128 mi[3][3];
        int rr = 0;
        for (int i = 0; i < 4; i++) {
            if (i == skip) continue;
            for (int j = 0; j < 3; j++) mi[rr][j] = P[i]->a[j];
            rr++;
        }
        i256 t = z_mul(z_from128(P[skip]->b), det3_exact(mi));
        acc = ((skip + 3) & 1) ? z_sub(acc, t) : z_add(acc, t);
    }
    return z_sign(acc);
}

/* -------------------------------------------------------------- polytope */
typedef struct {
    int pl[3];       /* plane ids */
    int nsign;       /* sign of det3 of the three normals (0 for a tet corner) */
    int corner;      /* tet corner index 0..3, or -1 */
    double x[3];     /* tet-local coordinates */
} vtx_t;

typedef struct {
    const int64_t *X;     /* nv x 3 */
    const int32_t *T;     /* nt x 4 */
    const int64_t *C;     /* ns x 3 */
    const int64_t *W;     /* ns (= r^2) */
    int64_t nv, nt, ns;
    /* per tet: owner bits (4 verts, 6 edges, 4 faces) and sharing counts */
    uint16_t *own;
    int32_t *nshare;      /* nt x 14 */
    int32_t *adj;         /* nt x 4 */
    const int32_t *subset;
    int64_t nsub;
    int nthreads;
    /* same-algorithm baseline only (K > 0): per mesh vertex the K nearest
     * spheres in power distance, their distances and the bound D+ */
    int K;
    int32_t *knn;
    int64_t *knd, *dplus;
} mesh_t;

typedef struct {
    /* pieces */
    int64_t np, cap_p;
    int32_t *p_t, *p_i;
    double *p_vol, *p_mom;
    /* element nodes */
    int64_t nn, cap_n;
    int32_t *n_kind, *n_key, *n_t, *n_own, *n_link;
    double *n_frac, *n_len;
    int status;
    int64_t ndeg;
    /* threading */
    const mesh_t *m;
    int64_t t_begin, t_end, t_stride;
} out_t;

static int grow_p(out_t *o) {
    if (o->np < o->cap_p) return 1;
    int64_t c = o->cap_p ? o->cap_p * 2 : 1024;
    void *a = realloc(o->p_t, c * 4), *b = realloc(o->p_i, c * 4);
    void *d = realloc(o->p_vol, c * 8), *e = realloc(o->p_mom, c * 24);
    if (a) o->p_t = a; if (b) o->p_i = b; if (d) o->p_vol = d; if (e) o->p_mom = e;
    if (!a || !b || !d || !e) return 0;
    o->cap_p = c;
    return 1;
}
static int grow_n(out_t *o) {
    if (o->nn < o->cap_n) return 1;
    int64_t c = o->cap_n ? o->cap_n * 2 : 4096;
    void *a = realloc(o->n_kind, c * 4), *b = realloc(o->n_key, c * 16), *d = realloc(o->n_t, c * 4);
    void *e = realloc(o->n_own, c * 4), *f = realloc(o->n_link, c * 4), *g = realloc(o->n_frac, c * 8);
    void *hl = realloc(o->n_len, c * 8);
    if (hl) o->n_len = hl;
    if (a) o->n_kind = a; if (b) o->n_key = b; if (d) o->n_t = d;
    if (e) o->n_own = e; if (f) o->n_link = f; if (g) o->n_frac = g;
    if (!a || !b || !d || !e || !f || !g || !hl) return 0;
    o->cap_n = c;
    return 1;
}

static int64_t pd64(const int64_t *x, const int64_t *c, int64_t w) {
    int64_t d0 = x[0] - c[0], d1 = x[1] - c[1], d2 = x[2] - c[2];
    return d0 * d0 + d1 * d1 + d2 * d2 - w;
}

/* local edge index of tet vertices (a,b), a != b */
static int edge_index(int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    static const int tab[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};
    return tab[a][b];
}

/* carrier slot (0..3 vertex, 4..9 edge, 10..13 face) of a plane subset; -1 = tet interior */
static int carrier_slot(const int *pl, int n) {
    int faces[3], nf = 0;
    for (int k = 0; k < n; k++) if (pl[k] < 4) faces[nf++] = pl[k];
    if (nf == 0) return -1;
    if (nf == 1) return 10 + faces[0];
    if (nf == 2) {
        int v[2], nvv = 0;
        for (int c = 0; c < 4; c++) if (c != faces[0] && c != faces[1]) v[nvv++] = c;
        return 4 + edge_index(v[0], v[1]);
    }
    return 6 - faces[0] - faces[1] - faces[2];
}

static int has(const int *pl, int p) { return pl[0] == p || pl[1] == p || pl[2] == p; }

/* Fan-triangulated volume and first moment (tet-local coordinates). */
static void vol_moment(const vtx_t *V, int nvx, double *vol, double mom[3]) {
    *vol = 0; mom[0] = mom[1] = mom[2] = 0;
    const double *ap = V[0].x;
    int planes[MAXV], np = 0;
    for (int v = 0; v < nvx; v++)
        for (int k = 0; k < 3; k++) {
            int p = V[v].pl[k], seen = 0;
            for (int q = 0; q < np; q++) if (planes[q] == p) { seen = 1; break; }
            if (!seen) planes[np++] = p;
        }
    int ring[MAXV];
    for (int q = 0; q < np; q++) {
        int p = planes[q];
        if (has(V[0].pl, p)) continue;
        int fv[MAXV], nfv = 0;
        for (int v = 0; v < nvx; v++) if (has(V[v].pl, p)) fv[nfv++] = v;
        /* walk the face cycle: neighbours share p and one more plane */
        int used[MAXV];
        memset(used, 0, sizeof(int) * nfv);
        ring[0] = fv[0]; used[0] = 1;
        int len = 1;
        while (len < nfv) {
            int cur = ring[len - 1], nxt = -1;
            for (int s = 0; s < nfv && nxt < 0; s++) {
                if (used[s]) continue;
                int common = 0;
                for (int a = 0; a < 3; a++) if (has(V[fv[s]].pl, V[cur].pl[a])) common++;
                if (common == 2) { nxt = s; }
            }
            if (nxt < 0) break;
            used[nxt] = 1;
            ring[len++] = fv[nxt];
        }
        for (int s = 1; s + 1 < len; s++) {
            const double *b = V[ring[0]].x, *c = V[ring[s]].x, *d = V[ring[s + 1]].x;
            double u[3] = {b[0] - ap[0], b[1] - ap[1], b[2] - ap[2]};
            double vv[3] = {c[0] - ap[0], c[1] - ap[1], c[2] - ap[2]};
            double w[3] = {d[0] - ap[0], d[1] - ap[1], d[2] - ap[2]};
            double det = u[0] * (vv[1] * w[2] - vv[2] * w[1]) - u[1] * (vv[0] * w[2] - vv[2] * w[0]) +
                         u[2] * (vv[0] * w[1] - vv[1] * w[0]);
            double tv = fabs(det) / 6.0;
            *vol += tv;
            for (int k = 0; k < 3; k++) mom[k] += tv * (ap[k] + b[k] + c[k] + d[k]) * 0.25;
        }
    }
}

typedef struct { int64_t d; int32_t k; } sortkey_t;
static int cmp_sk(const void *a, const void *b) {
    const sortkey_t *x = a, *y = b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    return x->k < y->k ? -1 : (x->k > y->k);
}

/* Clip tet t against the spheres of `cand` (ncand ids, ascending), or against
 * every sphere when cand is NULL (the brute force). */
static void process_tet(out_t *o, int64_t t, sortkey_t *order, vtx_t *V, vtx_t *V2, plane_t *bis,
                        const int32_t *cand, int64_t ncand) {
    const mesh_t *m = o->m;
    int64_t X[4][3];
    for (int a = 0; a < 4; a++)
        for (int k = 0; k < 3; k++) X[a][k] = m->X[(int64_t)m->T[t * 4 + a] * 3 + k];
    const int64_t *O = X[0];
    int64_t L[4][3];
    for (int a = 0; a < 4; a++)
        for (int k = 0; k < 3; k++) L[a][k] = X[a][k] - O[k];
    /* tet face planes, oriented so the opposite corner has h < 0 */
    plane_t F[4];
    for (int f = 0; f < 4; f++) {
        int v[3], n = 0;
        for (int c = 0; c < 4; c++) if (c != f) v[n++] = c;
        i128 e1[3], e2[3], nn[3];
        for (int k = 0; k < 3; k++) { e1[k] = L[v[1]][k] - L[v[0]][k]; e2[k] = L[v[2]][k] - L[v[0]][k]; }
        nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
        i128 s = 0, off = 0;
        for (int k = 0; k < 3; k++) { s += nn[k] * (L[f][k] - L[v[0]][k]); off += nn[k] * L[v[0]][k]; }
        int sg = s > 0 ? 1 : -1;
        /* inside iff sg * n.(x - p0) > 0  <=>  h = -sg*n.x + sg*n.p0 < 0 */
        for (int k = 0; k < 3; k++) F[f].a[k] = -sg * nn[k];
        F[f].b = sg * off;
    }
    /* spheres by power distance at the centroid (order only affects speed) */
    double cen[3];
    for (int k = 0; k < 3; k++) cen[k] = 0.25 * (double)(X[0][k] + X[1][k] + X[2][k] + X[3][k]);
    int64_t ns = cand ? ncand : m->ns;
    for (int64_t q0 = 0; q0 < ns; q0++) {
        int64_t s = cand ? cand[q0] : q0;
        double d = 0;
        for (int k = 0; k < 3; k++) { double q = cen[k] - (double)m->C[s * 3 + k]; d += q * q; }
        order[q0].d = (int64_t)llround(d - (double)m->W[s]);
        order[q0].k = (int32_t)s;
    }
    qsort(order, ns, sizeof(sortkey_t), cmp_sk);
    /* exact power distances of the corners */
    for (int64_t ii = 0; ii < ns; ii++) {
        const int64_t i = cand ? cand[ii] : ii;
        int nvx = 4;
        for (int a = 0; a < 4; a++) {
            int n = 0;
            for (int f = 0; f < 4; f++) if (f != a) V[a].pl[n++] = f;
            V[a].nsign = 0;
            V[a].corner = a;
            for (int k = 0; k < 3; k++) V[a].x[k] = (double)L[a][k];
        }
        int ci_[3];
        const int64_t *ci = m->C + i * 3;
        int64_t pdi[4];
        for (int a = 0; a < 4; a++) pdi[a] = pd64(X[a], ci, m->W[i]);
        (void)ci_;
        int alive = 1;
        for (int64_t r = 0; r < ns && alive; r++) {
            int64_t k = order[r].k;
            if (k == i) continue;
            const int64_t *ck = m->C + k * 3;
            /* radical plane h(x) = pd(x,i) - pd(x,k) in local coordinates */
            plane_t *H = &bis[k];
            int64_t cil[3], ckl[3];
            for (int q = 0; q < 3; q++) { cil[q] = ci[q] - O[q]; ckl[q] = ck[q] - O[q]; }
            for (int q = 0; q < 3; q++) H->a[q] = 2 * (i128)(ckl[q] - cil[q]);
            i128 pi = (i128)cil[0] * cil[0] + (i128)cil[1] * cil[1] + (i128)cil[2] * cil[2] - m->W[i];
            i128 pk = (i128)ckl[0] * ckl[0] + (i128)ckl[1] * ckl[1] + (i128)ckl[2] * ckl[2] - m->W[k];
            H->b = pi - pk;
            int side[MAXV], nin = 0, nout = 0;
            for (int v = 0; v < nvx; v++) {
                int s;
                if (V[v].corner >= 0) {
                    int64_t hv = pdi[V[v].corner] - pd64(X[V[v].corner], ck, m->W[k]);
                    s = (hv > 0) - (hv < 0);
                } else {
                    const plane_t *P[3];
                    for (int q = 0; q < 3; q++) P[q] = V[v].pl[q] < 4 ? &F[V[v].pl[q]] : &bis[V[v].pl[q] - 4];
                    s = det4_sign(P[0], P[1], P[2], H) * V[v].nsign;
                }
                if (s == 0) { o->status = ORC_DEGENERATE; o->ndeg++; return; }
                side[v] = s;
                if (s < 0) nin++; else nout++;
            }
            if (nout == 0) continue;
            if (nin == 0) { alive = 0; break; }
            int n2 = 0;
            for (int v = 0; v < nvx; v++) if (side[v] < 0) V2[n2++] = V[v];
            for (int u = 0; u < nvx; u++) {
                if (side[u] > 0) continue;
                for (int w = 0; w < nvx; w++) {
                    if (side[w] < 0) continue;
                    int cm[3], nc = 0;
                    for (int q = 0; q < 3; q++) if (has(V[w].pl, V[u].pl[q])) cm[nc++] = V[u].pl[q];
                    if (nc != 2) continue;
                    if (n2 >= MAXV) { o->status = ORC_OVERFLOW; return; }
                    vtx_t *nw = &V2[n2++];
                    nw->pl[0] = cm[0]; nw->pl[1] = cm[1]; nw->pl[2] = 4 + (int)k;
                    nw->corner = -1;
                    const plane_t *P[3];
                    for (int q = 0; q < 3; q++) P[q] = nw->pl[q] < 4 ? &F[nw->pl[q]] : &bis[nw->pl[q] - 4];
                    nw->nsign = normals_sign(P[0], P[1], P[2]);
                    if (nw->nsign == 0) { o->status = ORC_DEGENERATE; o->ndeg++; return; }
                    /* Cramer: x = -(b0 (a1 x a2) + b1 (a2 x a0) + b2 (a0 x a1)) / det */
                    double A[3][3], B[3];
                    for (int q = 0; q < 3; q++) {
                        for (int j = 0; j < 3; j++) A[q][j] = (double)P[q]->a[j];
                        B[q] = (double)P[q]->b;
                    }
                    double det = det3_d(A, NULL);
                    double c12[3] = {A[1][1] * A[2][2] - A[1][2] * A[2][1], A[1][2] * A[2][0] - A[1][0] * A[2][2],
                                     A[1][0] * A[2][1] - A[1][1] * A[2][0]};
                    double c20[3] = {A[2][1] * A[0][2] - A[2][2] * A[0][1], A[2][2] * A[0][0] - A[2][0] * A[0][2],
                                     A[2][0] * A[0][1] - A[2][1] * A[0][0]};
                    double c01[3] = {A[0][1] * A[1][2] - A[0][2] * A[1][1], A[0][2] * A[1][0] - A[0][0] * A[1][2],
                                     A[0][0] * A[1][1] - A[0][1] * A[1][0]};
                    for (int j = 0; j < 3; j++) nw->x[j] = -(B[0] * c12[j] + B[1] * c20[j] + B[2] * c01[j]) / det;
                }
            }
            memcpy(V, V2, sizeof(vtx_t) * n2);
            nvx = n2;
        }
        if (!alive || nvx < 4) continue;
        /* ---- piece output */
        double vol, mom[3];
        vol_moment(V, nvx, &vol, mom);
        if (!grow_p(o)) { o->status = ORC_OOM; return; }
        o->p_t[o->np] = (int32_t)t;
        o->p_i[o->np] = (int32_t)i;
        o->p_vol[o->np] = vol;
        for (int k = 0; k < 3; k++) o->p_mom[o->np * 3 + k] = mom[k] + vol * (double)O[k];
        o->np++;
        /* ---- elements: faces of the simple polytope are subsets of vertex plane sets */
        /* element J (set of radical planes) with i < min(J); chi = sum over faces Q > J */
        int bp[MAXV], nb = 0;
        for (int v = 0; v < nvx; v++)
            for (int q = 0; q < 3; q++) {
                int p = V[v].pl[q];
                if (p < 4) continue;
                int seen = 0;
                for (int z = 0; z < nb; z++) if (bp[z] == p) { seen = 1; break; }
                if (!seen) bp[nb++] = p;
            }
        /* enumerate candidate J: empty, singles, pairs, triples that occur in some vertex */
        int Jl[4 * MAXV][3], Jn[4 * MAXV], nJ = 0;
        Jn[nJ++] = 0;
        for (int v = 0; v < nvx; v++) {
            int b3[3], n3 = 0;
            for (int q = 0; q < 3; q++) if (V[v].pl[q] >= 4) b3[n3++] = V[v].pl[q];
            /* all nonempty subsets of b3 */
            for (int mask = 1; mask < (1 << n3); mask++) {
                int s[3], ns_ = 0;
                for (int q = 0; q < n3; q++) if (mask & (1 << q)) s[ns_++] = b3[q];
                /* sort */
                for (int a = 0; a < ns_; a++)
                    for (int b = a + 1; b < ns_; b++) if (s[b] < s[a]) { int tt = s[a]; s[a] = s[b]; s[b] = tt; }
                int dup = 0;
                for (int z = 0; z < nJ && !dup; z++) {
                    if (Jn[z] != ns_) continue;
                    int eq = 1;
                    for (int q = 0; q < ns_; q++) if (Jl[z][q] != s[q]) eq = 0;
                    dup = eq;
                }
                if (!dup) {
                    for (int q = 0; q < ns_; q++) Jl[nJ][q] = s[q];
                    Jn[nJ++] = ns_;
                }
            }
        }
        const uint16_t own = m->own[t];
        const int32_t *nsh = m->nshare + t * 14;
        for (int z = 0; z < nJ; z++) {
            int nj = Jn[z];
            if (nj > 0 && Jl[z][0] - 4 < i) continue;  /* emitted by the lowest sphere */
            /* faces Q containing J: enumerate vertices (3-sets), edges (2-sets), faces (1-sets), cell */
            int chi_own = 0;
            double chi_frac = 0;
            /* distinct Q of each size that contain J */
            int Qs[3 * MAXV][3], nQ = 0, Qsz[3 * MAXV];
            for (int v = 0; v < nvx; v++) {
                int ok = 1;
                for (int q = 0; q < nj; q++) if (!has(V[v].pl, Jl[z][q])) ok = 0;
                if (!ok) continue;
                for (int mask = 1; mask < 8; mask++) {
                    int s[3], sz = 0;
                    for (int q = 0; q < 3; q++) if (mask & (1 << q)) s[sz++] = V[v].pl[q];
                    /* must contain J */
                    int cj = 1;
                    for (int q = 0; q < nj; q++) {
                        int f = 0;
                        for (int a = 0; a < sz; a++) if (s[a] == Jl[z][q]) f = 1;
                        if (!f) cj = 0;
                    }
                    if (!cj) continue;
                    for (int a = 0; a < sz; a++)
                        for (int b = a + 1; b < sz; b++) if (s[b] < s[a]) { int tt = s[a]; s[a] = s[b]; s[b] = tt; }
                    int dup = 0;
                    for (int y = 0; y < nQ && !dup; y++) {
                        if (Qsz[y] != sz) continue;
                        int eq = 1;
                        for (int a = 0; a < sz; a++) if (Qs[y][a] != s[a]) eq = 0;
                        dup = eq;
                    }
                    if (!dup) { for (int a = 0; a < sz; a++) Qs[nQ][a] = s[a]; Qsz[nQ++] = sz; }
                }
            }
            /* the element itself when J is empty (the cell, dim 3, sign -1, weight 1) */
            if (nj == 0) { chi_own -= 1; chi_frac -= 1.0; }
            for (int y = 0; y < nQ; y++) {
                int sz = Qsz[y];
                int sgn = (sz == 3) ? 1 : (sz == 2 ? -1 : 1);  /* (-1)^(3-|Q|): dim 0:+, 1:-, 2:+ */
                int slot = carrier_slot(Qs[y], sz);
                int w_own = slot < 0 ? 1 : ((own >> slot) & 1);
                double w_frac = slot < 0 ? 1.0 : 1.0 / (double)nsh[slot];
                chi_own += sgn * w_own;
                chi_frac += sgn * w_frac;
            }
            /* links across tet faces f: J u {f} is a face of the piece */
            int link = 0;
            for (int f = 0; f < 4; f++) {
                if (m->adj[t * 4 + f] < 0) continue;
                int found = 0;
                for (int v = 0; v < nvx && !found; v++) {
                    if (!has(V[v].pl, f)) continue;
                    int ok = 1;
                    for (int q = 0; q < nj; q++) if (!has(V[v].pl, Jl[z][q])) ok = 0;
                    found = ok;
                }
                if (found) link |= 1 << f;
            }
            if (!grow_n(o)) { o->status = ORC_OOM; return; }
            int64_t n = o->nn++;
            o->n_kind[n] = nj + 1;
            o->n_key[n * 4 + 0] = (int32_t)i;
            for (int q = 0; q < 3; q++) o->n_key[n * 4 + 1 + q] = q < nj ? Jl[z][q] - 4 : -1;
            o->n_t[n] = (int32_t)t;
            o->n_own[n] = chi_own;
            o->n_frac[n] = chi_frac;
            o->n_link[n] = link;
            /* an edge element (two radical planes): its segment's length,
             * between the two piece vertices on both planes (grid units) */
            double seg = 0;
            if (nj == 2) {
                int ends[2], ne_ = 0;
                for (int v = 0; v < nvx && ne_ < 2; v++)
                    if (has(V[v].pl, Jl[z][0]) && has(V[v].pl, Jl[z][1])) ends[ne_++] = v;
                if (ne_ == 2) {
                    double d2 = 0;
                    for (int k = 0; k < 3; k++) {
                        double d = V[ends[0]].x[k] - V[ends[1]].x[k];
                        d2 += d * d;
                    }
                    seg = sqrt(d2);
                }
            }
            o->n_len[n] = seg;
        }
    }
}

/* ------------------------------------------- same-algorithm CPU baseline
 * Timed baseline of the benchmark, not a parity reference (a CPU test checks
 * that its pieces and elements equal the brute force's).  It follows the
 * neighbour and candidate algorithm of the GPU library, written here in plain
 * C from the same argument, with no code in common:
 *   - per mesh vertex x: the K spheres of smallest power distance pd(x, m)
 *     (exact 64-bit integers), found by a ring search over a uniform grid of
 *     sphere centres, and D+(x), a lower bound on pd(x, m) of every sphere m
 *     left out of the list;
 *   - per tet with corners x_a: if sphere i owns part of the tet then, for
 *     every sphere j, some corner has pd(x_a, i) <= pd(x_a, j), because
 *     pd(., i) - pd(., j) is affine.  With j = o_b, the nearest sphere of
 *     corner b, i lies in G = union over a of {m : pd(x_a, m) <= pd(x_a, o_b)},
 *     read from the lists when every list covers its threshold (D+(x_a) >
 *     pd(x_a, o_b)), else from a scan of all spheres;
 *   - G is filtered by the same corner test against every other member, and
 *     each remaining candidate is clipped by the other candidates' radical
 *     planes (process_tet), which gives the same pieces as clipping against
 *     every sphere. */
typedef struct {
    int64_t org[3], cell;
    int64_t dim[3];
    int64_t *start;   /* ncell + 1 */
    int32_t *ids;     /* sphere ids sorted by cell */
    int64_t wmax;
} sgrid_t;

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int64_t cell_coord(const sgrid_t *g, int a, int64_t x) {
    int64_t d = x - g->org[a];
    int64_t q = d >= 0 ? d / g->cell : -((-d + g->cell - 1) / g->cell);
    return clampi(q, 0, g->dim[a] - 1);
}

static int build_sgrid(const mesh_t *m, sgrid_t *g) {
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
    g->wmax = 0;
    for (int64_t s = 0; s < m->ns; s++) {
        for (int a = 0; a < 3; a++) {
            int64_t v = m->C[s * 3 + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
        if (m->W[s] > g->wmax) g->wmax = m->W[s];
    }
    double vol = 1;
    for (int a = 0; a < 3; a++) vol *= (double)(hi[a] - lo[a] + 1);
    int64_t cell = (int64_t)ceil(cbrt(vol / (double)m->ns));
    if (cell < 1) cell = 1;
    g->cell = cell;
    int64_t ncell = 1;
    for (int a = 0; a < 3; a++) {
        g->org[a] = lo[a];
        g->dim[a] = (hi[a] - lo[a]) / cell + 1;
        ncell *= g->dim[a];
    }
    g->start = calloc(ncell + 1, sizeof(int64_t));
    g->ids = malloc(sizeof(int32_t) * (m->ns > 0 ? m->ns : 1));
    int64_t *fill = malloc(sizeof(int64_t) * ncell);
    int64_t *cid = malloc(sizeof(int64_t) * (m->ns > 0 ? m->ns : 1));
    if (!g->start || !g->ids || !fill || !cid) { free(fill); free(cid); return ORC_OOM; }
    for (int64_t s = 0; s < m->ns; s++) {
        int64_t c = 0;
        for (int a = 2; a >= 0; a--) c = c * g->dim[a] + cell_coord(g, a, m->C[s * 3 + a]);
        cid[s] = c;
        g->start[c + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) g->start[c + 1] += g->start[c];
    for (int64_t c = 0; c < ncell; c++) fill[c] = g->start[c];
    for (int64_t s = 0; s < m->ns; s++) g->ids[fill[cid[s]]++] = (int32_t)s;
    free(fill); free(cid);
    return ORC_OK;
}

/* K nearest spheres of point x (sorted by (distance, id)) and D+(x). */
static void knn_point(const mesh_t *m, const sgrid_t *g, const int64_t *x, int K, int32_t *ids, int64_t *dist,
                      int64_t *dplus) {
    int cnt = 0;
    int64_t c0[3];
    for (int a = 0; a < 3; a++) c0[a] = cell_coord(g, a, x[a]);
    for (int64_t r = 0;; r++) {
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; a++) { lo[a] = c0[a] - r; hi[a] = c0[a] + r; }
        for (int64_t cz = clampi(lo[2], 0, g->dim[2] - 1); cz <= clampi(hi[2], 0, g->dim[2] - 1); cz++)
            for (int64_t cy = clampi(lo[1], 0, g->dim[1] - 1); cy <= clampi(hi[1], 0, g->dim[1] - 1); cy++)
                for (int64_t cx = clampi(lo[0], 0, g->dim[0] - 1); cx <= clampi(hi[0], 0, g->dim[0] - 1); cx++) {
                    /* only the cells of ring r (Chebyshev distance r from c0) */
                    int64_t dx = cx - c0[0], dy = cy - c0[1], dz = cz - c0[2];
                    int64_t cheb = llabs(dx);
                    if (llabs(dy) > cheb) cheb = llabs(dy);
                    if (llabs(dz) > cheb) cheb = llabs(dz);
                    if (cheb != r) continue;
                    int64_t c = (cz * g->dim[1] + cy) * g->dim[0] + cx;
                    for (int64_t q = g->start[c]; q < g->start[c + 1]; q++) {
                        int32_t sid = g->ids[q];
                        int64_t d = pd64(x, m->C + (int64_t)sid * 3, m->W[sid]);
                        if (cnt == K && (d > dist[K - 1] || (d == dist[K - 1] && sid > ids[K - 1]))) continue;
                        int pos = cnt < K ? cnt++ : K - 1;
                        while (pos > 0 && (dist[pos - 1] > d || (dist[pos - 1] == d && ids[pos - 1] > sid))) {
                            dist[pos] = dist[pos - 1];
                            ids[pos] = ids[pos - 1];
                            pos--;
                        }
                        dist[pos] = d;
                        ids[pos] = sid;
                    }
                }
        /* spheres outside the box of rings <= r lie beyond one of its
         * unclamped faces: their centre is at least `gap` away from x */
        int64_t gap = INT64_MAX;
        for (int a = 0; a < 3; a++) {
            if (lo[a] > 0) {
                int64_t gl = x[a] - (g->org[a] + lo[a] * g->cell);
                if (gl < 0) gl = 0;
                if (gl < gap) gap = gl;
            }
            if (hi[a] < g->dim[a] - 1) {
                int64_t gh = g->org[a] + (hi[a] + 1) * g->cell - x[a];
                if (gh < 0) gh = 0;
                if (gh < gap) gap = gh;
            }
        }
        const int64_t kth = cnt == K ? dist[K - 1] : INT64_MAX;
        if (gap == INT64_MAX) {   /* every cell visited */
            *dplus = kth;
            break;
        }
        const int64_t lb = gap * gap - g->wmax;
        if (cnt == K && lb > kth) {
            *dplus = kth;   /* evicted spheres are >= the K-th; the rest >= lb > kth */
            break;
        }
    }
    for (int k = cnt; k < K; k++) { ids[k] = -1; dist[k] = INT64_MAX; }
}

typedef struct {
    const mesh_t *m;
    const sgrid_t *g;
    const uint8_t *need;
    int64_t v_begin, v_end;
} knn_job_t;

static void *knn_worker(void *arg) {
    knn_job_t *j = arg;
    const mesh_t *m = j->m;
    for (int64_t v = j->v_begin; v < j->v_end; v++)
        if (j->need[v])
            knn_point(m, j->g, m->X + v * 3, m->K, m->knn + v * m->K, m->knd + v * m->K, m->dplus + v);
    return NULL;
}

static int compute_knn(mesh_t *m) {
    sgrid_t g = {0};
    int st = build_sgrid(m, &g);
    uint8_t *need = calloc(m->nv, 1);
    m->knn = malloc(sizeof(int32_t) * m->nv * m->K);
    m->knd = malloc(sizeof(int64_t) * m->nv * m->K);
    m->dplus = malloc(sizeof(int64_t) * m->nv);
    if (st != ORC_OK || !need || !m->knn || !m->knd || !m->dplus) { free(g.start); free(g.ids); free(need); return ORC_OOM; }
    int64_t count = m->subset ? m->nsub : m->nt;
    for (int64_t q = 0; q < count; q++) {
        int64_t t = m->subset ? m->subset[q] : q;
        for (int a = 0; a < 4; a++) need[m->T[t * 4 + a]] = 1;
    }
    int nth = m->nthreads;
    knn_job_t *jobs = malloc(sizeof(knn_job_t) * nth);
    pthread_t *th = malloc(sizeof(pthread_t) * nth);
    for (int k = 0; k < nth; k++) {
        jobs[k].m = m; jobs[k].g = &g; jobs[k].need = need;
        jobs[k].v_begin = m->nv * k / nth;
        jobs[k].v_end = m->nv * (k + 1) / nth;
        pthread_create(&th[k], NULL, knn_worker, &jobs[k]);
    }
    for (int k = 0; k < nth; k++) pthread_join(th[k], NULL);
    free(jobs); free(th); free(need); free(g.start); free(g.ids);
    return ORC_OK;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Candidate spheres of tet t (ascending ids) into cand; returns their count. */
static int64_t tet_candidates(const mesh_t *m, int64_t t, int32_t *cand, int64_t *gath_pd) {
    const int K = m->K;
    const int64_t *X[4];
    int32_t v[4];
    for (int a = 0; a < 4; a++) { v[a] = m->T[t * 4 + a]; X[a] = m->X + (int64_t)v[a] * 3; }
    int64_t n = 0;
    int bsel = -1;
    int64_t tau[4];
    for (int b = 0; b < 4 && bsel < 0; b++) {
        const int32_t ob = m->knn[(int64_t)v[b] * K];
        int ok = 1;
        for (int a = 0; a < 4; a++) {
            tau[a] = pd64(X[a], m->C + (int64_t)ob * 3, m->W[ob]);
            if (!(tau[a] < m->dplus[v[a]])) ok = 0;
        }
        if (ok) bsel = b;
    }
    if (bsel >= 0) {
        for (int a = 0; a < 4; a++)
            for (int k = 0; k < K; k++) {
                const int32_t sid = m->knn[(int64_t)v[a] * K + k];
                if (sid < 0 || m->knd[(int64_t)v[a] * K + k] > tau[a]) break;
                int dup = 0;
                for (int64_t z = 0; z < n && !dup; z++) dup = cand[z] == sid;
                if (!dup) cand[n++] = sid;
            }
    } else {   /* lists do not cover the thresholds of any corner: scan every sphere */
        const int32_t o0 = m->knn[(int64_t)v[0] * K];
        for (int a = 0; a < 4; a++) tau[a] = pd64(X[a], m->C + (int64_t)o0 * 3, m->W[o0]);
        for (int64_t s = 0; s < m->ns; s++) {
            int in = 0;
            for (int a = 0; a < 4 && !in; a++) in = pd64(X[a], m->C + s * 3, m->W[s]) <= tau[a];
            if (in) cand[n++] = (int32_t)s;
        }
    }
    /* exact corner filter: i survives iff for every other j some corner has
     * pd(x_a, i) <= pd(x_a, j) */
    for (int64_t q = 0; q < n; q++)
        for (int a = 0; a < 4; a++) gath_pd[q * 4 + a] = pd64(X[a], m->C + (int64_t)cand[q] * 3, m->W[cand[q]]);
    int64_t keep = 0;
    for (int64_t q = 0; q < n; q++) {
        int ok = 1;
        for (int64_t r = 0; r < n && ok; r++) {
            if (r == q) continue;
            int some = 0;
            for (int a = 0; a < 4 && !some; a++) some = gath_pd[q * 4 + a] <= gath_pd[r * 4 + a];
            ok = some;
        }
        if (ok) cand[keep++] = cand[q];
    }
    qsort(cand, keep, sizeof(int32_t), cmp_i32);
    return keep;
}

static void *worker(void *arg) {
    out_t *o = arg;
    const mesh_t *m = o->m;
    sortkey_t *order = malloc(sizeof(sortkey_t) * (m->ns > 0 ? m->ns : 1));
    vtx_t *V = malloc(sizeof(vtx_t) * MAXV), *V2 = malloc(sizeof(vtx_t) * MAXV);
    plane_t *bis = malloc(sizeof(plane_t) * (m->ns > 0 ? m->ns : 1));
    int32_t *cand = m->K > 0 ? malloc(sizeof(int32_t) * (m->ns > 0 ? m->ns : 1)) : NULL;
    int64_t *gpd = m->K > 0 ? malloc(sizeof(int64_t) * 4 * (m->ns > 0 ? m->ns : 1)) : NULL;
    if (!order || !V || !V2 || !bis || (m->K > 0 && (!cand || !gpd))) { o->status = ORC_OOM; goto done; }
    for (int64_t s = o->t_begin; s < o->t_end && o->status == ORC_OK; s += o->t_stride) {
        int64_t t = m->subset ? m->subset[s] : s;
        if (m->K > 0) {
            const int64_t nc = tet_candidates(m, t, cand, gpd);
            process_tet(o, t, order, V, V2, bis, cand, nc);
        } else {
            process_tet(o, t, order, V, V2, bis, NULL, 0);
        }
    }
done:
    free(order); free(V); free(V2); free(bis); free(cand); free(gpd);
    return NULL;
}

/* ------------------------------------------------------------- mesh tables */
typedef struct { uint64_t key; int32_t t; int32_t slot; } kt_t;
static int cmp_kt(const void *a, const void *b) {
    const kt_t *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->t < y->t ? -1 : (x->t > y->t);
}

static int build_tables(mesh_t *m) {
    int64_t nt = m->nt, nv = m->nv;
    m->own = calloc(nt, sizeof(uint16_t));
    m->nshare = calloc(nt * 14, sizeof(int32_t));
    m->adj = malloc(nt * 4 * sizeof(int32_t));
    int32_t *vmin = malloc(nv * sizeof(int32_t)), *vcnt = calloc(nv, sizeof(int32_t));
    kt_t *E = malloc(nt * 6 * sizeof(kt_t)), *Fk = malloc(nt * 4 * sizeof(kt_t));
    if (!m->own || !m->nshare || !m->adj || !vmin || !vcnt || !E || !Fk) return ORC_OOM;
    for (int64_t v = 0; v < nv; v++) vmin[v] = INT32_MAX;
    for (int64_t t = 0; t < nt; t++)
        for (int a = 0; a < 4; a++) {
            int32_t v = m->T[t * 4 + a];
            if (v < 0 || v >= nv) return ORC_INVALID;
            vcnt[v]++;
            if (t < vmin[v]) vmin[v] = (int32_t)t;
        }
    static const int EL[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int64_t t = 0; t < nt; t++) {
        for (int a = 0; a < 4; a++) {
            int32_t v = m->T[t * 4 + a];
            m->nshare[t * 14 + a] = vcnt[v];
            if (vmin[v] == t) m->own[t] |= 1u << a;
        }
        for (int e = 0; e < 6; e++) {
            uint64_t a = (uint64_t)m->T[t * 4 + EL[e][0]], b = (uint64_t)m->T[t * 4 + EL[e][1]];
            if (a > b) { uint64_t s = a; a = b; b = s; }
            E[t * 6 + e].key = a * (uint64_t)nv + b;
            E[t * 6 + e].t = (int32_t)t;
            E[t * 6 + e].slot = e;
        }
        for (int f = 0; f < 4; f++) {
            uint64_t v[3];
            int n = 0;
            for (int c = 0; c < 4; c++) if (c != f) v[n++] = (uint64_t)m->T[t * 4 + c];
            for (int a = 0; a < 3; a++)
                for (int b = a + 1; b < 3; b++) if (v[b] < v[a]) { uint64_t s = v[a]; v[a] = v[b]; v[b] = s; }
            Fk[t * 4 + f].key = (v[0] * (uint64_t)nv + v[1]) * (uint64_t)nv + v[2];
            Fk[t * 4 + f].t = (int32_t)t;
            Fk[t * 4 + f].slot = f;
        }
    }
    qsort(E, nt * 6, sizeof(kt_t), cmp_kt);
    for (int64_t s = 0; s < nt * 6;) {
        int64_t e = s;
        while (e < nt * 6 && E[e].key == E[s].key) e++;
        for (int64_t q = s; q < e; q++) {
            m->nshare[(int64_t)E[q].t * 14 + 4 + E[q].slot] = (int32_t)(e - s);
            if (q == s) m->own[E[q].t] |= 1u << (4 + E[q].slot);
        }
        s = e;
    }
    qsort(Fk, nt * 4, sizeof(kt_t), cmp_kt);
    for (int64_t t = 0; t < nt * 4; t++) m->adj[t] = -1;
    for (int64_t s = 0; s < nt * 4;) {
        int64_t e = s;
        while (e < nt * 4 && Fk[e].key == Fk[s].key) e++;
        if (e - s > 2) return ORC_NONMANIFOLD;
        for (int64_t q = s; q < e; q++) {
            m->nshare[(int64_t)Fk[q].t * 14 + 10 + Fk[q].slot] = (int32_t)(e - s);
            if (q == s) m->own[Fk[q].t] |= 1u << (10 + Fk[q].slot);
        }
        if (e - s == 2) {
            m->adj[(int64_t)Fk[s].t * 4 + Fk[s].slot] = Fk[s + 1].t;
            m->adj[(int64_t)Fk[s + 1].t * 4 + Fk[s + 1].slot] = Fk[s].t;
        }
        s = e;
    }
    free(vmin); free(vcnt); free(E); free(Fk);
    return ORC_OK;
}

/* ------------------------------------------------------------- C interface */
typedef struct {
    int status;
    int64_t ndeg;
    int64_t np, nn;
    int32_t *p_t, *p_i;
    double *p_vol, *p_mom;
    int32_t *n_kind, *n_key, *n_t, *n_own, *n_link;
    double *n_frac, *n_len;
    int32_t *adj;
} orc_result;

static int check_orient(const mesh_t *m) {
    for (int64_t t = 0; t < m->nt; t++) {
        const int64_t *p[4];
        for (int a = 0; a < 4; a++) p[a] = m->X + (int64_t)m->T[t * 4 + a] * 3;
        i128 u[3], v[3], w[3];
        for (int k = 0; k < 3; k++) { u[k] = p[1][k] - p[0][k]; v[k] = p[2][k] - p[0][k]; w[k] = p[3][k] - p[0][k]; }
        i128 d = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
                 u[2] * (v[0] * w[1] - v[1] * w[0]);
        if (d <= 0) return ORC_INVALID;
    }
    return ORC_OK;
}

static orc_result *run_common(int64_t nv, const int64_t *X, int64_t nt, const int32_t *T, int64_t ns,
                              const int64_t *C, const int64_t *R, const int32_t *subset, int64_t nsub, int nthreads,
                              int K) {
    orc_result *res = calloc(1, sizeof(orc_result));
    if (!res) return NULL;
    mesh_t m = {0};
    m.X = X; m.T = T; m.C = C; m.nv = nv; m.nt = nt; m.ns = ns;
    m.subset = subset; m.nsub = nsub; m.nthreads = nthreads > 0 ? nthreads : 1;
    m.K = K;
    int64_t *W = malloc(sizeof(int64_t) * (ns > 0 ? ns : 1));
    for (int64_t s = 0; s < ns; s++) W[s] = R[s] * R[s];
    m.W = W;
    for (int64_t v = 0; v < nv * 3; v++)
        if (X[v] > (1 << 21) || X[v] < -(1 << 21)) { res->status = ORC_INVALID; free(W); return res; }
    for (int64_t s = 0; s < ns * 3; s++)
        if (C[s] > (1 << 21) || C[s] < -(1 << 21)) { res->status = ORC_INVALID; free(W); return res; }
    int st = check_orient(&m);
    if (st == ORC_OK) st = build_tables(&m);
    if (st == ORC_OK && K > 0) st = compute_knn(&m);
    if (st != ORC_OK) { res->status = st; free(W); free(m.knn); free(m.knd); free(m.dplus); return res; }
    int nth = m.nthreads;
    int64_t count = subset ? nsub : nt;
    out_t *outs = calloc(nth, sizeof(out_t));
    pthread_t *th = malloc(sizeof(pthread_t) * nth);
    for (int k = 0; k < nth; k++) {
        outs[k].m = &m;
        outs[k].t_begin = k;
        outs[k].t_end = count;
        outs[k].t_stride = nth;
        pthread_create(&th[k], NULL, worker, &outs[k]);
    }
    for (int k = 0; k < nth; k++) pthread_join(th[k], NULL);
    int64_t np = 0, nn = 0;
    for (int k = 0; k < nth; k++) {
        if (outs[k].status != ORC_OK && res->status == ORC_OK) res->status = outs[k].status;
        res->ndeg += outs[k].ndeg;
        np += outs[k].np;
        nn += outs[k].nn;
    }
    res->np = np; res->nn = nn;
    res->p_t = malloc(4 * (np + 1)); res->p_i = malloc(4 * (np + 1));
    res->p_vol = malloc(8 * (np + 1)); res->p_mom = malloc(24 * (np + 1));
    res->n_kind = malloc(4 * (nn + 1)); res->n_key = malloc(16 * (nn + 1)); res->n_t = malloc(4 * (nn + 1));
    res->n_own = malloc(4 * (nn + 1)); res->n_link = malloc(4 * (nn + 1)); res->n_frac = malloc(8 * (nn + 1));
    res->n_len = malloc(8 * (nn + 1));
    int64_t pp = 0, qq = 0;
    for (int k = 0; k < nth; k++) {
        out_t *o = &outs[k];
        memcpy(res->p_t + pp, o->p_t, 4 * o->np); memcpy(res->p_i + pp, o->p_i, 4 * o->np);
        memcpy(res->p_vol + pp, o->p_vol, 8 * o->np); memcpy(res->p_mom + pp * 3, o->p_mom, 24 * o->np);
        memcpy(res->n_kind + qq, o->n_kind, 4 * o->nn); memcpy(res->n_key + qq * 4, o->n_key, 16 * o->nn);
        memcpy(res->n_t + qq, o->n_t, 4 * o->nn); memcpy(res->n_own + qq, o->n_own, 4 * o->nn);
        memcpy(res->n_link + qq, o->n_link, 4 * o->nn); memcpy(res->n_frac + qq, o->n_frac, 8 * o->nn);
        memcpy(res->n_len + qq, o->n_len, 8 * o->nn);
        pp += o->np; qq += o->nn;
        free(o->p_t); free(o->p_i); free(o->p_vol); free(o->p_mom);
        free(o->n_kind); free(o->n_key); free(o->n_t); free(o->n_own); free(o->n_link); free(o->n_frac);
        free(o->n_len);
    }
    res->adj = m.adj;
    free(outs); free(th); free(W); free(m.own); free(m.nshare);
    free(m.knn); free(m.knd); free(m.dplus);
    return res;
}

/* Brute force: every tet clipped against every other sphere. */
orc_result *orc_run(int64_t nv, const int64_t *X, int64_t nt, const int32_t *T, int64_t ns,
                    const int64_t *C, const int64_t *R, const int32_t *subset, int64_t nsub, int nthreads) {
    return run_common(nv, X, nt, T, ns, C, R, subset, nsub, nthreads, 0);
}

/* Same-algorithm CPU baseline: K power neighbours per vertex, candidates per
 * tet, each candidate clipped by the other candidates (bench only). */
orc_result *orc_run_knn(int64_t nv, const int64_t *X, int64_t nt, const int32_t *T, int64_t ns,
                        const int64_t *C, const int64_t *R, const int32_t *subset, int64_t nsub, int nthreads,
                        int K) {
    if (K < 1) K = 1;
    return run_common(nv, X, nt, T, ns, C, R, subset, nsub, nthreads, K);
}

int orc_status(const orc_result *r) { return r ? r->status : ORC_OOM; }
int64_t orc_npieces(const orc_result *r) { return r->np; }
int64_t orc_nnodes(const orc_result *r) { return r->nn; }

void orc_copy(const orc_result *r, int32_t *p_t, int32_t *p_i, double *p_vol, double *p_mom, int32_t *n_kind,
              int32_t *n_key, int32_t *n_t, int32_t *n_own, int32_t *n_link, double *n_frac, int32_t *adj,
              int64_t nt, double *n_len) {
    if (n_len) memcpy(n_len, r->n_len, 8 * r->nn);
    memcpy(p_t, r->p_t, 4 * r->np); memcpy(p_i, r->p_i, 4 * r->np);
    memcpy(p_vol, r->p_vol, 8 * r->np); memcpy(p_mom, r->p_mom, 24 * r->np);
    memcpy(n_kind, r->n_kind, 4 * r->nn); memcpy(n_key, r->n_key, 16 * r->nn);
    memcpy(n_t, r->n_t, 4 * r->nn); memcpy(n_own, r->n_own, 4 * r->nn);
    memcpy(n_link, r->n_link, 4 * r->nn); memcpy(n_frac, r->n_frac, 8 * r->nn);
    if (adj && r->adj) memcpy(adj, r->adj, 16 * nt);
}

void orc_free(orc_result *r) {
    if (!r) return;
    free(r->p_t); free(r->p_i); free(r->p_vol); free(r->p_mom);
    free(r->n_kind); free(r->n_key); free(r->n_t); free(r->n_own); free(r->n_link); free(r->n_frac);
    free(r->n_len);
    free(r->adj);
    free(r);
}

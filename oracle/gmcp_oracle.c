/*
 * gmcp_oracle.c -- plain, slow, FP64 CPU oracle of the GMCP contact pass.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA library against a direct
 * transcription of the method.  It shares no code, header or table with the
 * CUDA sources.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (see oracle/oracle.py).
 * -ffp-contract=off keeps every product and sum separately rounded, so the
 * decision predicates (candidate boxes, CCD) have a fixed meaning.
 *
 * What each part follows (paper: IsaacIPC / GMCP, arXiv 2605.24339):
 *   face samples ............ Sec. 4.1 "Face samples", Eq. (gap); fixed
 *                              slave-side centroid rule (reading R1); the
 *                              paper's clipped-polygon rule separately
 *                              (orc_face_clip_samples, reading R18)
 *   edge samples ............ Sec. 4.1 "Edge samples", Eqs. (edge_pos, gap_edge)
 *   point samples ........... Sec. 4.1 "Point samples"
 *   barycentric projection .. Sec. 3.2, Eq. (gram)
 *   potential ............... Sec. 4.2, Eq. (gmcp_potential); B from IPC
 *   gradient / Hessian ...... Sec. 4.2 (approximation with per-sample PSD clamp)
 *   gamma ................... Sec. 4.3, Eqs. (smoothstep, gamma)
 *   support radius .......... Sec. 4.4, Eq. (adaptive_eps)
 *   master rows ............. Sec. 4.3 with Eq. (gap): gradient with respect
 *                              to the master vertices (orc_master_grad) and
 *                              the blocks with master vertices (orc_master_hess)
 *   linearised step ......... Sec. 4.5, Eqs. (ccd, global_ccd)
 *   additive CCD ............ Li, Kaufman, Jiang 2021 (Codimensional IPC), Alg. 1
 *   Newton step ............. IPC problem statement, Sec. 2.1: minimise
 *                              inertia + elastic + contact over x with an
 *                              intersection-free line search
 *   dual-mesh mapper ........ Sec. 3.2, Eqs. (bary_proj), (decomp), (gram),
 *                              (bary_interp); nearest triangle by brute force
 *   warm-start MLP .......... not in the paper (a plain 4-layer perceptron)
 *
 * Parity pins live in tests/test_oracle_*.py.  The sample weights, the
 * smoothing factors gamma of faces and edges, the edge Gauss points and the
 * support radius of each sample kind are pinned by hand-worked closed forms
 * (tests/test_oracle_closed_forms.py, derivations in tests/golden/); the
 * derivatives by finite differences; candidates by brute force; CCD by
 * analytic times of impact.  Parts with no pin other than self-consistency
 * would be marked "parity unpinned" below: none at present.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* small vector helpers (every operation rounded separately)                 */
/* ------------------------------------------------------------------------- */
static void sub3(const double* a, const double* b, double* o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* ------------------------------------------------------------------------- */
/* Eq. (smoothstep): C1 Hermite step                                         */
/* ------------------------------------------------------------------------- */
ORC_API double orc_hermite(double x, double delta) {
    if (x <= 0.0) return 0.0;
    if (x >= delta) return 1.0;
    double t = x / delta;
    return 3.0 * t * t - 2.0 * t * t * t;
}

/* IPC log barrier B(g,eps) = -(g-eps)^2 ln(g/eps) on (0,eps), 0 for g>=eps,
 * +inf for g<=0 (Sec. 4.2: "B follows IPC"), with its first two derivatives. */
ORC_API void orc_barrier(double g, double eps, double* B, double* dB, double* d2B) {
    if (g >= eps) { *B = 0.0; *dB = 0.0; *d2B = 0.0; return; }
    if (g <= 0.0) { *B = INFINITY; *dB = -INFINITY; *d2B = INFINITY; return; }
    double d = g - eps;
    double L = log(g / eps);
    *B = -d * d * L;
    *dB = -2.0 * d * L - d * d / g;
    *d2B = -2.0 * L - 4.0 * d / g + d * d / (g * g);
}

/* Face-sample rule (reading R1): the 4^L sub-triangles of the uniform
 * midpoint subdivision of the slave triangle, one sample at each centroid,
 * weight 1/4^L.  With n = 2^L: upright cells (i,j,k), i+j+k = n-1, centroid
 * ((3i+1),(3j+1),(3k+1))/(3n); inverted cells i+j+k = n-2, centroid
 * ((3i+2),(3j+2),(3k+2))/(3n).  Returns the count. */
ORC_API int orc_face_rule(int L, double* beta) {
    int n = 1 << L, c = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; i + j < n; ++j) {
            int k = n - 1 - i - j;
            beta[3 * c + 0] = (double)(3 * i + 1) / (double)(3 * n);
            beta[3 * c + 1] = (double)(3 * j + 1) / (double)(3 * n);
            beta[3 * c + 2] = (double)(3 * k + 1) / (double)(3 * n);
            ++c;
        }
    for (int i = 0; i < n - 1; ++i)
        for (int j = 0; i + j < n - 1; ++j) {
            int k = n - 2 - i - j;
            beta[3 * c + 0] = (double)(3 * i + 2) / (double)(3 * n);
            beta[3 * c + 1] = (double)(3 * j + 2) / (double)(3 * n);
            beta[3 * c + 2] = (double)(3 * k + 2) / (double)(3 * n);
            ++c;
        }
    return c;
}

/* Eq. (gram): barycentric coordinates of the projection of q onto the plane
 * of (p0,p1,p2): solve the 2x2 Gram system for (v,w), u = 1-v-w. */
static void bary_gram(const double* q, const double* p0, const double* p1,
                      const double* p2, double* b) {
    double e1[3], e2[3], d[3];
    sub3(p1, p0, e1); sub3(p2, p0, e2); sub3(q, p0, d);
    double a = dot3(e1, e1), bb = dot3(e1, e2), c = dot3(e2, e2);
    double r1 = dot3(d, e1), r2 = dot3(d, e2);
    double det = a * c - bb * bb;
    double v = (c * r1 - bb * r2) / det;
    double w = (a * r2 - bb * r1) / det;
    b[0] = 1.0 - v - w; b[1] = v; b[2] = w;
}

static double min3(const double* b) { return dmin(b[0], dmin(b[1], b[2])); }

/* unit normal and area of a triangle */
static void tri_normal_area(const double* x0, const double* x1, const double* x2,
                            double* n, double* area) {
    double e1[3], e2[3], c[3];
    sub3(x1, x0, e1); sub3(x2, x0, e2); cross3(e1, e2, c);
    double len = sqrt(dot3(c, c));
    n[0] = c[0] / len; n[1] = c[1] / len; n[2] = c[2] / len;
    *area = 0.5 * len;
}

/* sample position ((b0 x0 + b1 x1) + b2 x2), unfused */
static void interp3(const double* b, const double* x0, const double* x1,
                    const double* x2, double* o) {
    for (int c = 0; c < 3; ++c) o[c] = b[0] * x0[c] + b[1] * x1[c] + b[2] * x2[c];
}

/* ------------------------------------------------------------------------- */
/* scene and derived topology                                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n_env;
    const int64_t *env_vert_off, *env_stri_off, *env_mvert_off, *env_mtri_off;
    int nv, ns, nmv, nmt;
    const double* X;       /* pad rest [nv][3] */
    const int32_t* stri;   /* [ns][3] */
    const double* Y0;      /* master positions at t=0 [nmv][3] */
    const int32_t* mtri;   /* [nmt][3] */
    double dhat, kappa, kappa_edge, kappa_point, delta_T, delta_e;
    int L;
    /* derived: master edges (sorted unique (a<b)), edge->tri CSR, vert->tri CSR */
    int nme;
    int32_t* medge;        /* [nme][2] */
    int32_t *me_tri_off, *me_tri;
    int32_t *mv_tri_off, *mv_tri;
    int32_t* stri_env;     /* env of each slave tri */
    int32_t* mtri_env;
    int32_t* medge_env;
    int32_t* mvert_env;
    int nk; double* rule;  /* face rule barycentrics [nk][3] */
    int all_pairs;         /* 1: skip the broad phase and test every pair */
    double dhat_guard, kappa_guard;  /* primitive guard barrier (0: off) */
    int face_clip;         /* 1: the paper's clipped-overlap face samples (reading R20) */
    int nsv, nse;
    int32_t* svert;        /* unique slave surface vertices */
    int32_t* sedge;        /* unique slave edges [nse][2] */
} orc_scene;

static int cmp_pair(const void* a, const void* b) {
    const int32_t* x = (const int32_t*)a; const int32_t* y = (const int32_t*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}
static int cmp_triple(const void* a, const void* b) {
    const int32_t* x = (const int32_t*)a; const int32_t* y = (const int32_t*)b;
    for (int i = 0; i < 3; ++i) if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

static int32_t env_of(const int64_t* off, int n_env, int64_t i) {
    int lo = 0, hi = n_env - 1;
    while (lo < hi) { int mid = (lo + hi + 1) / 2; if (off[mid] <= i) lo = mid; else hi = mid - 1; }
    return lo;
}

ORC_API orc_scene* orc_scene_create(int n_env, const int64_t* env_vert_off,
                                    const int64_t* env_stri_off, const int64_t* env_mvert_off,
                                    const int64_t* env_mtri_off, int nv, const double* X,
                                    int ns, const int32_t* stri, int nmv, const double* Y0,
                                    int nmt, const int32_t* mtri, double dhat, double kappa,
                                    double kappa_edge, double kappa_point, double delta_T,
                                    double delta_e, int L) {
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    s->n_env = n_env; s->env_vert_off = env_vert_off; s->env_stri_off = env_stri_off;
    s->env_mvert_off = env_mvert_off; s->env_mtri_off = env_mtri_off;
    s->nv = nv; s->X = X; s->ns = ns; s->stri = stri; s->nmv = nmv; s->Y0 = Y0;
    s->nmt = nmt; s->mtri = mtri; s->dhat = dhat; s->kappa = kappa;
    s->kappa_edge = kappa_edge; s->kappa_point = kappa_point;
    s->delta_T = delta_T; s->delta_e = delta_e; s->L = L;
    /* master edges: (min,max,tri) triples sorted */
    int32_t* tr = (int32_t*)malloc(sizeof(int32_t) * 9 * (size_t)nmt);
    for (int t = 0; t < nmt; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = mtri[3 * t + k], b = mtri[3 * t + (k + 1) % 3];
            tr[9 * t + 3 * k + 0] = a < b ? a : b;
            tr[9 * t + 3 * k + 1] = a < b ? b : a;
            tr[9 * t + 3 * k + 2] = t;
        }
    qsort(tr, (size_t)3 * nmt, 3 * sizeof(int32_t), cmp_triple);
    s->medge = (int32_t*)malloc(sizeof(int32_t) * 6 * (size_t)nmt);
    s->me_tri_off = (int32_t*)malloc(sizeof(int32_t) * (3 * (size_t)nmt + 1));
    s->me_tri = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)nmt);
    int ne = 0;
    for (int i = 0; i < 3 * nmt; ++i) {
        if (i == 0 || tr[3 * i] != tr[3 * (i - 1)] || tr[3 * i + 1] != tr[3 * (i - 1) + 1]) {
            s->medge[2 * ne] = tr[3 * i]; s->medge[2 * ne + 1] = tr[3 * i + 1];
            s->me_tri_off[ne] = i; ++ne;
        }
        s->me_tri[i] = tr[3 * i + 2];
    }
    s->me_tri_off[ne] = 3 * nmt;
    s->nme = ne;
    free(tr);
    /* vertex -> tri */
    s->mv_tri_off = (int32_t*)calloc((size_t)nmv + 1, sizeof(int32_t));
    s->mv_tri = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)nmt);
    for (int t = 0; t < nmt; ++t) for (int k = 0; k < 3; ++k) s->mv_tri_off[mtri[3 * t + k] + 1]++;
    for (int v = 0; v < nmv; ++v) s->mv_tri_off[v + 1] += s->mv_tri_off[v];
    int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nmv + 1));
    memcpy(cur, s->mv_tri_off, sizeof(int32_t) * ((size_t)nmv + 1));
    for (int t = 0; t < nmt; ++t) for (int k = 0; k < 3; ++k) s->mv_tri[cur[mtri[3 * t + k]]++] = t;
    free(cur);
    s->stri_env = (int32_t*)malloc(sizeof(int32_t) * ((size_t)ns + 1));
    for (int t = 0; t < ns; ++t) s->stri_env[t] = env_of(env_stri_off, n_env, t);
    s->mtri_env = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nmt + 1));
    for (int t = 0; t < nmt; ++t) s->mtri_env[t] = env_of(env_mtri_off, n_env, t);
    s->medge_env = (int32_t*)malloc(sizeof(int32_t) * ((size_t)ne + 1));
    for (int e = 0; e < ne; ++e) s->medge_env[e] = env_of(env_mvert_off, n_env, s->medge[2 * e]);
    s->mvert_env = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nmv + 1));
    for (int v = 0; v < nmv; ++v) s->mvert_env[v] = env_of(env_mvert_off, n_env, v);
    s->nk = 1 << (2 * L);
    s->rule = (double*)malloc(sizeof(double) * 3 * (size_t)s->nk);
    orc_face_rule(L, s->rule);
    /* unique slave vertices and edges */
    int32_t* vv = (int32_t*)malloc(sizeof(int32_t) * 6 * ((size_t)ns + 1));
    for (int i = 0; i < 3 * ns; ++i) { vv[2 * i] = stri[i]; vv[2 * i + 1] = 0; }
    qsort(vv, (size_t)3 * ns, 2 * sizeof(int32_t), cmp_pair);
    s->svert = (int32_t*)malloc(sizeof(int32_t) * (3 * (size_t)ns + 1));
    s->nsv = 0;
    for (int i = 0; i < 3 * ns; ++i) if (i == 0 || vv[2 * i] != vv[2 * (i - 1)]) s->svert[s->nsv++] = vv[2 * i];
    for (int t = 0; t < ns; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = stri[3 * t + k], b = stri[3 * t + (k + 1) % 3];
            vv[6 * t + 2 * k] = a < b ? a : b; vv[6 * t + 2 * k + 1] = a < b ? b : a;
        }
    qsort(vv, (size_t)3 * ns, 2 * sizeof(int32_t), cmp_pair);
    s->sedge = (int32_t*)malloc(sizeof(int32_t) * (6 * (size_t)ns + 2));
    s->nse = 0;
    for (int i = 0; i < 3 * ns; ++i)
        if (i == 0 || vv[2 * i] != vv[2 * (i - 1)] || vv[2 * i + 1] != vv[2 * (i - 1) + 1]) {
            s->sedge[2 * s->nse] = vv[2 * i]; s->sedge[2 * s->nse + 1] = vv[2 * i + 1]; s->nse++;
        }
    free(vv);
    return s;
}
ORC_API void orc_scene_set_guard(orc_scene* s, double dhat_guard, double kappa_guard) {
    s->dhat_guard = dhat_guard; s->kappa_guard = kappa_guard;
}

ORC_API void orc_scene_free(orc_scene* s) {
    if (!s) return;
    free(s->medge); free(s->me_tri_off); free(s->me_tri); free(s->mv_tri_off);
    free(s->mv_tri); free(s->stri_env); free(s->mtri_env); free(s->medge_env);
    free(s->mvert_env); free(s->rule); free(s->svert); free(s->sedge); free(s);
}
ORC_API int orc_scene_n_medges(const orc_scene* s) { return s->nme; }
ORC_API void orc_scene_set_all_pairs(orc_scene* s, int flag) { s->all_pairs = flag; }
ORC_API void orc_scene_set_face_clip(orc_scene* s, int flag) { s->face_clip = flag; }
static int g_verbose = 0;
ORC_API void orc_set_verbose(int v) { g_verbose = v; }
ORC_API void orc_scene_medges(const orc_scene* s, int32_t* out) {
    memcpy(out, s->medge, sizeof(int32_t) * 2 * (size_t)s->nme);
}

/* ------------------------------------------------------------------------- */
/* growable arrays                                                           */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t* a; int64_t n, cap; } ivec;
static void ivec_push2(ivec* v, int32_t x, int32_t y) {
    if (v->n + 2 > v->cap) { v->cap = v->cap ? 2 * v->cap : 1024; v->a = (int32_t*)realloc(v->a, sizeof(int32_t) * v->cap); }
    v->a[v->n++] = x; v->a[v->n++] = y;
}

/* ------------------------------------------------------------------------- */
/* candidate sets (broad phase by brute force; reading R10)                  */
/* ------------------------------------------------------------------------- */
static void tri_box(const double* P, const int32_t* t, double* lo, double* hi) {
    for (int c = 0; c < 3; ++c) {
        double a = P[3 * t[0] + c], b = P[3 * t[1] + c], d = P[3 * t[2] + c];
        lo[c] = dmin(a, dmin(b, d)); hi[c] = dmax(a, dmax(b, d));
    }
}

/* kind 0: face pairs (slave tri, master tri): some face sample of the slave
 *         tri lies in the master tri's box grown by dhat.
 * kind 1: edge pairs (slave tri, master edge): the slave tri's vertex box and
 *         the master edge's box grown by dhat overlap.
 * kind 2: point pairs (slave tri, master vertex): the master vertex grown by
 *         dhat overlaps the slave tri's vertex box.
 * Pairs are restricted to one env and returned sorted lexicographically.
 * Caller frees *out with orc_free. */
static int64_t candidates_sub(const orc_scene* s, int kind, const double* x, const double* xm,
                              const char* want, int32_t** out) {
    ivec v = {0, 0, 0};
    double eps = s->dhat;
    double* samp = (double*)malloc(sizeof(double) * 3 * (size_t)s->nk);
    for (int t = 0; t < s->ns; ++t) {
        if (want && !want[t]) continue;
        const int32_t* T = s->stri + 3 * t;
        const double *x0 = x + 3 * T[0], *x1 = x + 3 * T[1], *x2 = x + 3 * T[2];
        int e = s->stri_env[t];
        double slo[3], shi[3];
        tri_box(x, T, slo, shi);
        if (kind == 0 && s->face_clip) {
            /* clipped-overlap face samples (reading R20): the slave tri's box
             * meets the master tri's box grown by dhat */
            for (int64_t m = s->env_mtri_off[e]; m < s->env_mtri_off[e + 1]; ++m) {
                double lo[3], hi[3];
                tri_box(xm, s->mtri + 3 * m, lo, hi);
                int ok = 1;
                for (int c = 0; c < 3 && ok && !s->all_pairs; ++c) ok = slo[c] <= hi[c] + eps && lo[c] - eps <= shi[c];
                if (ok) ivec_push2(&v, t, (int32_t)m);
            }
        } else if (kind == 0) {
            for (int k = 0; k < s->nk; ++k) interp3(s->rule + 3 * k, x0, x1, x2, samp + 3 * k);
            for (int64_t m = s->env_mtri_off[e]; m < s->env_mtri_off[e + 1]; ++m) {
                double lo[3], hi[3];
                tri_box(xm, s->mtri + 3 * m, lo, hi);
                for (int c = 0; c < 3; ++c) { lo[c] = lo[c] - eps; hi[c] = hi[c] + eps; }
                int hit = s->all_pairs;
                for (int k = 0; k < s->nk && !hit; ++k) {
                    const double* q = samp + 3 * k;
                    hit = lo[0] <= q[0] && q[0] <= hi[0] && lo[1] <= q[1] && q[1] <= hi[1] &&
                          lo[2] <= q[2] && q[2] <= hi[2];
                }
                if (hit) ivec_push2(&v, t, (int32_t)m);
            }
        } else if (kind == 1) {
            for (int me = 0; me < s->nme; ++me) {
                if (s->medge_env[me] != e) continue;
                const double *a = xm + 3 * s->medge[2 * me], *b = xm + 3 * s->medge[2 * me + 1];
                int ok = 1;
                for (int c = 0; c < 3 && ok && !s->all_pairs; ++c) {
                    double lo = dmin(a[c], b[c]) - eps, hi = dmax(a[c], b[c]) + eps;
                    ok = slo[c] <= hi && lo <= shi[c];
                }
                if (ok) ivec_push2(&v, t, me);
            }
        } else {
            for (int64_t mv = s->env_mvert_off[e]; mv < s->env_mvert_off[e + 1]; ++mv) {
                if (s->mv_tri_off[mv + 1] == s->mv_tri_off[mv]) continue;
                const double* y = xm + 3 * mv;
                int ok = 1;
                for (int c = 0; c < 3 && ok && !s->all_pairs; ++c) ok = slo[c] <= y[c] + eps && y[c] - eps <= shi[c];
                if (ok) ivec_push2(&v, t, (int32_t)mv);
            }
        }
    }
    free(samp);
    qsort(v.a, (size_t)(v.n / 2), 2 * sizeof(int32_t), cmp_pair);
    *out = v.a;
    return v.n / 2;
}

ORC_API int64_t orc_candidates(const orc_scene* s, int kind, const double* x, const double* xm,
                               int32_t** out) {
    return candidates_sub(s, kind, x, xm, NULL, out);
}

ORC_API void orc_free(void* p) { free(p); }

/* ------------------------------------------------------------------------- */
/* contact samples (Sec. 4.1, 4.3, 4.4)                                      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int type;            /* 2 face, 1 edge, 0 point (the paper's q); guard pairs:
                            3 slave vertex-master tri, 4 master vertex-slave tri,
                            5 slave edge-master edge */
    int stri;            /* slave triangle (GMCP samples; -1 for guard 3/5) */
    int feat;            /* master tri / edge / vertex */
    int sv[3];           /* slave vertices carrying the gap gradient (-1 unused) */
    int mv[3];           /* master vertices used by x_m (-1 unused) */
    double bm[3];        /* their weights: beta^m, (1-eta, eta), (1) */
    double bs[3];        /* slave weights: beta^s (GMCP) or closest-point weights */
    double ns[3];        /* unit gap direction, slave to master (n_s for GMCP) */
    double g, eps, w, gamma, kq;
} orc_sample;

typedef struct { orc_sample* a; int64_t n, cap; } svec;
static void svec_push(svec* v, const orc_sample* s) {
    if (v->n + 1 > v->cap) { v->cap = v->cap ? 2 * v->cap : 1024; v->a = (orc_sample*)realloc(v->a, sizeof(orc_sample) * v->cap); }
    v->a[v->n++] = *s;
}

/* Face sample geometry: cast the slave sample xs along ns onto the plane of
 * the master triangle; facing iff N_m . ns < 0.  Returns 1 when the sample's
 * ray meets the plane of a facing master triangle with its hit point inside
 * the triangle (min beta^m >= 0) and g > 0; g and beta^m are written in all
 * facing cases.  Then x_m - x_s = g ns, which is Eq. (gap). */
static int face_geom(const double* xs, const double* ns, const double* y0, const double* y1,
                     const double* y2, double* g, double* bm, int* facing) {
    double e1[3], e2[3], N[3], d[3], p[3];
    sub3(y1, y0, e1); sub3(y2, y0, e2); cross3(e1, e2, N);
    double den = dot3(N, ns);
    *facing = den < 0.0;
    if (!(*facing)) return 0;
    sub3(y0, xs, d);
    *g = dot3(N, d) / den;
    for (int c = 0; c < 3; ++c) p[c] = xs[c] + (*g) * ns[c];
    bary_gram(p, y0, y1, y2, bm);
    return min3(bm) >= 0.0 && *g > 0.0;
}

/* support radius, Eq. (adaptive_eps), with g_ref taken at the rest
 * configuration (reading R5): eps = min(0.9 g_ref, eps_max) when the same
 * sample is geometrically valid at rest, else eps_max. */
static double eps_from_ref(int valid_ref, double g_ref, double eps_max) {
    if (!valid_ref) return eps_max;
    return dmin(0.9 * g_ref, eps_max);
}

static int any_facing(const orc_scene* s, const double* xm, const int32_t* tris, int n,
                      const double* ns) {
    for (int i = 0; i < n; ++i) {
        const int32_t* T = s->mtri + 3 * tris[i];
        double e1[3], e2[3], N[3];
        sub3(xm + 3 * T[1], xm + 3 * T[0], e1); sub3(xm + 3 * T[2], xm + 3 * T[0], e2);
        cross3(e1, e2, N);
        if (dot3(N, ns) < 0.0) return 1;
    }
    return 0;
}

/* forward declarations (definitions with the CCD code and the clipper below) */
ORC_API int orc_face_clip_samples(const double* xs, const double* xm, double* out);
static double ps_dist2(const double* p, const double* a, const double* b);
ORC_API double orc_pt_dist2(const double* p, const double* t0, const double* t1, const double* t2);
ORC_API double orc_ee_dist2(const double* a0, const double* a1, const double* b0, const double* b1);

/* closest point of triangle (t0,t1,t2) to p: weights w (barycentric of the
 * closest point), returns the squared distance */
static double pt_closest(const double* p, const double* t0, const double* t1, const double* t2,
                         double* w) {
    double b[3];
    bary_gram(p, t0, t1, t2, b);
    if (b[0] >= 0.0 && b[1] >= 0.0 && b[2] >= 0.0) {
        w[0] = b[0]; w[1] = b[1]; w[2] = b[2];
        return orc_pt_dist2(p, t0, t1, t2);
    }
    const double* P[3] = {t0, t1, t2};
    double best = INFINITY;
    for (int e = 0; e < 3; ++e) {
        const double *a = P[e], *c = P[(e + 1) % 3];
        double ab[3], ap[3], q[3], d[3];
        sub3(c, a, ab); sub3(p, a, ap);
        double t = dmin(dmax(dot3(ap, ab) / dot3(ab, ab), 0.0), 1.0);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + t * ab[k];
        sub3(p, q, d);
        double d2 = dot3(d, d);
        if (d2 < best) {
            best = d2; w[0] = w[1] = w[2] = 0.0; w[e] = 1.0 - t; w[(e + 1) % 3] = t;
        }
    }
    return best;
}

/* closest points of segments (a0,a1),(b0,b1): parameters s on a, t on b */
static double ee_closest(const double* a0, const double* a1, const double* b0, const double* b1,
                         double* s_out, double* t_out) {
    double u[3], v[3], w[3];
    sub3(a1, a0, u); sub3(b1, b0, v); sub3(a0, b0, w);
    double A = dot3(u, u), B = dot3(u, v), C = dot3(v, v), D = dot3(u, w), E = dot3(v, w);
    double cs[5], ct[5];
    cs[0] = 0.0; ct[0] = dmin(dmax(E / C, 0.0), 1.0);              /* a0 vs b */
    cs[1] = 1.0; ct[1] = dmin(dmax((E + B) / C, 0.0), 1.0);        /* a1 vs b */
    ct[2] = 0.0; cs[2] = dmin(dmax(-D / A, 0.0), 1.0);             /* b0 vs a */
    ct[3] = 1.0; cs[3] = dmin(dmax((B - D) / A, 0.0), 1.0);        /* b1 vs a */
    int n = 4;
    double den = A * C - B * B;
    if (den > 1e-14 * A * C) {
        double sc = (B * E - C * D) / den, tc = (A * E - B * D) / den;
        if (sc > 0.0 && sc < 1.0 && tc > 0.0 && tc < 1.0) { cs[4] = sc; ct[4] = tc; n = 5; }
    }
    double best = INFINITY;
    for (int i = 0; i < n; ++i) {
        double p[3], q[3], d[3];
        for (int k = 0; k < 3; ++k) { p[k] = a0[k] + cs[i] * u[k]; q[k] = b0[k] + ct[i] * v[k]; }
        sub3(q, p, d);
        double d2 = dot3(d, d);
        if (d2 < best) { best = d2; *s_out = cs[i]; *t_out = ct[i]; }
    }
    return best;
}

static int box_pt_overlap(const double* p, const double* lo, const double* hi, double r) {
    return lo[0] - r <= p[0] && p[0] <= hi[0] + r && lo[1] - r <= p[1] && p[1] <= hi[1] + r &&
           lo[2] - r <= p[2] && p[2] <= hi[2] + r;
}

/* Primitive guard barrier (not in the paper): pointwise samples on primitive
 * pairs closer than eps_g = min(0.9 d_ref, dhat_guard), d_ref the same pair's
 * distance at rest.  Gap = closest distance, direction = unit vector from
 * the slave closest point to the master closest point, weights = closest-
 * point weights; weight w = 1, gamma = 1, stiffness kappa_guard. */
static void collect_guard(const orc_scene* s, const double* x, const double* xm, const char* want,
                          svec* out) {
    double r = s->dhat_guard;
    const double *X = s->X, *Y0 = s->Y0;
    orc_sample smp;
    /* slave vertex - master triangle */
    for (int i = 0; i < s->nsv; ++i) {
        int v = s->svert[i];
        int e = env_of(s->env_vert_off, s->n_env, v);
        for (int64_t m = s->env_mtri_off[e]; m < s->env_mtri_off[e + 1]; ++m) {
            const int32_t* M = s->mtri + 3 * m;
            double lo[3], hi[3], w[3];
            tri_box(xm, M, lo, hi);
            if (!s->all_pairs && !box_pt_overlap(x + 3 * v, lo, hi, r)) continue;
            double d2 = pt_closest(x + 3 * v, xm + 3 * M[0], xm + 3 * M[1], xm + 3 * M[2], w);
            double d = sqrt(d2);
            double dref = sqrt(orc_pt_dist2(X + 3 * v, Y0 + 3 * M[0], Y0 + 3 * M[1], Y0 + 3 * M[2]));
            double eps = dmin(0.9 * dref, r);
            if (!(d > 0.0 && d < eps)) continue;
            memset(&smp, 0, sizeof(smp));
            smp.type = 3; smp.stri = -1; smp.feat = (int)m;
            smp.sv[0] = v; smp.sv[1] = -1; smp.sv[2] = -1;
            smp.bs[0] = 1.0;
            for (int c = 0; c < 3; ++c) {
                double q = w[0] * xm[3 * M[0] + c] + w[1] * xm[3 * M[1] + c] + w[2] * xm[3 * M[2] + c];
                smp.ns[c] = (q - x[3 * v + c]) / d;
                smp.mv[c] = M[c]; smp.bm[c] = w[c];
            }
            smp.g = d; smp.eps = eps; smp.w = 1.0; smp.gamma = 1.0; smp.kq = s->kappa_guard;
            svec_push(out, &smp);
        }
    }
    /* master vertex - slave triangle */
    for (int t = 0; t < s->ns; ++t) {
        if (!want[t]) continue;
        int e = s->stri_env[t];
        const int32_t* T = s->stri + 3 * t;
        double lo[3], hi[3], w[3];
        tri_box(x, T, lo, hi);
        for (int64_t u = s->env_mvert_off[e]; u < s->env_mvert_off[e + 1]; ++u) {
            if (s->mv_tri_off[u + 1] == s->mv_tri_off[u]) continue;
            if (!s->all_pairs && !box_pt_overlap(xm + 3 * u, lo, hi, r)) continue;
            double d2 = pt_closest(xm + 3 * u, x + 3 * T[0], x + 3 * T[1], x + 3 * T[2], w);
            double d = sqrt(d2);
            double dref = sqrt(orc_pt_dist2(Y0 + 3 * u, X + 3 * T[0], X + 3 * T[1], X + 3 * T[2]));
            double eps = dmin(0.9 * dref, r);
            if (!(d > 0.0 && d < eps)) continue;
            memset(&smp, 0, sizeof(smp));
            smp.type = 4; smp.stri = t; smp.feat = (int)u;
            for (int c = 0; c < 3; ++c) {
                double q = w[0] * x[3 * T[0] + c] + w[1] * x[3 * T[1] + c] + w[2] * x[3 * T[2] + c];
                smp.ns[c] = (xm[3 * u + c] - q) / d;
                smp.sv[c] = T[c]; smp.bs[c] = w[c];
            }
            smp.mv[0] = (int)u; smp.mv[1] = -1; smp.mv[2] = -1; smp.bm[0] = 1.0;
            smp.g = d; smp.eps = eps; smp.w = 1.0; smp.gamma = 1.0; smp.kq = s->kappa_guard;
            svec_push(out, &smp);
        }
    }
    /* slave edge - master edge */
    for (int i = 0; i < s->nse; ++i) {
        int a = s->sedge[2 * i], b = s->sedge[2 * i + 1];
        int e = env_of(s->env_vert_off, s->n_env, a);
        for (int me = 0; me < s->nme; ++me) {
            if (s->medge_env[me] != e) continue;
            int c0 = s->medge[2 * me], c1 = s->medge[2 * me + 1];
            if (!s->all_pairs) {
                int ok = 1;
                for (int c = 0; c < 3 && ok; ++c) {
                    double alo = dmin(x[3 * a + c], x[3 * b + c]), ahi = dmax(x[3 * a + c], x[3 * b + c]);
                    double blo = dmin(xm[3 * c0 + c], xm[3 * c1 + c]) - r, bhi = dmax(xm[3 * c0 + c], xm[3 * c1 + c]) + r;
                    ok = alo <= bhi && blo <= ahi;
                }
                if (!ok) continue;
            }
            double sp = 0.0, tp = 0.0;
            double d2 = ee_closest(x + 3 * a, x + 3 * b, xm + 3 * c0, xm + 3 * c1, &sp, &tp);
            double d = sqrt(d2);
            double dref = sqrt(orc_ee_dist2(X + 3 * a, X + 3 * b, Y0 + 3 * c0, Y0 + 3 * c1));
            double eps = dmin(0.9 * dref, r);
            if (!(d > 0.0 && d < eps)) continue;
            memset(&smp, 0, sizeof(smp));
            smp.type = 5; smp.stri = -1; smp.feat = me;
            smp.sv[0] = a; smp.sv[1] = b; smp.sv[2] = -1;
            smp.bs[0] = 1.0 - sp; smp.bs[1] = sp;
            smp.mv[0] = c0; smp.mv[1] = c1; smp.mv[2] = -1;
            smp.bm[0] = 1.0 - tp; smp.bm[1] = tp;
            for (int c = 0; c < 3; ++c) {
                double p = (1.0 - sp) * x[3 * a + c] + sp * x[3 * b + c];
                double q = (1.0 - tp) * xm[3 * c0 + c] + tp * xm[3 * c1 + c];
                smp.ns[c] = (q - p) / d;
            }
            smp.g = d; smp.eps = eps; smp.w = 1.0; smp.gamma = 1.0; smp.kq = s->kappa_guard;
            svec_push(out, &smp);
        }
    }
}

/* All active samples (0 < g < eps) of the given slave triangles (all when
 * subset == NULL).  Candidate pairs come from the brute-force sets above,
 * restricted to the subset. */
static void collect_samples(const orc_scene* s, const double* x, const double* xm,
                            int n_sub, const int32_t* sub, svec* out) {
    const double* X = s->X;
    const double* Y0 = s->Y0;
    double eps_max = s->dhat;
    char* want = (char*)calloc((size_t)s->ns + 1, 1);
    if (sub) for (int i = 0; i < n_sub; ++i) want[sub[i]] = 1;
    else memset(want, 1, (size_t)s->ns);
    for (int kind = 0; kind < 3; ++kind) {
        int32_t* pairs = NULL;
        int64_t np = candidates_sub(s, kind, x, xm, want, &pairs);
        for (int64_t p = 0; p < np; ++p) {
            int t = pairs[2 * p], f = pairs[2 * p + 1];
            if (!want[t]) continue;
            const int32_t* T = s->stri + 3 * t;
            const double *x0 = x + 3 * T[0], *x1 = x + 3 * T[1], *x2 = x + 3 * T[2];
            const double *X0 = X + 3 * T[0], *X1 = X + 3 * T[1], *X2 = X + 3 * T[2];
            double ns[3], As, ns0[3], As0;
            tri_normal_area(x0, x1, x2, ns, &As);
            tri_normal_area(X0, X1, X2, ns0, &As0);
            orc_sample smp;
            memset(&smp, 0, sizeof(smp));
            smp.stri = t; smp.feat = f;
            for (int c = 0; c < 3; ++c) smp.ns[c] = ns[c];
            if (kind == 0 && s->face_clip) {
                /* clipped-overlap face samples (Sec. 4.1 "Face samples", reading
                 * R20): the pair counts when the master tri faces the slave;
                 * each sample of the clipped overlap (orc_face_clip_samples) is
                 * active when 0 < g < eps, eps from the same slave point at
                 * rest (reading R5); weight = its Gauss weight, gamma =
                 * H(min beta^m, delta_T) */
                const int32_t* M = s->mtri + 3 * f;
                const double *y0 = xm + 3 * M[0], *y1 = xm + 3 * M[1], *y2 = xm + 3 * M[2];
                double e1[3], e2[3], N[3];
                sub3(y1, y0, e1); sub3(y2, y0, e2); cross3(e1, e2, N);
                if (!(dot3(N, ns) < 0.0)) continue;
                double xs9[9], xm9[9], cs[96];
                for (int c = 0; c < 3; ++c) {
                    xs9[c] = x0[c]; xs9[3 + c] = x1[c]; xs9[6 + c] = x2[c];
                    xm9[c] = y0[c]; xm9[3 + c] = y1[c]; xm9[6 + c] = y2[c];
                }
                int nsmp = orc_face_clip_samples(xs9, xm9, cs);
                for (int k = 0; k < nsmp; ++k) {
                    const double* o = cs + 8 * k;
                    double g = o[6];
                    if (!(g > 0.0)) continue;
                    double xs0[3], g0, bm0[3]; int facing0;
                    interp3(o, X0, X1, X2, xs0);
                    int ok0 = face_geom(xs0, ns0, Y0 + 3 * M[0], Y0 + 3 * M[1], Y0 + 3 * M[2], &g0, bm0, &facing0);
                    double eps = eps_from_ref(ok0, g0, eps_max);
                    if (!(g < eps)) continue;
                    smp.type = 2; smp.g = g; smp.eps = eps;
                    smp.sv[0] = T[0]; smp.sv[1] = T[1]; smp.sv[2] = T[2];
                    smp.w = o[7]; smp.gamma = orc_hermite(min3(o + 3), s->delta_T);
                    smp.kq = s->kappa;
                    for (int c = 0; c < 3; ++c) { smp.bs[c] = o[c]; smp.bm[c] = o[3 + c]; smp.mv[c] = M[c]; }
                    svec_push(out, &smp);
                }
            } else if (kind == 0) {
                /* face samples */
                const int32_t* M = s->mtri + 3 * f;
                const double *y0 = xm + 3 * M[0], *y1 = xm + 3 * M[1], *y2 = xm + 3 * M[2];
                const double *Y00 = Y0 + 3 * M[0], *Y01 = Y0 + 3 * M[1], *Y02 = Y0 + 3 * M[2];
                double omega = 1.0 / (double)s->nk;
                for (int k = 0; k < s->nk; ++k) {
                    const double* b = s->rule + 3 * k;
                    double xs[3], g, bm[3]; int facing;
                    interp3(b, x0, x1, x2, xs);
                    int ok = face_geom(xs, ns, y0, y1, y2, &g, bm, &facing);
                    if (!ok) continue;
                    double xs0[3], g0, bm0[3]; int facing0;
                    interp3(b, X0, X1, X2, xs0);
                    int ok0 = face_geom(xs0, ns0, Y00, Y01, Y02, &g0, bm0, &facing0);
                    double eps = eps_from_ref(ok0, g0, eps_max);
                    if (!(g < eps)) continue;
                    smp.type = 2; smp.g = g; smp.eps = eps;
                    smp.sv[0] = T[0]; smp.sv[1] = T[1]; smp.sv[2] = T[2];
                    smp.w = omega * As; smp.gamma = orc_hermite(min3(bm), s->delta_T);
                    smp.kq = s->kappa;
                    for (int c = 0; c < 3; ++c) { smp.bs[c] = b[c]; smp.bm[c] = bm[c]; smp.mv[c] = M[c]; }
                    svec_push(out, &smp);
                }
            } else if (kind == 1) {
                /* edge samples */
                int ia = s->medge[2 * f], ib = s->medge[2 * f + 1];
                int nadj = s->me_tri_off[f + 1] - s->me_tri_off[f];
                if (!any_facing(s, xm, s->me_tri + s->me_tri_off[f], nadj, ns)) continue;
                const double *ya = xm + 3 * ia, *yb = xm + 3 * ib;
                double bA[3], bB[3];
                bary_gram(ya, x0, x1, x2, bA);
                bary_gram(yb, x0, x1, x2, bB);
                double lo = 0.0, hi = 1.0; int empty = 0;
                for (int a = 0; a < 3; ++a) {
                    double D = bB[a] - bA[a];
                    if (D > 0.0) lo = dmax(lo, -bA[a] / D);
                    else if (D < 0.0) hi = dmin(hi, -bA[a] / D);
                    else if (bA[a] < 0.0) empty = 1;
                }
                if (empty || !(hi > lo)) continue;
                double tv[3], tp[3];
                sub3(yb, ya, tv);
                double tn = dot3(tv, ns);
                for (int c = 0; c < 3; ++c) tp[c] = tv[c] - tn * ns[c];
                double ell = (hi - lo) * sqrt(dot3(tp, tp));
                double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
                double gp = 1.0 / sqrt(3.0);
                for (int q = 0; q < 2; ++q) {
                    double eta = q == 0 ? mid - half * gp : mid + half * gp;
                    double xmk[3], bsk[3], xs[3], dv[3];
                    for (int c = 0; c < 3; ++c) xmk[c] = (1.0 - eta) * ya[c] + eta * yb[c];
                    bary_gram(xmk, x0, x1, x2, bsk);
                    interp3(bsk, x0, x1, x2, xs);
                    sub3(xmk, xs, dv);
                    double g = dot3(ns, dv);
                    if (!(g > 0.0)) continue;
                    /* the same sample (same eta) at rest */
                    double xm0[3], bs0[3], xs0[3], dv0[3];
                    const double *Ya = Y0 + 3 * ia, *Yb = Y0 + 3 * ib;
                    for (int c = 0; c < 3; ++c) xm0[c] = (1.0 - eta) * Ya[c] + eta * Yb[c];
                    bary_gram(xm0, X0, X1, X2, bs0);
                    interp3(bs0, X0, X1, X2, xs0);
                    sub3(xm0, xs0, dv0);
                    double g0 = dot3(ns0, dv0);
                    double eps = eps_from_ref(min3(bs0) >= 0.0 && g0 > 0.0, g0, eps_max);
                    if (!(g < eps)) continue;
                    smp.type = 1; smp.g = g; smp.eps = eps; smp.w = 0.5 * ell;
                    smp.sv[0] = T[0]; smp.sv[1] = T[1]; smp.sv[2] = T[2];
                    smp.gamma = orc_hermite(eta, s->delta_e) * orc_hermite(1.0 - eta, s->delta_e);
                    smp.kq = s->kappa_edge;
                    for (int c = 0; c < 3; ++c) smp.bs[c] = bsk[c];
                    smp.mv[0] = ia; smp.mv[1] = ib; smp.mv[2] = -1;
                    smp.bm[0] = 1.0 - eta; smp.bm[1] = eta; smp.bm[2] = 0.0;
                    svec_push(out, &smp);
                }
            } else {
                /* point samples */
                int nadj = s->mv_tri_off[f + 1] - s->mv_tri_off[f];
                if (!any_facing(s, xm, s->mv_tri + s->mv_tri_off[f], nadj, ns)) continue;
                const double* y = xm + 3 * f;
                double bs[3], xs[3], dv[3];
                bary_gram(y, x0, x1, x2, bs);
                if (!(min3(bs) >= 0.0)) continue;
                interp3(bs, x0, x1, x2, xs);
                sub3(y, xs, dv);
                double g = dot3(ns, dv);
                if (!(g > 0.0)) continue;
                double bs0[3], xs0[3], dv0[3];
                bary_gram(Y0 + 3 * f, X0, X1, X2, bs0);
                interp3(bs0, X0, X1, X2, xs0);
                sub3(Y0 + 3 * f, xs0, dv0);
                double g0 = dot3(ns0, dv0);
                double eps = eps_from_ref(min3(bs0) >= 0.0 && g0 > 0.0, g0, eps_max);
                if (!(g < eps)) continue;
                smp.type = 0; smp.g = g; smp.eps = eps; smp.w = 1.0; smp.gamma = 1.0;
                smp.sv[0] = T[0]; smp.sv[1] = T[1]; smp.sv[2] = T[2];
                smp.kq = s->kappa_point;
                for (int c = 0; c < 3; ++c) smp.bs[c] = bs[c];
                smp.mv[0] = f; smp.mv[1] = -1; smp.mv[2] = -1;
                smp.bm[0] = 1.0; smp.bm[1] = 0.0; smp.bm[2] = 0.0;
                svec_push(out, &smp);
            }
        }
        free(pairs);
    }
    /* guard pairs (whole scene only: they are not attached to one triangle) */
    if (s->kappa_guard > 0.0 && s->dhat_guard > 0.0 && !sub) collect_guard(s, x, xm, want, out);
    free(want);
}

/* ------------------------------------------------------------------------- */
/* potential, gradient, Hessian (Sec. 4.2)                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    double energy;
    int64_t n_samples[4];          /* active point, edge, face samples, guard pairs */
    double guard_energy;
    double* tri_energy;            /* [ns] */
    double* tri_coef;              /* [ns][9]: c1 (3) and S00 S01 S02 S11 S12 S22 */
    double* tri_normal;            /* [ns][3] */
    double* grad;                  /* [nv][3] */
    int64_t nblk;                  /* assembled Hessian blocks, sorted (i,j) */
    int32_t* blk_ij;               /* [nblk][2] */
    double* blk;                   /* [nblk][9] row-major */
} orc_contact_result;

static int cmp_blk(const void* a, const void* b) {
    const int32_t* x = (const int32_t*)a; const int32_t* y = (const int32_t*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

/* Eq. (gmcp_potential) and the approximate derivatives of Sec. 4.2:
 *   Psi      = sum_k kappa_q w_k gamma_k B(g_k, eps_k)
 *   grad_a   = sum_k kappa_q w_k gamma_k B'(g_k) dg_k/dx_a,  dg/dx_a = -beta^s_a n_s
 *   H_ab     = sum_k max(kappa_q w_k gamma_k B''(g_k), 0) beta_a beta_b n_s n_s^T
 * (rank-one per sample, so clamping the coefficient is the PSD projection).
 * The master is kinematic: its rows are not assembled. */
ORC_API orc_contact_result* orc_contact_eval(const orc_scene* s, const double* x, const double* xm,
                                             int n_sub, const int32_t* sub) {
    orc_contact_result* r = (orc_contact_result*)calloc(1, sizeof(orc_contact_result));
    svec v = {0, 0, 0};
    collect_samples(s, x, xm, n_sub, sub, &v);
    r->tri_energy = (double*)calloc((size_t)s->ns, sizeof(double));
    r->tri_coef = (double*)calloc((size_t)s->ns * 9, sizeof(double));
    r->tri_normal = (double*)calloc((size_t)s->ns * 3, sizeof(double));
    r->grad = (double*)calloc((size_t)s->nv * 3, sizeof(double));
    int64_t gn = 0, gcap = 0;
    int32_t* gij = NULL; double* gbv = NULL;
    for (int64_t i = 0; i < v.n; ++i) {
        const orc_sample* k = v.a + i;
        double B, dB, d2B;
        orc_barrier(k->g, k->eps, &B, &dB, &d2B);
        double coef = k->kq * k->w * k->gamma;
        double e = coef * B, c1 = coef * dB, c2 = dmax(coef * d2B, 0.0);
        r->energy += e;
        if (k->type >= 3) {
            r->n_samples[3]++;
            r->guard_energy += e;
            for (int a = 0; a < 3; ++a) {
                if (k->sv[a] < 0) continue;
                for (int c = 0; c < 3; ++c) r->grad[3 * (size_t)k->sv[a] + c] += -c1 * k->bs[a] * k->ns[c];
            }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    if (k->sv[a] < 0 || k->sv[b] < 0) continue;
                    if (gn + 1 > gcap) {
                        gcap = gcap ? 2 * gcap : 1024;
                        gij = (int32_t*)realloc(gij, sizeof(int32_t) * 2 * gcap);
                        gbv = (double*)realloc(gbv, sizeof(double) * 9 * gcap);
                    }
                    gij[2 * gn] = k->sv[a]; gij[2 * gn + 1] = k->sv[b];
                    for (int p = 0; p < 3; ++p)
                        for (int q = 0; q < 3; ++q) gbv[9 * gn + 3 * p + q] = c2 * k->bs[a] * k->bs[b] * k->ns[p] * k->ns[q];
                    gn++;
                }
            continue;
        }
        r->n_samples[k->type]++;
        r->tri_energy[k->stri] += e;
        double* C = r->tri_coef + 9 * (size_t)k->stri;
        C[0] += c1 * k->bs[0]; C[1] += c1 * k->bs[1]; C[2] += c1 * k->bs[2];
        C[3] += c2 * k->bs[0] * k->bs[0]; C[4] += c2 * k->bs[0] * k->bs[1];
        C[5] += c2 * k->bs[0] * k->bs[2]; C[6] += c2 * k->bs[1] * k->bs[1];
        C[7] += c2 * k->bs[1] * k->bs[2]; C[8] += c2 * k->bs[2] * k->bs[2];
        for (int c = 0; c < 3; ++c) r->tri_normal[3 * (size_t)k->stri + c] = k->ns[c];
    }
    /* gradient and blocks from the per-triangle coefficients */
    int64_t cap = 0;
    int32_t* ij = NULL; double* bv = NULL;
    for (int t = 0; t < s->ns; ++t) {
        const double* C = r->tri_coef + 9 * (size_t)t;
        int nz = 0;
        for (int q = 0; q < 9; ++q) nz |= C[q] != 0.0;
        if (!nz) continue;
        const int32_t* T = s->stri + 3 * t;
        const double* n = r->tri_normal + 3 * (size_t)t;
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) r->grad[3 * (size_t)T[a] + c] += -C[a] * n[c];
        static const int sidx[3][3] = {{3, 4, 5}, {4, 6, 7}, {5, 7, 8}};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                if (r->nblk + 1 > cap) {
                    cap = cap ? 2 * cap : 4096;
                    ij = (int32_t*)realloc(ij, sizeof(int32_t) * 2 * cap);
                    bv = (double*)realloc(bv, sizeof(double) * 9 * cap);
                }
                double Sab = C[sidx[a][b]];
                ij[2 * r->nblk] = T[a]; ij[2 * r->nblk + 1] = T[b];
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q) bv[9 * r->nblk + 3 * p + q] = Sab * n[p] * n[q];
                r->nblk++;
            }
    }
    for (int64_t i = 0; i < gn; ++i) {
        if (r->nblk + 1 > cap) {
            cap = cap ? 2 * cap : 4096;
            ij = (int32_t*)realloc(ij, sizeof(int32_t) * 2 * cap);
            bv = (double*)realloc(bv, sizeof(double) * 9 * cap);
        }
        ij[2 * r->nblk] = gij[2 * i]; ij[2 * r->nblk + 1] = gij[2 * i + 1];
        memcpy(bv + 9 * r->nblk, gbv + 9 * i, 9 * sizeof(double));
        r->nblk++;
    }
    free(gij); free(gbv);
    /* sort contributions by (i,j) and sum duplicates */
    int64_t nb = r->nblk;
    int32_t* key = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(nb + 1));
    for (int64_t i = 0; i < nb; ++i) { key[3 * i] = ij[2 * i]; key[3 * i + 1] = ij[2 * i + 1]; key[3 * i + 2] = (int32_t)i; }
    qsort(key, (size_t)nb, 3 * sizeof(int32_t), cmp_blk);
    r->blk_ij = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(nb + 1));
    r->blk = (double*)calloc((size_t)(nb + 1) * 9, sizeof(double));
    int64_t u = -1;
    for (int64_t i = 0; i < nb; ++i) {
        if (i == 0 || key[3 * i] != key[3 * (i - 1)] || key[3 * i + 1] != key[3 * (i - 1) + 1]) {
            ++u; r->blk_ij[2 * u] = key[3 * i]; r->blk_ij[2 * u + 1] = key[3 * i + 1];
        }
        for (int q = 0; q < 9; ++q) r->blk[9 * u + q] += bv[9 * (int64_t)key[3 * i + 2] + q];
    }
    r->nblk = u + 1;
    free(key); free(ij); free(bv); free(v.a);
    return r;
}

ORC_API void orc_contact_result_free(orc_contact_result* r) {
    if (!r) return;
    free(r->tri_energy); free(r->tri_coef); free(r->tri_normal); free(r->grad);
    free(r->blk_ij); free(r->blk); free(r);
}

/* Flat export of the active samples (for tests): per sample
 * [type, stri, feat, g, eps, w, gamma, kq, bs0, bs1, bs2]. */
ORC_API int64_t orc_samples(const orc_scene* s, const double* x, const double* xm,
                            int n_sub, const int32_t* sub, double** out) {
    svec v = {0, 0, 0};
    collect_samples(s, x, xm, n_sub, sub, &v);
    double* o = (double*)malloc(sizeof(double) * 11 * (size_t)(v.n + 1));
    for (int64_t i = 0; i < v.n; ++i) {
        const orc_sample* k = v.a + i;
        double row[11] = {k->type, k->stri, k->feat, k->g, k->eps, k->w, k->gamma, k->kq,
                          k->bs[0], k->bs[1], k->bs[2]};
        memcpy(o + 11 * i, row, sizeof(row));
    }
    free(v.a);
    *out = o;
    return v.n;
}

/* ------------------------------------------------------------------------- */
/* linearised step size, Eqs. (ccd) and (global_ccd)                         */
/* ------------------------------------------------------------------------- */
/* grad g_k . dx for a frozen sample: ns . (sum_a bm_a dy_a - sum_a bs_a dx_a) */
static double sample_dgdx(const orc_scene* s, const orc_sample* k, const double* dx,
                          const double* dy) {
    (void)s;
    double ds[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
        for (int a = 0; a < 3; ++a)
            if (k->sv[a] >= 0) ds[c] += k->bs[a] * dx[3 * k->sv[a] + c];
        if (dy)
            for (int a = 0; a < 3; ++a)
                if (k->mv[a] >= 0) dm[c] += k->bm[a] * dy[3 * k->mv[a] + c];
    }
    double d[3]; sub3(dm, ds, d);
    return dot3(k->ns, d);
}

/* alpha = min_k 0.9 g_k / (-grad g_k . dx) over active samples with
 * grad g_k . dx < 0; +inf when there is none.  dy (master displacement) may
 * be NULL. */
ORC_API double orc_alpha_lin(const orc_scene* s, const double* x, const double* xm,
                             const double* dx, const double* dy) {
    svec v = {0, 0, 0};
    collect_samples(s, x, xm, 0, NULL, &v);
    double alpha = INFINITY;
    for (int64_t i = 0; i < v.n; ++i) {
        double d = sample_dgdx(s, v.a + i, dx, dy);
        if (d < 0.0) alpha = dmin(alpha, 0.9 * v.a[i].g / (-d));
    }
    free(v.a);
    return alpha;
}

/* frozen-linear ("lagged") potential of the samples active at x, evaluated
 * at x + a dx for each a in alphas (reading R6): g~ = g + a (grad g . dx) */
/* Master rows of two-sided GMCP (Sec. 4.3 with Eq. gap): each sample's gap
 * is g = n_s . (x_m - x_s) with x_m = sum_j bm_j y_j, so with the sample's
 * normal and weights held fixed (as for the slave rows of orc_contact_eval)
 * master vertex y_j gets kappa_q w gamma B'(g) bm_j n_s.  GMCP samples only
 * (the primitive guard pairs are not included); n_sub > 0 restricts the
 * samples to the slave triangles sub[0..n_sub).  grad_m [nmv][3] is
 * overwritten. */
ORC_API void orc_master_grad(const orc_scene* s, const double* x, const double* xm, int n_sub,
                             const int32_t* sub, double* grad_m) {
    svec v = {0, 0, 0};
    collect_samples(s, x, xm, n_sub, sub, &v);
    memset(grad_m, 0, sizeof(double) * 3 * (size_t)s->nmv);
    for (int64_t i = 0; i < v.n; ++i) {
        const orc_sample* k = v.a + i;
        if (k->type > 2) continue;
        double B, dB, d2B;
        orc_barrier(k->g, k->eps, &B, &dB, &d2B);
        const double c1 = k->kq * k->w * k->gamma * dB;
        for (int j = 0; j < 3; ++j) {
            if (k->mv[j] < 0) continue;
            for (int c = 0; c < 3; ++c) grad_m[3 * (size_t)k->mv[j] + c] += c1 * k->bm[j] * k->ns[c];
        }
    }
    free(v.a);
}

/* Hessian blocks of two-sided GMCP that involve master vertices (Sec. 4.2
 * approximation, Sec. 4.3 with Eq. gap): a sample's gap gradient is
 * -bs_a n_s on slave vertex a and bm_j n_s on master vertex j; the block
 * (u, v) of two of them is max(kappa w gamma B''(g), 0) w_u w_v n_s n_s^T,
 * the same clamped curvature as the slave-slave blocks of orc_contact_eval.
 * Joint numbering: master vertex j is nv + j.  Written: (slave a, master j)
 * and (master i, master j) for every sample, unsorted, with repeats; at most
 * cap entries.  Returns the number of entries. */
ORC_API int64_t orc_master_hess(const orc_scene* s, const double* x, const double* xm, int n_sub,
                                const int32_t* sub, int64_t cap, int32_t* ij, double* blk) {
    svec v = {0, 0, 0};
    collect_samples(s, x, xm, n_sub, sub, &v);
    int64_t n = 0;
    for (int64_t i = 0; i < v.n; ++i) {
        const orc_sample* k = v.a + i;
        if (k->type > 2) continue;
        double B, dB, d2B;
        orc_barrier(k->g, k->eps, &B, &dB, &d2B);
        const double c2 = dmax(k->kq * k->w * k->gamma * d2B, 0.0);
        const int32_t* T = s->stri + 3 * (size_t)k->stri;
        for (int j = 0; j < 3; ++j) {
            if (k->mv[j] < 0) continue;
            /* rows: the three slave vertices, then the master vertices */
            for (int r = 0; r < 6; ++r) {
                int row;
                double wr;
                if (r < 3) { row = T[r]; wr = -k->bs[r]; }
                else {
                    if (k->mv[r - 3] < 0) continue;
                    row = s->nv + k->mv[r - 3]; wr = k->bm[r - 3];
                }
                if (n < cap) {
                    ij[2 * n] = row; ij[2 * n + 1] = s->nv + k->mv[j];
                    for (int p = 0; p < 3; ++p)
                        for (int q = 0; q < 3; ++q) blk[9 * n + 3 * p + q] = c2 * wr * k->bm[j] * k->ns[p] * k->ns[q];
                }
                ++n;
            }
        }
    }
    free(v.a);
    return n;
}

ORC_API void orc_contact_lagged(const orc_scene* s, const double* x, const double* xm,
                                const double* dx, int n_alpha, const double* alphas, double* out) {
    svec v = {0, 0, 0};
    collect_samples(s, x, xm, 0, NULL, &v);
    for (int j = 0; j < n_alpha; ++j) {
        double e = 0.0;
        for (int64_t i = 0; i < v.n; ++i) {
            const orc_sample* k = v.a + i;
            double gt = k->g + alphas[j] * sample_dgdx(s, k, dx, NULL);
            double B, dB, d2B;
            orc_barrier(gt, k->eps, &B, &dB, &d2B);
            e += k->kq * k->w * k->gamma * B;
        }
        out[j] = e;
    }
    free(v.a);
}

/* ------------------------------------------------------------------------- */
/* additive CCD (Li, Kaufman, Jiang 2021, Alg. 1), thickness 0               */
/* ------------------------------------------------------------------------- */
static double ps_dist2(const double* p, const double* a, const double* b) {
    double ab[3], ap[3], q[3], d[3];
    sub3(b, a, ab); sub3(p, a, ap);
    double t = dot3(ap, ab) / dot3(ab, ab);
    t = dmin(dmax(t, 0.0), 1.0);
    for (int c = 0; c < 3; ++c) q[c] = a[c] + t * ab[c];
    sub3(p, q, d);
    return dot3(d, d);
}

/* squared distance point p - triangle (t0,t1,t2): plane distance when the
 * projection falls inside, else the nearest edge */
ORC_API double orc_pt_dist2(const double* p, const double* t0, const double* t1, const double* t2) {
    double b[3];
    bary_gram(p, t0, t1, t2, b);
    if (b[0] >= 0.0 && b[1] >= 0.0 && b[2] >= 0.0) {
        double e1[3], e2[3], n[3], d[3];
        sub3(t1, t0, e1); sub3(t2, t0, e2); cross3(e1, e2, n); sub3(p, t0, d);
        double h = dot3(d, n);
        return h * h / dot3(n, n);
    }
    return dmin(ps_dist2(p, t0, t1), dmin(ps_dist2(p, t1, t2), ps_dist2(p, t2, t0)));
}

/* squared distance between segments (a0,a1) and (b0,b1): the four endpoint-
 * segment distances and, when the closest points of the two lines fall inside
 * both segments, the line-line distance */
ORC_API double orc_ee_dist2(const double* a0, const double* a1, const double* b0, const double* b1) {
    double d = dmin(dmin(ps_dist2(a0, b0, b1), ps_dist2(a1, b0, b1)),
                    dmin(ps_dist2(b0, a0, a1), ps_dist2(b1, a0, a1)));
    double u[3], v[3], w[3];
    sub3(a1, a0, u); sub3(b1, b0, v); sub3(a0, b0, w);
    double A = dot3(u, u), B = dot3(u, v), C = dot3(v, v), D = dot3(u, w), E = dot3(v, w);
    double den = A * C - B * B;
    if (den > 1e-14 * A * C) {
        double sc = (B * E - C * D) / den, tc = (A * E - B * D) / den;
        if (sc > 0.0 && sc < 1.0 && tc > 0.0 && tc < 1.0) {
            double n[3]; cross3(u, v, n);
            double h = dot3(w, n);
            d = dmin(d, h * h / dot3(n, n));
        }
    }
    return d;
}

/* brute-force minimum squared distance between two triangle surfaces (the
 * invariant a CCD-limited step must keep > 0): every vertex of one against
 * every triangle of the other, both ways, and every edge pair (edges taken
 * from the triangles, repeats included) */
ORC_API double orc_surface_min_dist2(const double* xa, const int32_t* ta, int64_t na,
                                     const double* xb, const int32_t* tb, int64_t nb) {
    double best = INFINITY;
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j) {
            const int32_t* A = ta + 3 * i;
            const int32_t* B = tb + 3 * j;
            for (int k = 0; k < 3; ++k) {
                best = dmin(best, orc_pt_dist2(xa + 3 * A[k], xb + 3 * B[0], xb + 3 * B[1], xb + 3 * B[2]));
                best = dmin(best, orc_pt_dist2(xb + 3 * B[k], xa + 3 * A[0], xa + 3 * A[1], xa + 3 * A[2]));
                for (int l = 0; l < 3; ++l)
                    best = dmin(best, orc_ee_dist2(xa + 3 * A[k], xa + 3 * A[(k + 1) % 3],
                                                   xb + 3 * B[l], xb + 3 * B[(l + 1) % 3]));
            }
        }
    return best;
}

/* ACCD for one primitive pair.  type 0: point x[0] vs triangle x[1..3];
 * type 1: edge x[0..1] vs edge x[2..3].  p[] are the displacements over the
 * step; returns the largest safe fraction found in [0, tc] (tc when no
 * collision is detected before tc).  s is the distance fraction at which the
 * iteration stops (0 < s < 1), the first advance closes (1-s) of the gap and
 * later ones 0.9 of the remaining gap over the bound lp of the relative
 * speed.  *iters receives the iteration count. */
ORC_API double orc_accd(int type, const double* x_in, const double* p_in, double s, double tc,
                        int max_iter, int* iters) {
    double x[12], p[12], pbar[3] = {0, 0, 0};
    memcpy(x, x_in, sizeof(x)); memcpy(p, p_in, sizeof(p));
    for (int i = 0; i < 4; ++i) for (int c = 0; c < 3; ++c) pbar[c] += p[3 * i + c];
    for (int c = 0; c < 3; ++c) pbar[c] = pbar[c] / 4.0;
    for (int i = 0; i < 4; ++i) for (int c = 0; c < 3; ++c) p[3 * i + c] -= pbar[c];
    double n[4];
    for (int i = 0; i < 4; ++i) n[i] = sqrt(dot3(p + 3 * i, p + 3 * i));
    double lp = type == 0 ? n[0] + dmax(n[1], dmax(n[2], n[3])) : dmax(n[0], n[1]) + dmax(n[2], n[3]);
    *iters = 0;
    if (lp == 0.0) return tc;
    double d2 = type == 0 ? orc_pt_dist2(x, x + 3, x + 6, x + 9) : orc_ee_dist2(x, x + 3, x + 6, x + 9);
    double d = sqrt(d2);
    if (d == 0.0) return 0.0;
    double gstop = s * d;
    double t = 0.0;
    double tl = (1.0 - s) * d / lp;
    for (int it = 0; it < max_iter; ++it) {
        *iters = it + 1;
        for (int i = 0; i < 12; ++i) x[i] = x[i] + tl * p[i];
        d2 = type == 0 ? orc_pt_dist2(x, x + 3, x + 6, x + 9) : orc_ee_dist2(x, x + 3, x + 6, x + 9);
        d = sqrt(d2);
        if (t > 0.0 && d < gstop) return t;
        t = t + tl;
        if (t > tc) return tc;
        tl = 0.9 * d / lp;
    }
    return t;
}

static void swept_box(const double* P, const double* D, const int32_t* idx, int n, double* lo,
                      double* hi) {
    for (int c = 0; c < 3; ++c) { lo[c] = INFINITY; hi[c] = -INFINITY; }
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            double a = P[3 * idx[i] + c];
            double b = D ? a + D[3 * idx[i] + c] : a;
            lo[c] = dmin(lo[c], dmin(a, b)); hi[c] = dmax(hi[c], dmax(a, b));
        }
}
static int box_overlap(const double* alo, const double* ahi, const double* blo, const double* bhi) {
    return alo[0] <= bhi[0] && blo[0] <= ahi[0] && alo[1] <= bhi[1] && blo[1] <= ahi[1] &&
           alo[2] <= bhi[2] && blo[2] <= ahi[2];
}

typedef struct { double alpha_accd; int64_t n_pt, n_ee, n_iter_total; int max_iter_hit; double alpha_type[3]; } orc_accd_info;

/* min over primitive pairs of one env whose swept boxes overlap:
 *  slave surface vertex / master triangle, master vertex / slave triangle,
 *  slave edge / master edge.  x moves by dx, the master from xm0 by dxm. */
ORC_API double orc_accd_min(const orc_scene* s, const double* x, const double* dx,
                            const double* xm0, const double* dxm, double slack, int max_iter,
                            orc_accd_info* info) {
    double alpha = 1.0;
    memset(info, 0, sizeof(*info));
    info->alpha_type[0] = info->alpha_type[1] = info->alpha_type[2] = 1.0;
    /* unique slave surface vertices and edges */
    int ns = s->ns;
    int32_t* svs = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)ns);
    int32_t* vv = (int32_t*)malloc(sizeof(int32_t) * 6 * (size_t)ns);
    for (int i = 0; i < 3 * ns; ++i) { vv[2 * i] = s->stri[i]; vv[2 * i + 1] = 0; }
    qsort(vv, (size_t)3 * ns, 2 * sizeof(int32_t), cmp_pair);
    int nsv = 0;
    for (int i = 0; i < 3 * ns; ++i) if (i == 0 || vv[2 * i] != vv[2 * (i - 1)]) svs[nsv++] = vv[2 * i];
    /* unique slave edges */
    int32_t* se = (int32_t*)malloc(sizeof(int32_t) * 6 * (size_t)ns);
    for (int t = 0; t < ns; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = s->stri[3 * t + k], b = s->stri[3 * t + (k + 1) % 3];
            se[6 * t + 2 * k] = a < b ? a : b; se[6 * t + 2 * k + 1] = a < b ? b : a;
        }
    qsort(se, (size_t)3 * ns, 2 * sizeof(int32_t), cmp_pair);
    int nse = 0;
    for (int i = 0; i < 3 * ns; ++i)
        if (i == 0 || se[2 * i] != se[2 * (i - 1)] || se[2 * i + 1] != se[2 * (i - 1) + 1]) {
            se[2 * nse] = se[2 * i]; se[2 * nse + 1] = se[2 * i + 1]; ++nse;
        }
    double X12[12], P12[12];
    int it;
    /* slave vertex - master triangle */
    for (int i = 0; i < nsv; ++i) {
        int v = svs[i];
        int e = env_of(s->env_vert_off, s->n_env, v);
        double vlo[3], vhi[3];
        swept_box(x, dx, &v, 1, vlo, vhi);
        for (int64_t m = s->env_mtri_off[e]; m < s->env_mtri_off[e + 1]; ++m) {
            double mlo[3], mhi[3];
            swept_box(xm0, dxm, s->mtri + 3 * m, 3, mlo, mhi);
            if (!box_overlap(vlo, vhi, mlo, mhi)) continue;
            const int32_t* M = s->mtri + 3 * m;
            for (int c = 0; c < 3; ++c) {
                X12[c] = x[3 * v + c]; P12[c] = dx[3 * v + c];
                for (int a = 0; a < 3; ++a) {
                    X12[3 + 3 * a + c] = xm0[3 * M[a] + c];
                    P12[3 + 3 * a + c] = dxm ? dxm[3 * M[a] + c] : 0.0;
                }
            }
            double t = orc_accd(0, X12, P12, slack, 1.0, max_iter, &it);
            info->n_pt++; info->n_iter_total += it; if (it >= max_iter) info->max_iter_hit = 1;
            alpha = dmin(alpha, t); info->alpha_type[0] = dmin(info->alpha_type[0], t);
        }
    }
    /* master vertex - slave triangle */
    for (int t = 0; t < ns; ++t) {
        int e = s->stri_env[t];
        const int32_t* T = s->stri + 3 * t;
        double tlo[3], thi[3];
        swept_box(x, dx, T, 3, tlo, thi);
        for (int64_t v = s->env_mvert_off[e]; v < s->env_mvert_off[e + 1]; ++v) {
            if (s->mv_tri_off[v + 1] == s->mv_tri_off[v]) continue;
            int32_t vi = (int32_t)v;
            double vlo[3], vhi[3];
            swept_box(xm0, dxm, &vi, 1, vlo, vhi);
            if (!box_overlap(vlo, vhi, tlo, thi)) continue;
            for (int c = 0; c < 3; ++c) {
                X12[c] = xm0[3 * v + c]; P12[c] = dxm ? dxm[3 * v + c] : 0.0;
                for (int a = 0; a < 3; ++a) { X12[3 + 3 * a + c] = x[3 * T[a] + c]; P12[3 + 3 * a + c] = dx[3 * T[a] + c]; }
            }
            double tt = orc_accd(0, X12, P12, slack, 1.0, max_iter, &it);
            info->n_pt++; info->n_iter_total += it; if (it >= max_iter) info->max_iter_hit = 1;
            alpha = dmin(alpha, tt); info->alpha_type[1] = dmin(info->alpha_type[1], tt);
        }
    }
    /* slave edge - master edge */
    for (int i = 0; i < nse; ++i) {
        int32_t ab[2] = {se[2 * i], se[2 * i + 1]};
        int e = env_of(s->env_vert_off, s->n_env, ab[0]);
        double alo[3], ahi[3];
        swept_box(x, dx, ab, 2, alo, ahi);
        for (int me = 0; me < s->nme; ++me) {
            if (s->medge_env[me] != e) continue;
            double blo[3], bhi[3];
            swept_box(xm0, dxm, s->medge + 2 * me, 2, blo, bhi);
            if (!box_overlap(alo, ahi, blo, bhi)) continue;
            for (int c = 0; c < 3; ++c) {
                X12[c] = x[3 * ab[0] + c]; P12[c] = dx[3 * ab[0] + c];
                X12[3 + c] = x[3 * ab[1] + c]; P12[3 + c] = dx[3 * ab[1] + c];
                int m0 = s->medge[2 * me], m1 = s->medge[2 * me + 1];
                X12[6 + c] = xm0[3 * m0 + c]; P12[6 + c] = dxm ? dxm[3 * m0 + c] : 0.0;
                X12[9 + c] = xm0[3 * m1 + c]; P12[9 + c] = dxm ? dxm[3 * m1 + c] : 0.0;
            }
            double tt = orc_accd(1, X12, P12, slack, 1.0, max_iter, &it);
            info->n_ee++; info->n_iter_total += it; if (it >= max_iter) info->max_iter_hit = 1;
            alpha = dmin(alpha, tt); info->alpha_type[2] = dmin(info->alpha_type[2], tt);
        }
    }
    free(svs); free(vv); free(se);
    info->alpha_accd = alpha;
    return alpha;
}

/* maximum step: min(1, alpha_lin, alpha_accd) for the motion x -> x + dx,
 * master xm0 -> xm1 (xm1 may be NULL for a static master) */
ORC_API double orc_ccd_max_step(const orc_scene* s, const double* x, const double* dx,
                                const double* xm0, const double* xm1, double slack, int max_iter,
                                double* alpha_lin_out, double* alpha_accd_out) {
    double* dxm = NULL;
    if (xm1) {
        dxm = (double*)malloc(sizeof(double) * 3 * (size_t)s->nmv);
        for (int i = 0; i < 3 * s->nmv; ++i) dxm[i] = xm1[i] - xm0[i];
    }
    double al = orc_alpha_lin(s, x, xm0, dx, dxm);
    orc_accd_info info;
    double aa = orc_accd_min(s, x, dx, xm0, dxm, slack, max_iter, &info);
    free(dxm);
    if (alpha_lin_out) *alpha_lin_out = al;
    if (alpha_accd_out) *alpha_accd_out = aa;
    return dmin(1.0, dmin(al, aa));
}

/* ========================================================================= */
/* elasticity: compressible Neo-Hookean tets (reading R7)                    */
/* Psi = V [ mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2 ]             */
/* F = Ds Dm^-1 (row-major 3x3); vec(F) index 3*i + j                        */
/* ========================================================================= */
static double det3(const double* A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}
static void inv3(const double* A, double* I) {
    double d = det3(A);
    I[0] = (A[4] * A[8] - A[5] * A[7]) / d; I[1] = (A[2] * A[7] - A[1] * A[8]) / d;
    I[2] = (A[1] * A[5] - A[2] * A[4]) / d; I[3] = (A[5] * A[6] - A[3] * A[8]) / d;
    I[4] = (A[0] * A[8] - A[2] * A[6]) / d; I[5] = (A[2] * A[3] - A[0] * A[5]) / d;
    I[6] = (A[3] * A[7] - A[4] * A[6]) / d; I[7] = (A[1] * A[6] - A[0] * A[7]) / d;
    I[8] = (A[0] * A[4] - A[1] * A[3]) / d;
}
static void mul3(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

/* cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 12):
 * on return A is diagonal (eigenvalues) and V holds eigenvectors in columns */
static void jacobi_eig(int n, double* A, double* V) {
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) { tot += A[i * n + j] * A[i * n + j]; if (i != j) off += A[i * n + j] * A[i * n + j]; }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq; A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk; A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq; V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

/* projection of a symmetric n x n matrix onto the PSD cone: V max(L,0) V^T */
ORC_API void orc_psd_project(int n, double* A) {
    double W[144], V[144];
    memcpy(W, A, sizeof(double) * n * n);
    jacobi_eig(n, W, V);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) {
                double l = W[k * n + k];
                if (l > 0.0) s += V[i * n + k] * l * V[j * n + k];
            }
            A[i * n + j] = s;
        }
}

/* d - log1p(d), without the cancellation of the plain difference when d is
 * small: its Taylor series d^2/2 - d^3/3 + ... - d^9/9 for |d| < 1e-2
 * (truncation below 1e-17 relative), else the plain difference. */
static double d_minus_log1p(double d) {
    if (fabs(d) < 1e-2)
        return d * d * (1.0 / 2 - d * (1.0 / 3 - d * (1.0 / 4 - d * (1.0 / 5 - d * (1.0 / 6 - d * (1.0 / 7 - d * (1.0 / 8 - d / 9.0)))))));
    return d - log1p(d);
}

/* One tet: energy, gradient [12] (vertex-major), PSD Hessian [12x12] (the
 * 9x9 dP/dF is projected, then mapped by dF/dx).  X4 are the rest positions
 * of the four vertices, x4 the current ones.  Returns 0 if J <= 0.
 * Reading R15: the energy is evaluated from the displacement gradient
 * H = F - I = (Ds - Dm) Dm^-1 as
 *   Psi/V = mu ((J-1) - ln J - q) + mu/2 |H|^2 + lambda/2 (ln J)^2,
 *   J - 1 = tr H + q,  q = (sum of principal 2x2 minors of H) + det H,
 * which is the textbook mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2
 * rearranged (tr F^T F - 3 = 2 tr H + |H|^2) so that its first-order terms
 * cancel analytically instead of in rounding. */
ORC_API int orc_nh_tet(const double* Dminv, double vol, double mu, double lam, const double* X4,
                       const double* x4, double* psi, double* grad, double* hess) {
    double Du[9], H[9], F[9], Fi[9], G[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Du[3 * r + c] = (x4[3 * (c + 1) + r] - X4[3 * (c + 1) + r]) - (x4[r] - X4[r]);
    mul3(Du, Dminv, H);
    for (int i = 0; i < 9; ++i) F[i] = H[i];
    F[0] += 1.0; F[4] += 1.0; F[8] += 1.0;
    const double trH = H[0] + H[4] + H[8];
    const double minors = (H[0] * H[4] - H[1] * H[3]) + (H[0] * H[8] - H[2] * H[6]) + (H[4] * H[8] - H[5] * H[7]);
    const double q = minors + det3(H);
    const double jm1 = trH + q;
    if (!(jm1 > -1.0)) { *psi = INFINITY; return 0; }
    double nH = 0.0;
    for (int i = 0; i < 9; ++i) nH += H[i] * H[i];
    const double lnJ = log1p(jm1);
    *psi = vol * (mu * (d_minus_log1p(jm1) - q) + 0.5 * mu * nH + 0.5 * lam * lnJ * lnJ);
    inv3(F, Fi);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) G[3 * i + j] = Fi[3 * j + i];
    double D[12];   /* D[m][j]: dF_ij / dx_{m,i} */
    for (int j = 0; j < 3; ++j) {
        D[3 * 1 + j] = Dminv[0 * 3 + j]; D[3 * 2 + j] = Dminv[1 * 3 + j]; D[3 * 3 + j] = Dminv[2 * 3 + j];
        D[j] = -(D[3 + j] + D[6 + j] + D[9 + j]);
    }
    if (grad) {
        double P[9];
        for (int i = 0; i < 9; ++i) P[i] = mu * (F[i] - G[i]) + lam * lnJ * G[i];
        for (int m = 0; m < 4; ++m)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) s += P[3 * i + j] * D[3 * m + j];
                grad[3 * m + i] = vol * s;
            }
    }
    if (hess) {
        double H9[81];
        double cc = mu - lam * lnJ;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l)
                    for (int k = 0; k < 3; ++k)
                        H9[(3 * i + j) * 9 + 3 * l + k] = (i == l && j == k ? mu : 0.0) +
                                                          cc * G[3 * i + k] * G[3 * l + j] +
                                                          lam * G[3 * i + j] * G[3 * l + k];
        orc_psd_project(9, H9);
        for (int m = 0; m < 4; ++m)
            for (int a = 0; a < 3; ++a)
                for (int n = 0; n < 4; ++n)
                    for (int b = 0; b < 3; ++b) {
                        double s = 0.0;
                        for (int j = 0; j < 3; ++j)
                            for (int k = 0; k < 3; ++k)
                                s += D[3 * m + j] * H9[(3 * a + j) * 9 + 3 * b + k] * D[3 * n + k];
                        hess[(3 * m + a) * 12 + 3 * n + b] = vol * s;
                    }
    }
    return 1;
}

/* ========================================================================= */
/* implicit-Euler time step (reading R7/R8)                                  */
/* ========================================================================= */
typedef struct {
    orc_scene* sc;
    int nv, nt;
    const double* X; const int32_t* tets; const uint8_t* dir;
    double *Dminv, *vol, *mass;
    double h, rho, E, nu, mu, lam, grav[3];
    double tol, pcg_tol; int max_newton, max_pcg, max_halv; double slack; int ccd_max_iter;
    int32_t* rp; int32_t* ci; int64_t nnzb;
    double* xm;     /* current master positions (kinematic master) */
    /* deformable master (joint step): the system's vertices are the pad's
     * npad vertices followed by the master's; own copies of the system's
     * rest positions, tets and Dirichlet flags; external nodal forces */
    int joint, npad;
    double* Xsys; int32_t* Tsys; uint8_t* Dsys;
    double* fext;
} orc_sim;

typedef struct {
    int status;              /* 0 ok, 3 infeasible, 5 not converged, 6 line search */
    int newton_iters, pcg_iters_total;
    double residual, res0, alpha0, last_alpha;
    double energy;
    int pred_used;           /* 1 if the predicted start was taken */
} orc_stats;

/* extra (row, col) pairs of the block pattern, both orders (joint step) */
typedef struct { int32_t* a; int64_t n, cap; } pvec;
static void pvec_push(pvec* v, int32_t i, int32_t j) {
    if (v->n + 2 > v->cap) { v->cap = v->cap ? 2 * v->cap : 4096; v->a = (int32_t*)realloc(v->a, sizeof(int32_t) * 2 * v->cap); }
    v->a[2 * v->n] = i; v->a[2 * v->n + 1] = j; ++v->n;
    v->a[2 * v->n] = j; v->a[2 * v->n + 1] = i; ++v->n;
}

static orc_sim* sim_init(orc_sim* s, orc_scene* sc, int nv, const double* X, int nt, const int32_t* tets,
                         const uint8_t* dir, double h, double rho, double E, double nu,
                         const double* grav, double tol, double pcg_tol, int max_newton,
                         int max_pcg, int max_halv, double slack, int ccd_max_iter, const pvec* extra);

ORC_API orc_sim* orc_sim_create(orc_scene* sc, int nv, const double* X, int nt, const int32_t* tets,
                                const uint8_t* dir, double h, double rho, double E, double nu,
                                const double* grav, double tol, double pcg_tol, int max_newton,
                                int max_pcg, int max_halv, double slack, int ccd_max_iter) {
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    return sim_init(s, sc, nv, X, nt, tets, dir, h, rho, E, nu, grav, tol, pcg_tol, max_newton, max_pcg,
                    max_halv, slack, ccd_max_iter, NULL);
}

/* Joint step with a deformable master (Sec. 4.2-4.3 with Eq. gap: the
 * contact potential depends on the master vertices through x_m): the system
 * is the pad (npad vertices, ntp tets, Dirichlet flags dir) followed by the
 * master body (the scene's nmv master vertices at rest sc->Y0, nmt4 tets
 * mtets over master vertex indices, Dirichlet flags mdir), one material.
 * The block pattern also holds every (slave-triangle vertex, master-triangle
 * vertex) pair of the same environment, so every contact block has a place.
 * Single environment. */
ORC_API orc_sim* orc_sim_create_joint(orc_scene* sc, int npad, const double* X, int ntp, const int32_t* tets,
                                      const uint8_t* dir, int nmt4, const int32_t* mtets, const uint8_t* mdir,
                                      double h, double rho, double E, double nu, const double* grav, double tol,
                                      double pcg_tol, int max_newton, int max_pcg, int max_halv, double slack,
                                      int ccd_max_iter) {
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    const int nm = (int)sc->nmv, nsys = npad + nm, nts = ntp + nmt4;
    s->joint = 1;
    s->npad = npad;
    s->Xsys = (double*)malloc(sizeof(double) * 3 * (size_t)nsys);
    s->Tsys = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)(nts > 0 ? nts : 1));
    s->Dsys = (uint8_t*)calloc((size_t)nsys, 1);
    memcpy(s->Xsys, X, sizeof(double) * 3 * (size_t)npad);
    memcpy(s->Xsys + 3 * (size_t)npad, sc->Y0, sizeof(double) * 3 * (size_t)nm);
    memcpy(s->Tsys, tets, sizeof(int32_t) * 4 * (size_t)ntp);
    for (int64_t e = 0; e < 4 * (int64_t)nmt4; ++e) s->Tsys[4 * (int64_t)ntp + e] = npad + mtets[e];
    memcpy(s->Dsys, dir, (size_t)npad);
    if (mdir) memcpy(s->Dsys + npad, mdir, (size_t)nm);
    pvec extra = {0, 0, 0};
    for (int64_t t = 0; t < sc->ns; ++t)
        for (int64_t m = 0; m < sc->nmt; ++m) {
            if (sc->stri_env[t] != sc->mtri_env[m]) continue;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) pvec_push(&extra, sc->stri[3 * t + a], npad + sc->mtri[3 * m + b]);
        }
    for (int64_t m = 0; m < sc->nmt; ++m)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (a != b) pvec_push(&extra, npad + sc->mtri[3 * m + a], npad + sc->mtri[3 * m + b]);
    sim_init(s, sc, nsys, s->Xsys, nts, s->Tsys, s->Dsys, h, rho, E, nu, grav, tol, pcg_tol, max_newton, max_pcg,
             max_halv, slack, ccd_max_iter, &extra);
    free(extra.a);
    return s;
}

/* external nodal forces f [nsys][3] (joint step): the energy gains
 * -h^2 f.(x - xhat), i.e. -h^2 f.x up to a constant of the step */
ORC_API void orc_sim_set_fext(orc_sim* s, const double* f) {
    if (!s->fext) s->fext = (double*)malloc(sizeof(double) * 3 * (size_t)s->nv);
    memcpy(s->fext, f, sizeof(double) * 3 * (size_t)s->nv);
}

static orc_sim* sim_init(orc_sim* s, orc_scene* sc, int nv, const double* X, int nt, const int32_t* tets,
                         const uint8_t* dir, double h, double rho, double E, double nu,
                         const double* grav, double tol, double pcg_tol, int max_newton,
                         int max_pcg, int max_halv, double slack, int ccd_max_iter, const pvec* extra) {
    s->sc = sc; s->nv = nv; s->nt = nt; s->X = X; s->tets = tets; s->dir = dir;
    s->h = h; s->rho = rho; s->E = E; s->nu = nu;
    s->mu = E / (2.0 * (1.0 + nu)); s->lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    for (int c = 0; c < 3; ++c) s->grav[c] = grav[c];
    s->tol = tol; s->pcg_tol = pcg_tol; s->max_newton = max_newton; s->max_pcg = max_pcg;
    s->max_halv = max_halv; s->slack = slack; s->ccd_max_iter = ccd_max_iter;
    s->Dminv = (double*)malloc(sizeof(double) * 9 * (size_t)nt);
    s->vol = (double*)malloc(sizeof(double) * (size_t)nt);
    s->mass = (double*)calloc((size_t)nv, sizeof(double));
    for (int t = 0; t < nt; ++t) {
        const int32_t* T = tets + 4 * t;
        double Dm[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Dm[3 * r + c] = X[3 * T[c + 1] + r] - X[3 * T[0] + r];
        s->vol[t] = fabs(det3(Dm)) / 6.0;
        inv3(Dm, s->Dminv + 9 * t);
        for (int a = 0; a < 4; ++a) s->mass[T[a]] += rho * s->vol[t] / 4.0;
    }
    /* block pattern: vertex adjacency through tets, plus the diagonal */
    const int64_t nx = extra ? extra->n : 0;
    int32_t* pr = (int32_t*)malloc(sizeof(int32_t) * 2 * (16 * (size_t)nt + nv + (size_t)nx));
    int64_t np = 0;
    for (int v = 0; v < nv; ++v) { pr[2 * np] = v; pr[2 * np + 1] = v; ++np; }
    for (int64_t e = 0; e < nx; ++e) { pr[2 * np] = extra->a[2 * e]; pr[2 * np + 1] = extra->a[2 * e + 1]; ++np; }
    for (int t = 0; t < nt; ++t)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b) { pr[2 * np] = tets[4 * t + a]; pr[2 * np + 1] = tets[4 * t + b]; ++np; }
    qsort(pr, (size_t)np, 2 * sizeof(int32_t), cmp_pair);
    s->rp = (int32_t*)calloc((size_t)nv + 1, sizeof(int32_t));
    s->ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)np);
    int64_t u = 0;
    for (int64_t i = 0; i < np; ++i) {
        if (i > 0 && pr[2 * i] == pr[2 * (i - 1)] && pr[2 * i + 1] == pr[2 * (i - 1) + 1]) continue;
        s->ci[u++] = pr[2 * i + 1]; s->rp[pr[2 * i] + 1]++;
    }
    for (int v = 0; v < nv; ++v) s->rp[v + 1] += s->rp[v];
    s->nnzb = u;
    free(pr);
    s->xm = (double*)malloc(sizeof(double) * 3 * (size_t)sc->nmv);
    memcpy(s->xm, sc->Y0, sizeof(double) * 3 * (size_t)sc->nmv);
    return s;
}

ORC_API void orc_sim_free(orc_sim* s) {
    if (!s) return;
    free(s->Dminv); free(s->vol); free(s->mass); free(s->rp); free(s->ci); free(s->xm);
    free(s->Xsys); free(s->Tsys); free(s->Dsys); free(s->fext); free(s);
}
ORC_API int64_t orc_sim_nnzb(const orc_sim* s) { return s->nnzb; }
ORC_API void orc_sim_mass(const orc_sim* s, double* out) { memcpy(out, s->mass, sizeof(double) * s->nv); }
ORC_API void orc_sim_set_master(orc_sim* s, const double* xm) {
    memcpy(s->xm, xm, sizeof(double) * 3 * (size_t)s->sc->nmv);
}

static int64_t blk_index(const orc_sim* s, int i, int j) {
    int lo = s->rp[i], hi = s->rp[i + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (s->ci[mid] == j) return mid;
        if (s->ci[mid] < j) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* elastic energy (and gradient / blocks when non-NULL); returns 0 if some tet
 * has J <= 0 */
static int elastic_eval(const orc_sim* s, const double* x, double* E, double* grad, double* blk) {
    double e = 0.0;
    for (int t = 0; t < s->nt; ++t) {
        const int32_t* T = s->tets + 4 * t;
        double x4[12], X4[12], psi, g12[12], h144[144];
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) { x4[3 * a + c] = x[3 * T[a] + c]; X4[3 * a + c] = s->X[3 * T[a] + c]; }
        if (!orc_nh_tet(s->Dminv + 9 * t, s->vol[t], s->mu, s->lam, X4, x4, &psi, grad ? g12 : NULL,
                        blk ? h144 : NULL)) { *E = INFINITY; return 0; }
        e += psi;
        if (grad) for (int a = 0; a < 4; ++a) for (int c = 0; c < 3; ++c) grad[3 * T[a] + c] += g12[3 * a + c];
        if (blk)
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) {
                    int64_t k = blk_index(s, T[a], T[b]);
                    for (int p = 0; p < 3; ++p)
                        for (int q = 0; q < 3; ++q) blk[9 * k + 3 * p + q] += h144[(3 * a + p) * 12 + 3 * b + q];
                }
    }
    *E = e;
    return 1;
}

static double vdot(int n, const double* a, const double* b) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void spmv(const orc_sim* s, const double* A, const double* x, double* y) {
    for (int i = 0; i < s->nv; ++i) {
        double acc[3] = {0, 0, 0};
        for (int k = s->rp[i]; k < s->rp[i + 1]; ++k) {
            const double* B = A + 9 * (size_t)k;
            const double* xj = x + 3 * (size_t)s->ci[k];
            for (int p = 0; p < 3; ++p) acc[p] += B[3 * p] * xj[0] + B[3 * p + 1] * xj[1] + B[3 * p + 2] * xj[2];
        }
        for (int p = 0; p < 3; ++p) y[3 * i + p] = acc[p];
    }
}

/* block-Jacobi preconditioned CG for A p = b; returns iterations */
static int pcg(const orc_sim* s, const double* A, const double* b, double* x, double rel_tol, int max_it) {
    int n = 3 * s->nv;
    double *r = (double*)malloc(sizeof(double) * n), *z = (double*)malloc(sizeof(double) * n);
    double *p = (double*)malloc(sizeof(double) * n), *Ap = (double*)malloc(sizeof(double) * n);
    double* Pinv = (double*)malloc(sizeof(double) * 9 * (size_t)s->nv);
    for (int i = 0; i < s->nv; ++i) inv3(A + 9 * (size_t)blk_index(s, i, i), Pinv + 9 * (size_t)i);
    for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
    double bn = sqrt(vdot(n, b, b));
    int it = 0;
    if (bn > 0.0) {
        for (int i = 0; i < s->nv; ++i)
            for (int q = 0; q < 3; ++q)
                z[3 * i + q] = Pinv[9 * i + 3 * q] * r[3 * i] + Pinv[9 * i + 3 * q + 1] * r[3 * i + 1] + Pinv[9 * i + 3 * q + 2] * r[3 * i + 2];
        memcpy(p, z, sizeof(double) * n);
        double rz = vdot(n, r, z);
        for (it = 0; it < max_it; ++it) {
            spmv(s, A, p, Ap);
            double pAp = vdot(n, p, Ap);
            if (!(pAp > 0.0)) break;
            double al = rz / pAp;
            for (int i = 0; i < n; ++i) { x[i] += al * p[i]; r[i] -= al * Ap[i]; }
            if (sqrt(vdot(n, r, r)) <= rel_tol * bn) { ++it; break; }
            for (int i = 0; i < s->nv; ++i)
                for (int q = 0; q < 3; ++q)
                    z[3 * i + q] = Pinv[9 * i + 3 * q] * r[3 * i] + Pinv[9 * i + 3 * q + 1] * r[3 * i + 1] + Pinv[9 * i + 3 * q + 2] * r[3 * i + 2];
            double rz2 = vdot(n, r, z);
            double be = rz2 / rz;
            rz = rz2;
            for (int i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
        }
    }
    free(r); free(z); free(p); free(Ap); free(Pinv);
    return it;
}

/* total incremental potential at x_i: E, gradient G (Dirichlet rows zero),
 * blocks A (Dirichlet rows/cols identity) and the frozen active samples */
static int newton_eval(const orc_sim* s, const double* x, const double* xhat, double* E, double* G,
                       double* A, svec* samples) {
    int nv = s->nv;
    double h2 = s->h * s->h;
    memset(G, 0, sizeof(double) * 3 * nv);
    if (A) memset(A, 0, sizeof(double) * 9 * (size_t)s->nnzb);
    double Ee;
    if (!elastic_eval(s, x, &Ee, G, A)) return 0;
    for (int i = 0; i < 3 * nv; ++i) G[i] *= h2;
    if (A) for (int64_t i = 0; i < 9 * s->nnzb; ++i) A[i] *= h2;
    double Ein = 0.0;
    for (int i = 0; i < nv; ++i)
        for (int c = 0; c < 3; ++c) {
            double d = x[3 * i + c] - xhat[3 * i + c];
            Ein += 0.5 * s->mass[i] * d * d;
            G[3 * i + c] += s->mass[i] * d;
        }
    if (A) for (int i = 0; i < nv; ++i) { int64_t k = blk_index(s, i, i); for (int c = 0; c < 3; ++c) A[9 * k + 4 * c] += s->mass[i]; }
    /* external forces (joint step): -h^2 f.(x - xhat), the work -h^2 f.x
     * up to a constant of the step (same gradient and minimiser; relative to
     * xhat it stays small, so its rounding does not swamp the line search) */
    double Ef = 0.0;
    if (s->fext)
        for (int i = 0; i < 3 * nv; ++i) { Ef -= s->fext[i] * (x[i] - xhat[i]); G[i] -= h2 * s->fext[i]; }
    samples->n = 0;
    const double* xm = s->joint ? x + 3 * (size_t)s->npad : s->xm;
    collect_samples(s->sc, x, xm, 0, NULL, samples);
    double Ec = 0.0;
    for (int64_t q = 0; q < samples->n; ++q) {
        const orc_sample* k = samples->a + q;
        double B, dB, d2B;
        orc_barrier(k->g, k->eps, &B, &dB, &d2B);
        double coef = k->kq * k->w * k->gamma;
        Ec += coef * B;
        double c1 = coef * dB, c2 = dmax(coef * d2B, 0.0);
        const int* T = k->sv;
        for (int a = 0; a < 3; ++a) {
            if (T[a] < 0) continue;
            for (int c = 0; c < 3; ++c) G[3 * T[a] + c] += h2 * (-c1 * k->bs[a] * k->ns[c]);
            if (A)
                for (int b = 0; b < 3; ++b) {
                    if (T[b] < 0) continue;
                    int64_t bi = blk_index(s, T[a], T[b]);
                    for (int p = 0; p < 3; ++p)
                        for (int qq = 0; qq < 3; ++qq) A[9 * bi + 3 * p + qq] += h2 * c2 * k->bs[a] * k->bs[b] * k->ns[p] * k->ns[qq];
                }
        }
        if (!s->joint) continue;
        /* deformable master: the gap gradient is bm_j n_s on master vertex
         * j; its rows and its blocks with the slave and master vertices */
        for (int j = 0; j < 3; ++j) {
            if (k->mv[j] < 0) continue;
            const int mj = s->npad + k->mv[j];
            for (int c = 0; c < 3; ++c) G[3 * mj + c] += h2 * c1 * k->bm[j] * k->ns[c];
            if (!A) continue;
            for (int r = 0; r < 6; ++r) {
                int row;
                double wr;
                if (r < 3) { if (T[r] < 0) continue; row = T[r]; wr = -k->bs[r]; }
                else { if (k->mv[r - 3] < 0) continue; row = s->npad + k->mv[r - 3]; wr = k->bm[r - 3]; }
                const int64_t b1 = blk_index(s, row, mj), b2 = blk_index(s, mj, row);
                if (b1 < 0 || b2 < 0) { fprintf(stderr, "orc: contact block outside the pattern\n"); abort(); }
                for (int p = 0; p < 3; ++p)
                    for (int qq = 0; qq < 3; ++qq) {
                        const double v = h2 * c2 * wr * k->bm[j] * k->ns[p] * k->ns[qq];
                        A[9 * b1 + 3 * p + qq] += v;
                        if (r < 3) A[9 * b2 + 3 * p + qq] += v;   /* its transpose (n n^T is symmetric) */
                    }
            }
        }
    }
    *E = Ein + h2 * (Ee + Ec + Ef);
    for (int i = 0; i < nv; ++i)
        if (s->dir[i]) {
            for (int c = 0; c < 3; ++c) G[3 * i + c] = 0.0;
            if (A)
                for (int k = s->rp[i]; k < s->rp[i + 1]; ++k) {
                    int j = s->ci[k];
                    memset(A + 9 * (size_t)k, 0, 9 * sizeof(double));
                    if (j == i) { A[9 * (size_t)k] = 1.0; A[9 * (size_t)k + 4] = 1.0; A[9 * (size_t)k + 8] = 1.0; }
                    else { int64_t kt = blk_index(s, j, i); memset(A + 9 * kt, 0, 9 * sizeof(double)); }
                }
        }
    return 1;
}

/* change of the lagged energy from x_i to x_i + a p (reading R22):
 *   dE = sum_v m_v (a p_v.(x_v - xhat_v) + a^2/2 |p_v|^2)
 *      + h^2 ( sum_tets [psi(x + a p) - psi(x)]
 *            + sum_k kappa w gamma [B(g + a dg) - B(g)]  -  a f.p ),
 * each term's change formed on its own before the sums, so that the test
 * against the predicted decrease is not lost in the rounding of the total
 * energy; +inf if a tet inverts or a sample's gap reaches 0 */
static double lagged_delta(const orc_sim* s, const double* x, const double* xhat, const svec* smp,
                           const double* p, double a) {
    const int nv = s->nv;
    double dEe = 0.0;
    for (int t = 0; t < s->nt; ++t) {
        const int32_t* T = s->tets + 4 * t;
        double x4[12], y4[12], X4[12], psi0, psi1;
        for (int q = 0; q < 4; ++q)
            for (int c = 0; c < 3; ++c) {
                x4[3 * q + c] = x[3 * T[q] + c];
                y4[3 * q + c] = x[3 * T[q] + c] + a * p[3 * T[q] + c];
                X4[3 * q + c] = s->X[3 * T[q] + c];
            }
        if (!orc_nh_tet(s->Dminv + 9 * t, s->vol[t], s->mu, s->lam, X4, y4, &psi1, NULL, NULL)) return INFINITY;
        orc_nh_tet(s->Dminv + 9 * t, s->vol[t], s->mu, s->lam, X4, x4, &psi0, NULL, NULL);
        dEe += psi1 - psi0;
    }
    double dEin = 0.0;
    for (int i = 0; i < nv; ++i)
        for (int c = 0; c < 3; ++c) {
            const double pc = p[3 * i + c];
            dEin += s->mass[i] * (a * pc * (x[3 * i + c] - xhat[3 * i + c]) + 0.5 * a * a * pc * pc);
        }
    double dEc = 0.0;
    const double* pm = s->joint ? p + 3 * (size_t)s->npad : NULL;
    for (int64_t q = 0; q < smp->n; ++q) {
        const orc_sample* k = smp->a + q;
        double gt = k->g + a * sample_dgdx(s->sc, k, p, pm);
        if (!(gt > 0.0)) return INFINITY;
        double B1, B0, dB, d2B;
        orc_barrier(gt, k->eps, &B1, &dB, &d2B);
        orc_barrier(k->g, k->eps, &B0, &dB, &d2B);
        dEc += k->kq * k->w * k->gamma * (B1 - B0);
    }
    double dEf = 0.0;
    if (s->fext)
        for (int i = 0; i < 3 * nv; ++i) dEf -= a * s->fext[i] * p[i];
    return dEin + s->h * s->h * (dEe + dEc + dEf);
}

static double max_step_to(const orc_sim* s, const double* x, const double* dP) {
    if (!s->joint) return orc_ccd_max_step(s->sc, x, dP, s->xm, NULL, s->slack, s->ccd_max_iter, NULL, NULL);
    /* both bodies move: the master part of x and dP is its motion */
    const double* xm = x + 3 * (size_t)s->npad;
    const double* dm = dP + 3 * (size_t)s->npad;
    orc_accd_info info;
    const double al = orc_alpha_lin(s->sc, x, xm, dP, dm);
    const double aa = orc_accd_min(s->sc, x, dP, xm, dm, s->slack, s->ccd_max_iter, &info);
    return dmin(1.0, dmin(al, aa));
}

/* start point: Dirichlet vertices at xhat, free vertices moved toward P by
 * the CCD-limited fraction, halved until every tet keeps J > 0 */
static int start_point(const orc_sim* s, const double* x, const double* xhat, const double* P,
                       double* x0, double* alpha0) {
    int nv = s->nv;
    double* xi = (double*)malloc(sizeof(double) * 3 * nv);
    double* dP = (double*)calloc(3 * (size_t)nv, sizeof(double));
    int has_dir = 0;
    for (int i = 0; i < nv; ++i) if (s->dir[i]) { has_dir = 1; for (int c = 0; c < 3; ++c) dP[3 * i + c] = xhat[3 * i + c] - x[3 * i + c]; }
    memcpy(xi, x, sizeof(double) * 3 * nv);
    double Ed;
    if (has_dir) {
        if (max_step_to(s, x, dP) < 1.0) { free(xi); free(dP); return 0; }
        for (int i = 0; i < nv; ++i) if (s->dir[i]) for (int c = 0; c < 3; ++c) xi[3 * i + c] = xhat[3 * i + c];
        if (!elastic_eval(s, xi, &Ed, NULL, NULL)) { free(xi); free(dP); return 0; }
    }
    for (int i = 0; i < nv; ++i)
        for (int c = 0; c < 3; ++c) dP[3 * i + c] = s->dir[i] ? 0.0 : P[3 * i + c] - xi[3 * i + c];
    double a = max_step_to(s, xi, dP);
    for (int hv = 0;; ++hv) {
        for (int i = 0; i < 3 * nv; ++i) x0[i] = xi[i] + a * dP[i];
        if (elastic_eval(s, x0, &Ed, NULL, NULL)) break;
        if (hv >= s->max_halv) { free(xi); free(dP); return 0; }
        a *= 0.5;
    }
    *alpha0 = a;
    free(xi); free(dP);
    return 1;
}

static double free_norm(const orc_sim* s, const double* G) {
    double q = 0.0;
    for (int i = 0; i < s->nv; ++i) if (!s->dir[i]) for (int c = 0; c < 3; ++c) q += G[3 * i + c] * G[3 * i + c];
    return sqrt(q);
}

/* One implicit-Euler step (reading R7): x, v in/out; xm_next the master at
 * t+1 (NULL: unchanged); dx_pred the learned displacement (NULL: x + h v).
 * Convergence: ||G_free(x)|| <= tol * max(||G_free(x~)||, floor), x~ the
 * CCD-filtered plain predictor (reading R8). */
ORC_API int orc_newton_step(orc_sim* s, double* x, double* v, const double* xm_next,
                            const double* dx_pred, orc_stats* st) {
    int nv = s->nv, n = 3 * nv;
    memset(st, 0, sizeof(*st));
    double h = s->h;
    double *xhat = (double*)malloc(sizeof(double) * n), *xt = (double*)malloc(sizeof(double) * n);
    double *G = (double*)malloc(sizeof(double) * n), *p = (double*)malloc(sizeof(double) * n);
    double *tmp = (double*)malloc(sizeof(double) * n), *P = (double*)malloc(sizeof(double) * n);
    double* A = (double*)malloc(sizeof(double) * 9 * (size_t)s->nnzb);
    svec smp = {0, 0, 0};
    memcpy(xt, x, sizeof(double) * n);
    for (int i = 0; i < nv; ++i) for (int c = 0; c < 3; ++c) xhat[3 * i + c] = x[3 * i + c] + h * v[3 * i + c] + h * h * s->grav[c];
    int status = 0;
    /* master motion with the pad held at x^t (kinematic master only) */
    if (xm_next && !s->joint) {
        double* z = (double*)calloc((size_t)n, sizeof(double));
        double a = orc_ccd_max_step(s->sc, x, z, s->xm, xm_next, s->slack, s->ccd_max_iter, NULL, NULL);
        free(z);
        if (a < 1.0) { status = 3; goto done; }
        memcpy(s->xm, xm_next, sizeof(double) * 3 * (size_t)s->sc->nmv);
    }
    /* residual scale from the CCD-filtered plain predictor */
    double a0, Etmp, gscale;
    if (!start_point(s, x, xhat, xhat, tmp, &a0)) { status = 3; goto done; }
    if (!newton_eval(s, tmp, xhat, &Etmp, G, NULL, &smp)) { status = 3; goto done; }
    gscale = free_norm(s, G);
    /* a predicted start is admitted through the same CCD-filtered start
     * point, and kept only if its residual is not worse than the plain
     * predictor's (reading R16) */
    {
        int use_pred = 0;
        if (dx_pred) {
            double* xl = (double*)malloc(sizeof(double) * n);
            double al;
            for (int i = 0; i < n; ++i) P[i] = x[i] + dx_pred[i];
            if (start_point(s, x, xhat, P, xl, &al) && newton_eval(s, xl, xhat, &Etmp, G, NULL, &smp) &&
                free_norm(s, G) <= gscale) {
                memcpy(x, xl, sizeof(double) * n);
                a0 = al;
                use_pred = 1;
            }
            free(xl);
        }
        if (!use_pred) memcpy(x, tmp, sizeof(double) * n);
        st->pred_used = use_pred;
    }
    st->alpha0 = a0;
    st->res0 = gscale;
    {
        /* floor: force of a 1e-3 strain on one element, h^2 E lbar^2 1e-3,
         * lbar = cube root of the mean tet volume */
        double vsum = 0.0;
        for (int t = 0; t < s->nt; ++t) vsum += s->vol[t];
        double lbar = cbrt(vsum / (double)s->nt);
        gscale = dmax(gscale, 1e-3 * h * h * s->E * lbar * lbar);
    }
    for (int it = 0;; ++it) {
        double E;
        if (!newton_eval(s, x, xhat, &E, G, A, &smp)) { status = 3; break; }
        st->energy = E;
        st->residual = free_norm(s, G) / gscale;
        if (g_verbose) fprintf(stderr, "  it %d E %.6e res %.3e nsamp %lld\n", it, E, st->residual, (long long)smp.n);
        if (st->residual <= s->tol) break;
        if (it >= s->max_newton) { status = 5; break; }
        st->newton_iters = it + 1;
        for (int i = 0; i < n; ++i) tmp[i] = -G[i];
        st->pcg_iters_total += pcg(s, A, tmp, p, s->pcg_tol, s->max_pcg);
        for (int i = 0; i < nv; ++i) if (s->dir[i]) for (int c = 0; c < 3; ++c) p[3 * i + c] = 0.0;
        double gp = vdot(n, G, p);
        double al = max_step_to(s, x, p);
        if (g_verbose) {
            double a_l = orc_alpha_lin(s->sc, x, s->xm, p, NULL);
            orc_accd_info inf;
            orc_accd_min(s->sc, x, p, s->xm, NULL, s->slack, s->ccd_max_iter, &inf);
            fprintf(stderr, "     gp %.3e alpha %.3e (lin %.3e accd sv-mt %.3e mv-st %.3e ee %.3e)\n", gp, al, a_l,
                    inf.alpha_type[0], inf.alpha_type[1], inf.alpha_type[2]);
        }
        double c0 = 1e-4;
        int ok = 0;
        for (int hv = 0; hv <= s->max_halv; ++hv) {
            double dE = lagged_delta(s, x, xhat, &smp, p, al);
            if (dE <= c0 * al * gp) { ok = 1; break; }
            al *= 0.5;
        }
        if (!ok) { status = 6; break; }
        st->last_alpha = al;
        for (int i = 0; i < n; ++i) x[i] = x[i] + al * p[i];
    }
    if (status == 0 || status == 5)
        for (int i = 0; i < n; ++i) v[i] = (x[i] - xt[i]) / h;
done:
    if (status != 0 && status != 5) memcpy(x, xt, sizeof(double) * n);
    st->status = status;
    free(xhat); free(xt); free(G); free(p); free(tmp); free(P); free(A); free(smp.a);
    return status;
}

/* dense symmetric system for tests: assemble A (free DOFs only) and G at x */
ORC_API int orc_newton_system(orc_sim* s, const double* x, const double* v, double* E, double* G,
                              double* Ablk) {
    int n = 3 * s->nv;
    double* xhat = (double*)malloc(sizeof(double) * n);
    for (int i = 0; i < s->nv; ++i) for (int c = 0; c < 3; ++c) xhat[3 * i + c] = x[3 * i + c] + s->h * v[3 * i + c] + s->h * s->h * s->grav[c];
    svec smp = {0, 0, 0};
    int ok = newton_eval(s, x, xhat, E, G, Ablk, &smp);
    free(xhat); free(smp.a);
    return ok;
}
ORC_API void orc_sim_pattern(const orc_sim* s, int32_t* rp, int32_t* ci) {
    memcpy(rp, s->rp, sizeof(int32_t) * ((size_t)s->nv + 1));
    memcpy(ci, s->ci, sizeof(int32_t) * (size_t)s->nnzb);
}
ORC_API int orc_pcg_solve(const orc_sim* s, const double* A, const double* b, double* x, double tol, int max_it) {
    return pcg(s, A, b, x, tol, max_it);
}

/* ------------------------------------------------------------------------
 * Dual-mesh mapper, Sec. 3.2 (Eqs. bary_proj, decomp, gram, bary_interp).
 *
 * Precomputation: every visual vertex p is embedded on the simulation
 * surface.  Its triangle is the nearest one (smallest point-triangle
 * distance, orc_pt_dist2; on a tie the lowest index).  With e1 = v1 - v0,
 * e2 = v2 - v0, n = e1 x e2 / |e1 x e2| and d = p - v0, the offset is
 * delta = d . n (Eq. decomp), and (v, w) solve the 2x2 Gram system of
 * Eq. (gram), written out by Cramer's rule; u = 1 - v - w.
 * Per-frame update: p' = u v0' + v v1' + w v2' + delta n' (Eq. bary_interp),
 * n' the unit normal of the deformed triangle.
 * ------------------------------------------------------------------------ */
ORC_API void orc_dual_map_coords(const double* p, const double* v0, const double* v1, const double* v2,
                                 double* uvwd) {
    double e1[3], e2[3], n[3], d[3];
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    const double len = sqrt(dot3(n, n));
    for (int c = 0; c < 3; ++c) n[c] = n[c] / len;
    sub3(p, v0, d);
    const double g11 = dot3(e1, e1), g12 = dot3(e1, e2), g22 = dot3(e2, e2);
    const double r1 = dot3(d, e1), r2 = dot3(d, e2);
    const double det = g11 * g22 - g12 * g12;
    const double v = (r1 * g22 - g12 * r2) / det;
    const double w = (g11 * r2 - g12 * r1) / det;
    uvwd[0] = 1.0 - v - w;
    uvwd[1] = v;
    uvwd[2] = w;
    uvwd[3] = dot3(d, n);
}

ORC_API void orc_dual_map_build(const double* V, const int32_t* T, int64_t nt, const double* P, int64_t np,
                                int32_t* tri, double* uvwd, double* dist2) {
    for (int64_t i = 0; i < np; ++i) {
        const double* p = P + 3 * i;
        double best = INFINITY;
        int64_t bt = -1;
        for (int64_t t = 0; t < nt; ++t) {
            const int32_t* F = T + 3 * t;
            const double d2 = orc_pt_dist2(p, V + 3 * F[0], V + 3 * F[1], V + 3 * F[2]);
            if (d2 < best) { best = d2; bt = t; }
        }
        tri[i] = (int32_t)bt;
        if (dist2) dist2[i] = best;
        if (bt < 0) { uvwd[4 * i] = uvwd[4 * i + 1] = uvwd[4 * i + 2] = uvwd[4 * i + 3] = NAN; continue; }
        const int32_t* F = T + 3 * bt;
        orc_dual_map_coords(p, V + 3 * F[0], V + 3 * F[1], V + 3 * F[2], uvwd + 4 * i);
    }
}

ORC_API void orc_dual_map_apply(const double* V, const int32_t* T, const int32_t* tri, const double* uvwd,
                                int64_t np, double* out) {
    for (int64_t i = 0; i < np; ++i) {
        const int32_t* F = T + 3 * (int64_t)tri[i];
        const double *v0 = V + 3 * F[0], *v1 = V + 3 * F[1], *v2 = V + 3 * F[2];
        double e1[3], e2[3], n[3];
        sub3(v1, v0, e1);
        sub3(v2, v0, e2);
        cross3(e1, e2, n);
        const double len = sqrt(dot3(n, n));
        const double* c4 = uvwd + 4 * i;
        for (int c = 0; c < 3; ++c)
            out[3 * i + c] = c4[0] * v0[c] + c4[1] * v1[c] + c4[2] * v2[c] + c4[3] * (n[c] / len);
    }
}

/* ------------------------------------------------------------------------
 * Paper-exact face samples, Sec. 4.1 "Face samples": both triangles are
 * projected onto the tangent plane of the slave triangle T_s, the projected
 * master triangle is clipped by T_s (Sutherland-Hodgman), the clipped polygon
 * is fan-triangulated from its first vertex, and each sub-triangle gets the
 * 3-point, degree-2 Gauss rule (interior points with barycentric coordinates
 * (2/3, 1/6, 1/6) and permutations, weight one third of the area; reading
 * R18).  Each sample is a point x_s on T_s (slave barycentrics beta^s); it
 * is cast along the slave normal n_s onto the master plane, which gives the
 * gap g (Eq. gap) and the master barycentrics beta^m (Eq. gram).
 *
 * Plane coordinates: origin x_s0, t1 = (x_s1 - x_s0)/|.|, t2 = n_s x t1,
 * n_s = (x_s1 - x_s0) x (x_s2 - x_s0) normalised; T_s is counter-clockwise
 * there.  Output per sample, 8 doubles: beta^s[3], beta^m[3], g, w.
 * Returns the sample count (0 when the overlap has no area or the master
 * plane is parallel to n_s), at most 12.
 * ------------------------------------------------------------------------ */
static double cross2(const double* a, const double* b, const double* p) {
    return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0]);
}

ORC_API int orc_face_clip_samples(const double* xs, const double* xm, double* out) {
    const double *s0 = xs, *s1 = xs + 3, *s2 = xs + 6;
    double e1[3], e2[3], n[3], t1[3], t2[3];
    sub3(s1, s0, e1);
    sub3(s2, s0, e2);
    cross3(e1, e2, n);
    const double nl = sqrt(dot3(n, n));
    for (int c = 0; c < 3; ++c) n[c] = n[c] / nl;
    const double l1 = sqrt(dot3(e1, e1));
    for (int c = 0; c < 3; ++c) t1[c] = e1[c] / l1;
    cross3(n, t1, t2);
    /* slave triangle and projected master triangle in plane coordinates */
    double A[3][2], P[3][2];
    for (int k = 0; k < 3; ++k) {
        double d[3];
        sub3(xs + 3 * k, s0, d);
        A[k][0] = dot3(d, t1); A[k][1] = dot3(d, t2);
        sub3(xm + 3 * k, s0, d);
        P[k][0] = dot3(d, t1); P[k][1] = dot3(d, t2);
    }
    /* Sutherland-Hodgman: keep the part on the left of each directed edge */
    double poly[12][2], tmp[12][2];
    int m = 3;
    for (int k = 0; k < 3; ++k) { poly[k][0] = P[k][0]; poly[k][1] = P[k][1]; }
    for (int e = 0; e < 3 && m > 0; ++e) {
        const double* a = A[e];
        const double* b = A[(e + 1) % 3];
        int mo = 0;
        for (int k = 0; k < m; ++k) {
            const double* p = poly[(k + m - 1) % m];
            const double* q = poly[k];
            const double sp = cross2(a, b, p), sq = cross2(a, b, q);
            if (sq >= 0.0) {
                if (sp < 0.0) {
                    const double t = sp / (sp - sq);
                    tmp[mo][0] = p[0] + t * (q[0] - p[0]); tmp[mo][1] = p[1] + t * (q[1] - p[1]); ++mo;
                }
                tmp[mo][0] = q[0]; tmp[mo][1] = q[1]; ++mo;
            } else if (sp >= 0.0) {
                const double t = sp / (sp - sq);
                tmp[mo][0] = p[0] + t * (q[0] - p[0]); tmp[mo][1] = p[1] + t * (q[1] - p[1]); ++mo;
            }
        }
        m = mo;
        for (int k = 0; k < m; ++k) { poly[k][0] = tmp[k][0]; poly[k][1] = tmp[k][1]; }
    }
    if (m < 3) return 0;
    /* master plane */
    double f1[3], f2[3], N[3];
    sub3(xm + 3, xm, f1);
    sub3(xm + 6, xm, f2);
    cross3(f1, f2, N);
    const double den = dot3(N, n);
    if (den == 0.0) return 0;
    /* slave barycentrics of a plane point: 2x2 solve in the plane */
    const double a11 = A[1][0] - A[0][0], a12 = A[2][0] - A[0][0];
    const double a21 = A[1][1] - A[0][1], a22 = A[2][1] - A[0][1];
    const double det = a11 * a22 - a12 * a21;
    static const double G[3][3] = {{2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0},
                                   {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0},
                                   {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}};
    int ns = 0;
    for (int k = 1; k + 1 < m; ++k) {
        const double *q0 = poly[0], *q1 = poly[k], *q2 = poly[k + 1];
        const double area = 0.5 * fabs((q1[0] - q0[0]) * (q2[1] - q0[1]) - (q1[1] - q0[1]) * (q2[0] - q0[0]));
        if (!(area > 0.0)) continue;
        for (int gp = 0; gp < 3; ++gp) {
            const double u = G[gp][0] * q0[0] + G[gp][1] * q1[0] + G[gp][2] * q2[0];
            const double v = G[gp][0] * q0[1] + G[gp][1] * q1[1] + G[gp][2] * q2[1];
            const double ru = u - A[0][0], rv = v - A[0][1];
            const double b1 = (a22 * ru - a12 * rv) / det;
            const double b2 = (a11 * rv - a21 * ru) / det;
            double* o = out + 8 * ns;
            o[0] = 1.0 - b1 - b2; o[1] = b1; o[2] = b2;
            double x[3], d[3], hit[3];
            for (int c = 0; c < 3; ++c) x[c] = o[0] * s0[c] + o[1] * s1[c] + o[2] * s2[c];
            sub3(xm, x, d);
            const double g = dot3(N, d) / den;
            for (int c = 0; c < 3; ++c) hit[c] = x[c] + g * n[c];
            bary_gram(hit, xm, xm + 3, xm + 6, o + 3);
            o[6] = g;
            o[7] = area / 3.0;
            ++ns;
        }
    }
    return ns;
}

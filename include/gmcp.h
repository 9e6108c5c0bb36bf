/*
 * gmcp.h -- C ABI of libgmcp: the per-Newton-iteration contact pass of
 * incremental potential contact under the Geometric Mortar Contact Potential
 * (GMCP) of IsaacIPC (arXiv 2605.24339), on one NVIDIA B300 (sm_103a).
 *
 * Problem statement followed (paper Sec. 2.1 and Sec. 4): minimise
 *   E(x) = 1/2 (x - xhat)^T M (x - xhat) + h^2 (Psi_elastic(x) + Psi_GMCP(x))
 * over the pad positions x, subject to an intersection-free trajectory, with
 *   Psi_GMCP = sum_q sum_k kappa_q w_k gamma_k B(g_k, eps_k)   (Eq. gmcp_potential)
 * over face, edge and point samples of the slave (tactile) surface (Sec. 4.1),
 * gamma from the C1 Hermite step (Sec. 4.3, Eqs. smoothstep, gamma), eps_k the
 * adaptive support radius (Sec. 4.4, Eq. adaptive_eps), B the IPC log barrier
 * -(g-eps)^2 ln(g/eps), and the step bound of Sec. 4.5 (Eqs. ccd, global_ccd)
 * combined with additive CCD.
 *
 * Conventions for every entry point
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; host
 *    pointers are named *_host or are plain structs.  Positions are
 *    contiguous FP64 [n][3] (x, y, z per vertex).
 *  - All GPU work is queued on params.stream (a cudaStream_t; NULL = the
 *    legacy default stream).  Calls that return a host scalar synchronise
 *    that stream.
 *  - Nothing throws across the ABI.  Every call returns an ipc_status; on
 *    failure the text of the error is available from ipc_last_error(ctx)
 *    and caller-owned outputs are left unchanged unless stated otherwise.
 *  - One context per host thread; a context is not reentrant.
 *  - The library has no CPU fallback: a call on a machine without a usable
 *    CUDA device fails with IPC_ERR_CUDA.
 */
#ifndef GMCP_H
#define GMCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IPC_OK = 0,
    IPC_ERR_ARG = 1,            /* invalid argument (NULL, size, layout) */
    IPC_ERR_CUDA = 2,           /* CUDA runtime error or no usable device */
    IPC_ERR_OOM = 3,            /* device allocation failed */
    IPC_ERR_INFEASIBLE = 4,     /* non-positive gap, inverted tet or touching pair */
    IPC_ERR_CAPACITY = 5,       /* a fixed-capacity buffer overflowed */
    IPC_ERR_NOT_CONVERGED = 6,  /* Newton hit max_newton (x holds the last iterate) */
    IPC_ERR_LINESEARCH = 7,     /* backtracking exhausted max_halvings */
    IPC_ERR_TIMEOUT = 8         /* a device loop hit its iteration cap */
} ipc_status;

typedef enum { IPC_PREC_FP64 = 0, IPC_PREC_MIXED = 1 } ipc_precision;

/* Parameters (SI units).  Paper constants: dhat is eps_max of Eq.
 * (adaptive_eps); kappa, kappa_edge, kappa_point are kappa_q for q = face,
 * edge, point in Eq. (gmcp_potential); delta_T, delta_e the transition widths
 * of Sec. 4.3.  face_rule_level L gives 4^L face samples per slave triangle. */
typedef struct {
    int32_t precision;          /* ipc_precision */
    double dhat, kappa, kappa_edge, kappa_point, delta_T, delta_e;
    int32_t face_rule_level;    /* 1 (4 samples/tri) or 2 (16 samples/tri) */
    double h, density, youngs, poisson, gravity[3];
    double newton_tol, pcg_rel_tol;
    int32_t max_newton, max_pcg, max_halvings;
    double ccd_slack;           /* ACCD stop fraction s in (0,1) */
    int32_t ccd_max_iter;       /* ACCD iteration cap per primitive pair */
    double dhat_guard, kappa_guard;  /* primitive guard barrier; kappa_guard 0 = off */
    int32_t device;             /* CUDA device ordinal */
    void* stream;               /* cudaStream_t */
    int32_t use_graphs;         /* 1: replay repeated contact passes and PCG iteration
                                   chunks as captured CUDA graphs (same results) */
    int32_t face_sampler;       /* face samples: 0 = the fixed slave-side rule of
                                   face_rule_level (4^L centroids per slave triangle);
                                   1 = the paper's clipped-overlap rule (Sec. 4.1: the
                                   master triangle projected on the slave plane, clipped
                                   by the slave triangle, fan-triangulated, 3-point Gauss
                                   per sub-triangle; see ipc_face_clip_samples), with face
                                   candidates the (slave tri, master tri) pairs whose boxes
                                   meet within dhat */
} ipc_params;

/* Scene: a batch of independent environments concatenated; indices are
 * global.  All arrays are HOST arrays read during ipc_create only. */
typedef struct {
    int32_t n_env;
    const int64_t* env_vert_off;    /* [n_env+1] pad vertex ranges */
    const int64_t* env_tet_off;     /* [n_env+1] */
    const int64_t* env_stri_off;    /* [n_env+1] slave triangle ranges */
    const int64_t* env_mvert_off;   /* [n_env+1] master vertex ranges */
    const int64_t* env_mtri_off;    /* [n_env+1] master triangle ranges */
    int64_t n_vert, n_tet, n_stri, n_mvert, n_mtri;
    const double* pad_rest;         /* [n_vert][3] rest positions X */
    const int32_t* tets;            /* [n_tet][4] positive volume at rest */
    const int32_t* s_tris;          /* [n_stri][3] slave triangles, normal toward the master */
    const uint8_t* dirichlet;       /* [n_vert] 1 = prescribed vertex */
    const double* m_rest;           /* [n_mvert][3] master positions at t = 0 */
    const int32_t* m_tris;          /* [n_mtri][3] master triangles, outward */
} ipc_scene;

typedef struct ipc_ctx ipc_ctx;

/* Candidate-pair counts of the last broad phase (Sec. 4.1 features). */
typedef struct {
    int64_t face;     /* (slave tri, master tri) pairs */
    int64_t edge;     /* (slave tri, master edge) pairs */
    int64_t point;    /* (slave tri, master vertex) pairs */
    int32_t max_per_tri[3];   /* largest per-triangle list of each kind */
} ipc_candidate_counts;

/* Active-sample counts of the last contact evaluation. */
typedef struct {
    int64_t face, edge, point, guard;
    int64_t face_evaluated;   /* (face sample, candidate) pairs tested */
    int64_t query_tris;       /* slave tris whose grown box reached a non-empty
                                 grid cell (the exact candidate tests ran on these) */
} ipc_sample_counts;

/* View of a context-owned block-sparse (3x3) matrix.  Valid until the next
 * call on the context.  vals is FP64 [nnzb][3][3] (row-major blocks) in
 * IPC_PREC_FP64 and FP32 in IPC_PREC_MIXED. */
typedef struct {
    int64_t n_rows;
    int64_t nnzb;
    const int32_t* row_ptr_dev;     /* [n_rows+1] */
    const int32_t* col_idx_dev;     /* [nnzb] */
    const void* vals_dev;
    int32_t dtype;                  /* 0 = FP64, 1 = FP32 */
} ipc_bsr_view;

typedef struct {
    double alpha;          /* min(1, alpha_lin, alpha_accd) */
    double alpha_lin;      /* Eq. (global_ccd); +inf when no sample closes */
    double alpha_accd;     /* additive CCD minimum over primitive pairs */
    int64_t n_pairs_pt, n_pairs_ee;
    int32_t iter_cap_hit;  /* 1 if some pair stopped at ccd_max_iter.  Pairs run with the
                              smallest bound found so far as their upper time, so a pair whose
                              time of impact lies above the minimum may stop before the cap;
                              the flag then reports the pairs that could set alpha_accd */
    int64_t swept_tris;    /* slave tris whose swept box reached a non-empty grid cell */
} ipc_ccd_info;

typedef struct {
    int32_t newton_iters;          /* Newton iterations taken (solves) */
    int32_t pcg_iters_total;       /* PCG iterations summed over the solves */
    int32_t line_search_halvings;  /* halvings summed over the line searches */
    double residual;       /* final ||G_free|| / max(||G_free(x~)||, floor), x~ the
                              CCD-filtered plain predictor, floor = 1e-3 h^2 E lbar^2
                              (lbar = cube root of the mean tet volume) */
    double res0;           /* ||G_free(x~)|| (before the floor) */
    double alpha0;         /* CCD fraction admitted for the Newton start */
    double last_alpha;     /* step length of the last accepted line search */
    double energy;         /* incremental potential at the final iterate */
    double ms_total;       /* host wall time of the call */
    int32_t pred_used;     /* 1 if dx_pred gave the Newton start (see ipc_newton_step) */
} ipc_step_stats;

/* ---------------------------------------------------------------------- */

/* Create a context on params->device: copies the scene to the device,
 * builds the derived topology (master edges, adjacency, ownership, BSR
 * patterns) and sizes the broad-phase grid from the rest positions.
 * *out receives the context (NULL on failure).  The params are copied. */
ipc_status ipc_create(const ipc_params* params, const ipc_scene* scene, ipc_ctx** out);

/* Release every device and host resource of the context.  NULL is a no-op. */
void ipc_destroy(ipc_ctx* ctx);

/* Text of the last error on this context (never NULL; "" when none).  With
 * ctx == NULL: the last error of a failed ipc_create on this thread. */
const char* ipc_last_error(const ipc_ctx* ctx);

/* Broad phase (spatial hash), Sec. 4.1's features within eps_max = dhat:
 * candidate (slave tri, master tri / edge / vertex) pairs for the
 * configuration x_dev [n_vert][3], xm_dev [n_mvert][3] (device).  Face
 * pairs: some face sample of the slave tri lies in the master tri's box
 * grown by dhat; edge and point pairs: the slave tri's vertex box overlaps
 * the master feature's box grown by dhat.  Pairs never cross environments.
 * The lists are stored in the context, sorted per slave triangle; the
 * per-triangle capacities grow automatically (the query is then repeated).
 * counts (host, may be NULL) receives totals and synchronises the stream. */
ipc_status ipc_candidates(ipc_ctx* ctx, const double* x_dev, const double* xm_dev,
                          ipc_candidate_counts* counts);

/* Copy the last candidate list of kind 0 (face), 1 (edge) or 2 (point) to
 * pairs_host [capacity][2] as (slave tri, master feature) sorted
 * lexicographically; master edges are numbered in the lexicographic order
 * of their (min, max) vertex pairs.  *n_out receives the count; with
 * pairs_host == NULL only the count is returned.  IPC_ERR_CAPACITY if
 * capacity is too small (nothing written).  Synchronous. */
ipc_status ipc_candidates_copy(ipc_ctx* ctx, int32_t kind, int32_t* pairs_host, int64_t capacity,
                               int64_t* n_out);

/* Contact pass at (x_dev, xm_dev), Sec. 4.1-4.4: runs the broad phase,
 * builds the face, edge and point samples and evaluates Eq.
 * (gmcp_potential) with the gradient and the PSD Gauss-Newton Hessian of
 * Sec. 4.2 (per-sample coefficient clamped at zero).
 *  energy_dev  (device FP64 scalar, may be NULL) receives Psi;
 *  energy_host (host, may be NULL) receives Psi and synchronises;
 *  grad_dev    (device, may be NULL) receives dPsi/dx [n_vert][3], FP64 in
 *              IPC_PREC_FP64 and FP32 in IPC_PREC_MIXED (the master is
 *              kinematic: its rows are not formed);
 *  hess        (host struct, may be NULL) receives a view of the contact
 *              Hessian in BSR form over the pad vertices (the pattern holds
 *              every vertex pair of every slave triangle);
 *  counts      (host, may be NULL) receives active-sample counts and
 *              synchronises.
 * Gradient and Hessian are assembled by deterministic gathers (no float
 * atomics): repeated calls give bitwise identical results. */
ipc_status ipc_barrier_eval(ipc_ctx* ctx, const double* x_dev, const double* xm_dev,
                            double* energy_dev, double* energy_host, void* grad_dev,
                            ipc_bsr_view* hess, ipc_sample_counts* counts);

/* Gradient of the contact potential Psi with respect to the master vertex
 * positions: the master rows of two-sided GMCP (Sec. 4.3, Eq. gap).  Each
 * active sample has x_m = sum_j bm_j y_j (face: the master barycentrics of
 * the cast point, Eq. gram; edge: (1 - eta, eta) at its Gauss point; point:
 * the vertex itself) and g = n_s . (x_m - x_s) with n_s and the weights held
 * fixed, as for the slave rows of ipc_barrier_eval, so vertex y_j gets
 * kappa_q w gamma B'(g) bm_j n_s.  The rows of one sample sum to the negative
 * of its slave rows (equal and opposite forces, zero net torque).
 *  x_dev [n_vert][3], xm_dev [n_mvert][3] (device, FP64): the state;
 *  grad_m_dev [n_mvert][3] (device, FP64, caller-owned): overwritten.
 * Samples are evaluated in FP64 in both precision modes; each row is summed
 * in a fixed order (the sample entries sorted by master vertex, then by
 * value), so repeated calls agree bitwise.  Synchronises params.stream. */
ipc_status ipc_master_grad(ipc_ctx* ctx, const double* x_dev, const double* xm_dev, double* grad_m_dev);

/* Hessian blocks of the contact potential that involve master vertices
 * (two-sided GMCP, Sec. 4.2-4.3 with Eq. gap), in the Gauss-Newton form of
 * the slave-slave blocks of ipc_barrier_eval: a sample with slave weights
 * beta_a and master weights bm_j has the gap gradient -beta_a n_s on slave
 * vertex a and bm_j n_s on master vertex j, and adds
 * max(kappa_q w gamma B''(g), 0) w_u w_v n_s n_s^T to the block (u, v).
 * Vertices are numbered jointly: pad vertex i is i, master vertex j is
 * n_vert + j.  Written are the slave-master blocks (row a pad vertex, column
 * a master vertex; their transposes are the master-slave blocks) and the
 * master-master blocks, one entry per sample and vertex pair, unsorted and
 * with repeats (sum repeated (row, col) entries); together with the pad
 * blocks of ipc_barrier_eval every block row sums to zero.
 *  x_dev, xm_dev (device, FP64): the state;
 *  capacity: entries the caller's arrays hold;
 *  ij_dev [capacity][2] int32 (row, col) and blk_dev [capacity][9] FP64
 *  row-major 3x3 (device, caller-owned);
 *  n_host (host): the number of entries.
 * Samples are evaluated in FP64 in both precision modes.  Synchronises
 * params.stream.  IPC_ERR_CAPACITY when *n_host > capacity (nothing past
 * capacity is written; call again with room for *n_host). */
ipc_status ipc_master_hess(ipc_ctx* ctx, const double* x_dev, const double* xm_dev, int64_t capacity,
                           int32_t* ij_dev, double* blk_dev, int64_t* n_host);

/* Largest admissible step for the motion x -> x + alpha dx (pad) and
 * xm0 -> xm0 + alpha (xm1 - xm0) (master; xm1_dev NULL = static master):
 * alpha = min(1, alpha_lin, alpha_accd), alpha_lin from Eqs. (ccd) and
 * (global_ccd) over the active samples at (x, xm0) (rounded down by a
 * relative 1e-10 so that rounding-order differences can only shrink it),
 * alpha_accd the additive-CCD minimum (Li et al. 2021, Alg. 1) over
 * primitive pairs (slave surface vertex / master tri, master vertex / slave
 * tri, slave edge / master edge) whose swept boxes overlap.  alpha_host
 * receives alpha and synchronises; info (host) may be NULL. */
ipc_status ipc_ccd_max_step(ipc_ctx* ctx, const double* x_dev, const double* dx_dev,
                            const double* xm0_dev, const double* xm1_dev, double* alpha_host,
                            ipc_ccd_info* info);

/* One full contact pass for a Newton iteration (Sec. 4.1-4.5 together): the
 * broad phase at (x_dev, xm0_dev) runs once and serves both
 *  - the potential, gradient and Hessian of ipc_barrier_eval (energy_dev,
 *    energy_host, grad_dev, hess, counts: same meaning and may be NULL), and
 *  - the step bound of ipc_ccd_max_step for the motion x -> x + alpha dx_dev,
 *    xm0 -> xm0 + alpha (xm1 - xm0) (xm1_dev NULL = static master; then the
 *    additive CCD reuses the grid of the broad phase).  The linearised-gap
 *    bound of Eq. (ccd) is computed in the same sample kernel.
 * dx_dev may be NULL (no step bound; alpha_host and info are then left
 * untouched).  alpha_host / info (host, may be NULL) receive the bound as in
 * ipc_ccd_max_step; asking for any host output synchronises the stream.
 * Results equal those of ipc_barrier_eval followed by ipc_ccd_max_step. */
ipc_status ipc_contact_pass(ipc_ctx* ctx, const double* x_dev, const double* xm0_dev,
                            const double* xm1_dev, const double* dx_dev, double* energy_dev,
                            double* energy_host, void* grad_dev, ipc_bsr_view* hess,
                            double* alpha_host, ipc_ccd_info* info, ipc_sample_counts* counts);

/* ipc_contact_pass with the pass's per-step inputs in host memory: the
 * positions xs_host and displacements dxs_host ([n_svert][3] FP64, the
 * slave-surface vertices in the order ipc_slave_vertices returns, the only
 * pad vertices the pass reads) are copied to the device and scattered into
 * x_dev and dx_dev (written: x_dev[ids[k]] = xs_host[k]), then the pass runs
 * as ipc_contact_pass(ctx, x_dev, xm0_dev, xm1_dev, dx_dev, ...) with the
 * same outputs.  The displacements' copy runs on a copy stream behind the
 * positions' while the broad phase runs (only the swept query and the
 * sample evaluation read them), and the copies are part of the pass's CUDA
 * graph.  Both host buffers must be page-locked (cudaHostAlloc /
 * cudaHostRegister; else IPC_ERR_ARG) and must not change until the call
 * returns; dxs_host and dx_dev are both given or both NULL (no step bound).
 * The results are bitwise those of the scatter followed by ipc_contact_pass. */
ipc_status ipc_contact_pass_host(ipc_ctx* ctx, const double* xs_host, const double* dxs_host, double* x_dev,
                                 double* dx_dev, const double* xm0_dev, const double* xm1_dev,
                                 double* energy_dev, double* energy_host, void* grad_dev, ipc_bsr_view* hess,
                                 double* alpha_host, ipc_ccd_info* info, ipc_sample_counts* counts);

/* One implicit-Euler time step (paper Sec. 2.1 problem statement): minimises
 *   E(x) = 1/2 (x - xhat)^T M (x - xhat) + h^2 (Psi_NH(x) + Psi_GMCP(x)),
 *   xhat = x^t + h v^t + h^2 gravity,
 * over the free vertices by projected Newton.  Each iteration i evaluates
 * the contact pass at x_i (Sec. 4.1-4.4) and freezes its samples (normal,
 * barycentrics, weight, gamma, eps), so the contact term of the line search
 * is sum kappa w gamma B(g + alpha dg) with the linearised gap change dg;
 * the system H p = -G (H = M + h^2 (PSD elastic + contact), lumped mass,
 * Dirichlet rows and columns eliminated) is solved by block-Jacobi PCG to
 * pcg_rel_tol; the step starts at min(1, alpha_lin, alpha_accd) (Sec. 4.5)
 * and is halved until E_i(x + alpha p) <= E_i(x) + 1e-4 alpha G^T p (at most
 * max_halvings times).  Stops when residual <= newton_tol (see
 * ipc_step_stats).  Elasticity: compressible Neo-Hookean,
 * mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2 per tet with its 9x9
 * dP/dF projected onto the PSD cone.
 * Precision: IPC_PREC_FP64 evaluates every term in FP64; IPC_PREC_MIXED
 * takes the contact terms of the mixed contact pass, FP32 Hessian blocks,
 * matrix and PCG vectors, and the elastic energy, gradient and inversion
 * test in double-float (FP32 pairs, ~48 bits), with energies, residuals
 * and the line-search test summed in FP64.
 *  x_dev [n_vert][3] (device, FP64) holds x^t on entry and x^{t+1} on exit;
 *  v_dev the velocity, updated to (x^{t+1} - x^t) / h; Dirichlet vertices
 *  are moved to x + h v (their motion must be admissible);
 *  xm_next_dev: master at t+1 (NULL = unchanged); the context keeps the
 *  current master, which starts at m_rest;
 *  dx_pred_dev: a predicted displacement; its start point x^t + alpha0
 *  dx_pred (alpha0 the CCD-admissible fraction, halved until every tet keeps
 *  J > 0) replaces the plain predictor's start only if it exists and its
 *  residual ||G_free|| is not larger than the plain start's (NULL: the
 *  plain predictor x^t + h v^t);
 *  stats (host) may be NULL.
 * The first call builds the time-stepper state (tet data, mass, the global
 * block pattern).  The call synchronises params.stream several times per
 * iteration.  Returns IPC_ERR_NOT_CONVERGED after max_newton iterations
 * (x and v then hold the last iterate); on IPC_ERR_INFEASIBLE and
 * IPC_ERR_LINESEARCH x and v are left at x^t, v^t.
 * Environments: each is a time step of its own, as ipc_newton_step_envs
 * describes; the status is IPC_OK when every environment converged, else
 * that of the first environment that did not, and stats (n_env > 1) sums
 * pcg_iters_total, line_search_halvings and energy, takes the largest
 * newton_iters, residual and res0 and the smallest alpha0 and last_alpha,
 * and counts in pred_used the environments that took the prediction. */
ipc_status ipc_newton_step(ipc_ctx* ctx, double* x_dev, double* v_dev, const double* xm_next_dev,
                           const double* dx_pred_dev, ipc_step_stats* stats);

/* Deformable master (Sec. 4.2-4.3 with Eq. gap: the contact potential
 * depends on the master vertices through x_m, so a master body that
 * deforms takes its share of every sample's force and stiffness).  The
 * master vertices of the scene become simulated vertices of a second
 * elastic body (the context's material, density and gravity); its tets
 * index master vertices.  Call before the first time step of the context;
 * ipc_newton_step_joint then steps both bodies in one system. */
typedef struct {
    int64_t n_mtet;
    const int32_t* m_tets;        /* [n_mtet][4] master vertex indices, positive volume at m_rest (host) */
    const uint8_t* m_dirichlet;   /* [n_mvert] 1 = prescribed master vertex; NULL = none (host) */
    double pattern_radius;        /* slave-master block pattern: every (slave triangle vertex,
                                     master triangle vertex) pair whose triangles' rest boxes are
                                     within this distance; 0 = 2 x the larger mean edge length of
                                     the two surfaces + 2 dhat.  Contact between triangles farther
                                     apart at rest fails the step with IPC_ERR_CAPACITY. */
} ipc_master_body;

/* Attach the master body (host arrays, copied).  Single environment.
 * Errors: IPC_ERR_ARG (indices out of range, n_env > 1, or the time-stepper
 * state already built by an earlier step). */
ipc_status ipc_set_master_body(ipc_ctx* ctx, const ipc_master_body* body);

/* One implicit-Euler step of the pad and the deformable master together:
 * the step of ipc_newton_step over the joint system (pad vertices, then
 * master vertices), with the contact rows and blocks of the master vertices
 * (each sample's gap gradient is bm_j n_s on master vertex j, Eq. gap with
 * the frozen linearisation) and, on both bodies, the step bound of Sec. 4.5
 * and the additive CCD with both sides moving.
 *  x_dev, v_dev: device FP64 [n_vert + n_mvert][3], the pad's vertices then
 *  the master's, in and out as for ipc_newton_step (Dirichlet vertices of
 *  either body move to x + h v);
 *  f_ext_dev: external nodal forces, device FP64 [n_vert + n_mvert][3]
 *  (NULL = none); the incremental potential gains -h^2 f.x (written as
 *  -h^2 f.(x - xhat), which differs by a constant of the step);
 *  stats (host) may be NULL.
 * The master rows and blocks are summed in a fixed order (entries sorted by
 * destination, then by value), so the step is deterministic.  Errors as
 * ipc_newton_step, plus IPC_ERR_ARG without ipc_set_master_body and
 * IPC_ERR_CAPACITY when a contact block falls outside the block pattern. */
ipc_status ipc_newton_step_joint(ipc_ctx* ctx, double* x_dev, double* v_dev, const double* f_ext_dev,
                                 ipc_step_stats* stats);

/* The time step of ipc_newton_step for every environment of the scene at
 * once (the paper's batched environments, Sec. 5): each environment has its
 * own incremental potential, residual scale, Newton iterate, PCG solve
 * (stopping per environment), step bound (Sec. 4.5, minimum over its own
 * samples and pairs), line search and stopping.  Every sum and minimum of
 * environment e is the one a context holding that environment alone
 * computes, in the same order, so its result is bit for bit that of
 * stepping it alone with the same parameters.  Environments run side by
 * side: one that has stopped keeps its state while the others iterate.
 * An environment whose master cannot move to xm_next keeps its master pose.
 *  x_dev, v_dev, xm_next_dev, dx_pred_dev: as for ipc_newton_step, for the
 *  whole scene;
 *  stats_host (host [n_env], may be NULL): each environment's statistics;
 *  status_host (host [n_env], may be NULL): each environment's ipc_status
 *  (IPC_OK, IPC_ERR_INFEASIBLE, IPC_ERR_NOT_CONVERGED, IPC_ERR_LINESEARCH);
 *  x and v of an environment follow its own status as for ipc_newton_step.
 * Returns what ipc_newton_step returns. */
ipc_status ipc_newton_step_envs(ipc_ctx* ctx, double* x_dev, double* v_dev, const double* xm_next_dev,
                                const double* dx_pred_dev, ipc_step_stats* stats_host, int32_t* status_host);

/* Autotuner (not part of the method): times full contact passes at (x_dev,
 * xm0_dev) with step dx_dev (may be NULL) for candidate launch shapes -- the
 * persistent broad-phase / CCD grid (2, 4, 8, 16, 32 blocks per SM), then the
 * sample kernel's grid (1, 2, 4, 8, 16 blocks per SM) -- by coordinate
 * search, the median of `reps` passes each (CUDA events), and keeps the
 * fastest in the context.  Results of every entry point are identical for
 * every launch shape (each slave triangle's sums have a fixed order); only
 * the time changes.  Outputs (host, may be NULL): the chosen shapes and the
 * best pass time in ms.  Synchronises. */
ipc_status ipc_autotune(ipc_ctx* ctx, const double* x_dev, const double* xm0_dev, const double* dx_dev,
                        int32_t reps, int32_t* samples_bpsm_out, int32_t* query_bpsm_out, double* ms_out);

/* Set the launch shapes directly (blocks per SM, each in [1, 64]). */
ipc_status ipc_set_launch_shape(ipc_ctx* ctx, int32_t samples_bpsm, int32_t query_bpsm);

/* Capacity of the sample-item buffer of the item-parallel evaluation (items
 * = face candidates x samples + 2 x edge candidates + point candidates).  A
 * set of items larger than the capacity is evaluated by the warp-per-
 * triangle kernel instead, with the same results; ipc_contact_pass then
 * grows the buffer for its next calls.  capacity in [1, 2^31 - 1]; the
 * buffers themselves only grow.  Invalidates the captured pass graph. */
ipc_status ipc_set_item_capacity(ipc_ctx* ctx, int64_t capacity);

/* The contact pass reads the pad positions and displacements of the slave
 * (tactile) surface vertices only.  ipc_slave_vertices writes their ids
 * (ascending; ids_host int32 [n], may be NULL) and *n_host their count.
 * Synchronises (a device-to-host copy). */
ipc_status ipc_slave_vertices(ipc_ctx* ctx, int32_t* ids_host, int64_t* n_host);

/* x_dev[ids[k]] = xs_dev[k] (device FP64 [n][3] into [nv][3]) for the slave
 * vertices of ipc_slave_vertices: a caller that streams only the surface
 * positions (or displacements) from the host scatters them into its full
 * device arrays.  Queued on params.stream. */
ipc_status ipc_scatter_slave(ipc_ctx* ctx, const double* xs_dev, double* x_dev);

/* Section profiler (not part of the method): CUDA events recorded on the
 * context stream around each group of launches (grid build, candidate
 * query, sample kernel, gathers, reductions, step bounds).
 *  mode 1: reset the totals and start recording;
 *  mode 0: stop recording;
 *  mode 2: synchronise on the recorded events and report, for up to
 *          max_sections sections, the name (names_host, 32 bytes each,
 *          NUL-terminated), the summed milliseconds (ms_host) and the number
 *          of recorded calls (calls_host); *n_sections receives the count.
 * Recording adds two event records per section and no synchronisation. */
ipc_status ipc_profile(ipc_ctx* ctx, int32_t mode, int32_t max_sections, char* names_host,
                       double* ms_host, int64_t* calls_host, int32_t* n_sections);

/* Allocation-free additive-CCD step bound.  The paper has no counterpart;
 * this entry point exists for callers that must not allocate device memory
 * once they are running -- for example a robot controller's real-time loop,
 * where cudaMalloc may block and synchronise the device, or a host framework
 * that routes every device allocation through its own pool.  Given a context
 * created beforehand, it returns in *alpha_accd_host the same value as the
 * alpha_accd field of ipc_ccd_max_step for the same arguments (additive CCD
 * over the owned primitive pairs whose swept boxes overlap; 1.0 when nothing
 * closes), in n_pairs_host (may be NULL, else 2 entries) the point-triangle
 * and edge-edge pair counts, and in *iter_cap_hit_host (may be NULL) 1 when
 * some pair's additive CCD reached params.ccd_max_iter iterations (its bound
 * is then the last safe time, as in ipc_ccd_max_step's iter_cap_hit), else
 * 0.  It calls no allocator: its scratch is a 4 MiB array built
 * into the library, which every GPU that loads the library keeps until the
 * process exits.  A moving master (xm1_dev != NULL) needs 24 bytes of it per
 * master vertex, so scenes with more than 174,752 master vertices are
 * rejected with IPC_ERR_CAPACITY when xm1_dev is given.  Every call looks up
 * the array's device address with the context's device current (the lookup
 * allocates nothing once the library's module is loaded on that device; the
 * first call on a device may load it, so make that first call before
 * capturing any stream).  Every call on every context of
 * the process uses the same array, clearing it first: calls whose GPU work
 * overlaps (two streams, two threads) race and must be serialised by the
 * caller.  Pairs are enumerated by brute force (slave triangles x master
 * triangles of each environment), so this is meant for small scenes.
 * Synchronises params.stream. */
ipc_status ipc_accd_min_noalloc(ipc_ctx* ctx, const double* x_dev, const double* dx_dev,
                                const double* xm0_dev, const double* xm1_dev,
                                double* alpha_accd_host, int64_t* n_pairs_host, int32_t* iter_cap_hit_host);

/* ---------------------------------------------------------------------- */
/* Learned warm start.  The paper has no learned component; this follows
 * the project's own design: a per-vertex network 32-256-256-256-3 (affine
 * layers, ReLU between them) predicts the correction of the plain
 * predictor,
 *   dx_pred = h v + disp_scale * y(features),
 * and ipc_newton_step admits dx_pred only through its CCD-filtered start
 * (so intersection-freedom never depends on the network).  Weights are kept
 * in FP32 (Adam's master copy) with BF16 copies for the tensor cores; every
 * matrix product has BF16 operands and FP32 accumulation.  Parameters are a
 * flattened FP32 vector of IPC_WS_NPARAM values: W1 [256][32], b1 [256],
 * W2 [256][256], b2, W3 [256][256], b3, W4 [3][256], b4 [3] (row-major).
 *
 * Features (BF16 [n][32] per pad vertex): (x - X)/pos_scale, h v /
 * disp_scale, the rest position mapped to [-1, 1] over the pad's box, the
 * Dirichlet and slave-surface flags, the contact force at x (the negative
 * barrier gradient of the contact pass) / force_scale clamped to +-8, a
 * contact-active flag, sin and cos of pi k Xn (k = 1, 2) per axis, zeros. */
#define IPC_WS_NPARAM 140803

typedef struct {
    const float* params_host;   /* [IPC_WS_NPARAM] initial parameters */
    double lr, beta1, beta2, eps;   /* Adam */
    double pos_scale;           /* m: displacement feature scale */
    double disp_scale;          /* m: per-step displacement scale (features and output) */
    double force_scale;         /* N: contact-force feature scale */
} ipc_ws_params;

/* Create (or replace) the network of the context.  Allocates activations for
 * every pad vertex (about 3 KB per vertex). */
ipc_status ipc_ws_create(ipc_ctx* ctx, const ipc_ws_params* params);

/* Features of state (x_dev, v_dev) with the master at xm_dev (device, FP64
 * [n][3]); runs a contact pass at (x, xm) for the contact force.  They are
 * kept in the context for the next ipc_ws_forward / ipc_ws_grads /
 * ipc_ws_train_step called with feats_dev == NULL; feats_dev (device, may
 * be NULL) also receives a copy, BF16 [n][32].  Synchronises. */
ipc_status ipc_ws_features(ipc_ctx* ctx, const double* x_dev, const double* v_dev, const double* xm_dev,
                           void* feats_dev);

/* Network output y (device FP32 [n][3]) for features feats_dev (BF16
 * [n][32]; NULL = the context's last features).  Synchronises. */
ipc_status ipc_ws_forward(ipc_ctx* ctx, const void* feats_dev, float* out_dev);

/* Loss sum_v m_v |y_v - t_v|^2 / (3 sum_v m_v) for target_dev (FP32 [n][3])
 * and mask_dev (FP32 [n], per-vertex weights), and its gradient with respect
 * to the parameters (grads_host, FP32 [IPC_WS_NPARAM], may be NULL), without
 * updating anything.  Synchronises. */
ipc_status ipc_ws_grads(ipc_ctx* ctx, const void* feats_dev, const float* target_dev, const float* mask_dev,
                        double* loss_host, float* grads_host);

/* One training step: the loss and gradient of ipc_ws_grads, then one Adam
 * update (bias-corrected) of the FP32 parameters and of their BF16 copies.
 * loss_host (may be NULL) receives the loss before the update.  Synchronises. */
ipc_status ipc_ws_train_step(ipc_ctx* ctx, const void* feats_dev, const float* target_dev,
                             const float* mask_dev, double* loss_host);

/* Copy the FP32 parameters to params_host [IPC_WS_NPARAM].  Synchronises. */
ipc_status ipc_ws_get_params(ipc_ctx* ctx, float* params_host);

/* Predicted displacement dx_dev (device FP64 [n][3]) = h v + disp_scale *
 * y(features(x, v, xm)), the dx_pred argument of ipc_newton_step.
 * Synchronises.  IPC_ERR_TIMEOUT if a tensor-core wait reached its cap. */
ipc_status ipc_ws_predict(ipc_ctx* ctx, const double* x_dev, const double* v_dev, const double* xm_dev,
                          double* dx_dev);

/* Kernel launches one ipc_contact_pass makes: the kernel nodes of the CUDA
 * graph the context captured for its last graph-replayed pass (params.use_graphs
 * set), or -1 if no graph is held.  Not part of the method: for launch counts
 * in measurements. */
ipc_status ipc_contact_pass_kernels(ipc_ctx* ctx, int64_t* kernels_host);

/* Measured CUDA-core arithmetic rate of a device (not part of the method: a
 * measurement utility for roofline fractions).  kind 0: FP32 fused
 * multiply-add, kind 1: FP64 fused multiply-add; one FMA counts as two
 * operations.  Runs a kernel of independent FMA chains on every SM of
 * `device` on `stream` (a cudaStream_t, 0 = default), times its second launch
 * with CUDA events and writes TFLOP/s to *tflops_host.  Synchronises the
 * stream; errors through ipc_last_error(NULL). */
ipc_status ipc_alu_peak(int32_t kind, int32_t device, void* stream, double* tflops_host);

/* ------------------------------------------------------------------------
 * Checkpoint and resume (not in the paper: the library's own subsystem).
 * ------------------------------------------------------------------------ */

/* Write a snapshot of a time-stepping context to the file at path: the pad
 * state x_dev, v_dev (device FP64 [n_vert][3], as passed to
 * ipc_newton_step), the kinematic master's current pose (m_rest until the
 * first ipc_newton_step), the number of time steps ipc_newton_step has
 * completed, and, if the context has a network (ipc_ws_create), its FP32
 * parameters, Adam moments, Adam step and settings.  Together with the scene
 * and ipc_params the context was created with, this is everything a time
 * step depends on: a context created from the same scene and parameters and
 * given the snapshot by ipc_load continues bit for bit.  The file has a
 * versioned header, the sizes of the scene and an FNV-1a checksum; it is
 * written beside path and renamed, so a failed write leaves no torn file.
 * Synchronises params.stream.  IPC_ERR_ARG for NULL arguments, a file
 * that cannot be written, or a context with a master body (ipc_set_master_body;
 * not supported). */
ipc_status ipc_save(ipc_ctx* ctx, const char* path, const double* x_dev, const double* v_dev);

/* Read a snapshot written by ipc_save into a context created from the same
 * scene (same sizes) and parameters: x_dev and v_dev (device FP64
 * [n_vert][3]) receive the pad state, the context takes the master pose,
 * the step count (also returned in *step_count_host, may be NULL) and the
 * network (created if the context has none).  Nothing is changed unless the
 * whole file reads and checks: IPC_ERR_ARG for a missing or corrupt file
 * (bad magic, version or checksum) or one written for other sizes.
 * Synchronises params.stream. */
ipc_status ipc_load(ipc_ctx* ctx, const char* path, double* x_dev, double* v_dev, int64_t* step_count_host);

/* ------------------------------------------------------------------------
 * Dual-mesh mapper (Sec. 3.2, Eqs. bary_proj, decomp, gram, bary_interp).
 * Context-free: errors are reported through ipc_last_error(NULL).
 * ------------------------------------------------------------------------ */

/* Embed the visual vertices P_dev (device FP64 [np][3]) on the simulation
 * surface (V_dev device FP64 [nv][3], triangles T_dev device int32 [nt][3]):
 * for each vertex the nearest triangle (smallest point-triangle distance; on
 * a tie the lowest index) into tri_dev (device int32 [np]), and into
 * uvwd_dev (device FP64 [np][4], 16-byte aligned) the barycentric
 * coordinates (u, v, w) of its projection onto that triangle's plane (the
 * 2x2 Gram system of Eq. gram; they may be negative when the projection
 * falls outside the triangle) and the signed offset delta = (p - v0) . n,
 * n = (v1 - v0) x (v2 - v0) normalised.  dist2_dev (device FP64 [np], may be
 * NULL) receives the squared distances.  Allocates and frees its scratch (a
 * uniform grid of the triangles' boxes) and synchronises stream (a
 * cudaStream_t).  IPC_ERR_ARG for NULL pointers, an empty mesh or a
 * non-finite vertex. */
ipc_status ipc_dual_map_build(const double* V_dev, int64_t nv, const int32_t* T_dev, int64_t nt,
                              const double* P_dev, int64_t np, int32_t* tri_dev, double* uvwd_dev,
                              double* dist2_dev, void* stream);

/* Per-frame update, Eq. (bary_interp): out_dev[i] (device FP64 [np][3]) =
 * u v0' + v v1' + w v2' + delta n' for the deformed simulation vertices
 * V_dev (same vertex count and triangles T_dev [nt][3] as the build) and the
 * triangles and coordinates of ipc_dual_map_build.  A triangle index
 * outside [0, nt) gives NaN.  Queued on stream, no synchronisation. */
ipc_status ipc_dual_map_apply(const double* V_dev, const int32_t* T_dev, int64_t nt, const int32_t* tri_dev,
                              const double* uvwd_dev, int64_t np, double* out_dev, void* stream);

/* Paper-exact face samples (Sec. 4.1 "Face samples"), for a list of pairs
 * pairs_dev (device int32 [n][2]: slave triangle, master triangle) of the
 * slave mesh (xs_dev FP64 [nvs][3], ts_dev int32 [nts][3]) and the master
 * mesh (xm_dev FP64 [nvm][3], tm_dev int32 [ntm][3]), all device memory.
 * Both triangles are projected onto the slave triangle's tangent plane, the
 * projected master triangle is clipped by the slave triangle
 * (Sutherland-Hodgman), the polygon is fan-triangulated from its first
 * vertex and each sub-triangle gets the 3-point degree-2 Gauss rule (points
 * (2/3, 1/6, 1/6) and permutations, weight area/3).  Each sample is cast
 * along the slave normal n_s = (xs1 - xs0) x (xs2 - xs0) normalised onto the
 * master plane.  samples_dev (device FP64 [n][12][8]) receives per sample
 * beta^s[3], beta^m[3], the gap g and the weight w; count_dev (device int32
 * [n]) the number of samples (0 to 12; 0 when the overlap has no area or
 * the master plane contains n_s; -1 for a pair with a triangle or vertex
 * index out of range, which gets no samples).  The contact pass does not use
 * it (it keeps the fixed slave-side rule).  Context-free (errors through
 * ipc_last_error(NULL)); asynchronous on stream, allocates nothing.
 * IPC_ERR_ARG for a NULL pointer or n < 0. */
ipc_status ipc_face_clip_samples(const double* xs_dev, int64_t nvs, const int32_t* ts_dev, int64_t nts,
                                 const double* xm_dev, int64_t nvm, const int32_t* tm_dev, int64_t ntm,
                                 const int32_t* pairs_dev, int64_t n, double* samples_dev, int32_t* count_dev,
                                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GMCP_H */

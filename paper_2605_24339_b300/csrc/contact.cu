// contact.cu -- GMCP samples, barrier, gradient / Hessian coefficients,
// deterministic gathers, and the linearised-gap step bound.
//
// Work decomposition (one warp per active slave triangle, persistent grid;
// the triangles' frames come from a thread-per-triangle pass):
//   face items  = (sample k, candidate master tri)  -> lane handles items
//                 lane, lane+32, ...; since 32 is a multiple of the 4 or 16
//                 samples per triangle, each lane keeps one fixed sample k
//   edge items  = (candidate master edge, Gauss point)
//   point items = candidate master vertex
// Each lane accumulates the triangle's energy (FP64) and the coefficients
//   G_a  = sum_k c1_k beta^s_a,k            (c1 = kappa_q w gamma B')
//   S_ab = sum_k c2_k beta^s_a beta^s_b      (c2 = max(kappa_q w gamma B'', 0))
// and a fixed xor-shuffle tree reduces them, so the result does not depend
// on scheduling.  Per vertex the gradient is -sum_tris G_a n_s and per block
// the Hessian sum_tris S_ab n_s n_s^T (Sec. 4.2 with dg/dx_a = -beta_a n_s),
// gathered in a fixed order by k_gather_* (no float atomics).
//
// Rounding.  This file is compiled without fused multiply-add and its FP64
// geometry follows the operation order of a plain evaluation of the same
// formulas, so the sample membership decisions (which are not continuous in
// the weight for point samples and for edges lying on slave edges) come out
// identical to a plain IEEE evaluation even on coincident meshes.
//
// Precision.  FP64 path: everything in double.  Mixed path: every sample is
// first pre-tested in FP32 in a local frame anchored at the slave
// triangle's first vertex (coordinate differences formed in FP64, then
// rounded), with slacks that bound the FP32 error, so only samples that
// cannot be active are dropped; the survivors are built and decided in FP64
// exactly as in the FP64 path.  Barrier, gradient and Hessian coefficients
// are FP32; the energy sum stays FP64.
#include <cfloat>

#include "faceclip.cuh"
#include "gmcp_internal.cuh"

namespace gmcp {
namespace {

constexpr int MODE_EVAL = 0;
constexpr int MODE_ALPHA = 1;
constexpr int MODE_LAGGED = 2;
constexpr int MODE_MASTER_HESS = 4;   // the master vertices' entries: gradient rows and Hessian blocks

// outputs of the modes beyond the evaluation.  MODE_LAGGED: the frozen-
// linear energy changes, per active sample kappa w gamma [B(g + a_j dg) -
// B(g)] for up to 8 step sizes a_j along the direction dx.  MODE_MASTER_HESS:
// the master vertices' entries (gradient rows and Hessian blocks), appended
// to a list that the caller sorts and sums in a fixed order.
struct ModeArgs {
    const double* alphas = nullptr;
    int na = 0;
    double* triE8 = nullptr;   // [8][ns]
    int64_t ns = 0;
    // MODE_MASTER_HESS: blocks (row, col) with value coef n n^T, appended at
    // *h_count (entries past h_cap are counted, not written)
    int32_t* h_ij = nullptr;   // [h_cap][2]
    double* h_blk = nullptr;   // [h_cap][9]
    unsigned long long* h_count = nullptr;
    int64_t h_cap = 0;
    int32_t m_off = 0;         // index of master vertex 0 in the joint numbering
    // with h_rows: the gradient rows of the master vertices are appended to
    // the same list as entries (row, -1) whose first three values are the row
    bool h_rows = false;
    bool h_blocks = true;      // with false: the rows alone
    // MODE_ALPHA: the bound of a sample on slave triangle t goes to
    // alpha_bits[alpha_stride * env(t)] (0: one bound for the whole scene)
    int alpha_stride = 0;
    // MODE_LAGGED: the step sizes of slave triangle t are at
    // alphas[alphas_stride * env(t)] (0: the same for the whole scene)
    int alphas_stride = 0;
};


template <class R>
struct V3 { R x, y, z; };

template <class R> __device__ __forceinline__ V3<R> operator-(V3<R> a, V3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class R> __device__ __forceinline__ V3<R> operator+(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class R> __device__ __forceinline__ V3<R> operator*(R s, V3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class R> __device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class R> __device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3<double> ld3(const double* p, int64_t i) {
    return {p[3 * i], p[3 * i + 1], p[3 * i + 2]};
}
__device__ __forceinline__ V3<float> tof(V3<double> a) { return {(float)a.x, (float)a.y, (float)a.z}; }

template <class R> __device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }
template <class R> __device__ __forceinline__ R rmax(R a, R b) { return a > b ? a : b; }
template <class R> __device__ __forceinline__ R min3(const R* b) { return rmin(b[0], rmin(b[1], b[2])); }

// Eq. (gram): barycentric coordinates of the projection of q on (p0,p1,p2)
template <class R>
__device__ __forceinline__ void bary(V3<R> q, V3<R> p0, V3<R> p1, V3<R> p2, R* b) {
    V3<R> e1 = p1 - p0, e2 = p2 - p0, d = q - p0;
    R a = dot(e1, e1), bb = dot(e1, e2), c = dot(e2, e2);
    R r1 = dot(d, e1), r2 = dot(d, e2);
    R det = a * c - bb * bb;
    R v = (c * r1 - bb * r2) / det;
    R w = (a * r2 - bb * r1) / det;
    b[0] = R(1) - v - w; b[1] = v; b[2] = w;
}

template <class R>
__device__ __forceinline__ V3<R> interp(const R* b, V3<R> x0, V3<R> x1, V3<R> x2) {
    return {b[0] * x0.x + b[1] * x1.x + b[2] * x2.x, b[0] * x0.y + b[1] * x1.y + b[2] * x2.y,
            b[0] * x0.z + b[1] * x1.z + b[2] * x2.z};
}

// Eq. (smoothstep)
template <class R>
__device__ __forceinline__ R hermite(R x, R delta) {
    if (x <= R(0)) return R(0);
    if (x >= delta) return R(1);
    R t = x / delta;
    return R(3) * t * t - R(2) * t * t * t;
}

// IPC barrier and derivatives on (0, eps); the caller guarantees 0 < g < eps
__device__ __forceinline__ void barrier(double g, double eps, double& B, double& dB, double& d2B) {
    double d = g - eps, L = log(g / eps);
    B = -d * d * L;
    dB = -2.0 * d * L - d * d / g;
    d2B = -2.0 * L - 4.0 * d / g + d * d / (g * g);
}
// FP32 values from the FP64 gap: d = g - eps and d / eps are formed in FP64
// and rounded once, and L = ln(g/eps) = log1p(d/eps).  Rounding g and eps to
// FP32 before subtracting would leave d (and so B, B', B'') only
// ~6e-8 eps / |d| relatively accurate near g = eps.  On (0, eps) the terms of
// B' (-2dL, -d^2/g: both < 0) and of B'' (-2L, -4d/g, d^2/g^2: all > 0) never
// cancel, so each value keeps FP32's relative precision.
__device__ __forceinline__ void barrier(double g64, double eps64, float& B, float& dB, float& d2B) {
    const double d64 = g64 - eps64;
    const float d = (float)d64, g = (float)g64;
    const float L = log1pf((float)(d64 / eps64));
    const float r = d / g;
    B = -d * d * L;
    dB = -2.0f * d * L - d * r;
    d2B = -2.0f * L - 4.0f * r + r * r;
}


// face-rule barycentrics per level (index L-1), filled at context creation;
// c_rule_f the same rounded to FP32 (the certified FP32 items)
__constant__ double c_rule[2][16][3];
__constant__ float c_rule_f[2][16][3];

// Face ray cast of Sec. 4.1 (fixed slave-side rule): from xs along ns onto
// the plane of (y0,y1,y2).  Returns true when the master tri faces the slave,
// the hit is inside it and g > 0; then x_m - x_s = g n_s (Eq. gap).
template <class R>
__device__ __forceinline__ bool face_geom(V3<R> xs, V3<R> ns, V3<R> y0, V3<R> y1, V3<R> y2, R& g,
                                          R* bm) {
    V3<R> e1 = y1 - y0, e2 = y2 - y0, N = cross(e1, e2);
    R den = dot(N, ns);
    if (!(den < R(0))) return false;
    g = dot(N, y0 - xs) / den;
    V3<R> p = xs + g * ns;
    bary(p, y0, y1, y2, bm);
    return min3(bm) >= R(0) && g > R(0);
}

// FP32 pre-test of a face sample in the slave triangle's local frame: false
// only when the exact FP64 test (face_geom<double> with g < eps <= eps_max)
// certainly fails.  Near-grazing casts (|N.n_s| < 1e-3 |N|) always go to the
// FP64 test.  With |den| >= 1e-3 |N| the FP32 gap is within 1e-3 (|d| + |g|)
// of the FP64 one (inputs rounded once, a handful of operations of relative
// error 6e-8 each, divided by |den|/|N| >= 1e-3), and the barycentric error
// is that gap error over the triangle's smallest height plus 1e-2 slack.
__device__ __forceinline__ bool face_maybe(V3<float> xs, V3<float> ns, V3<float> y0, V3<float> y1,
                                           V3<float> y2, float eps_max) {
    const V3<float> e1 = y1 - y0, e2 = y2 - y0, N = cross(e1, e2);
    const float nN = sqrtf(dot(N, N));
    const float den = dot(N, ns);
    if (den >= 1e-3f * nN) return false;          // faces away (facing needs den < 0)
    if (den > -1e-3f * nN) return true;           // grazing: let FP64 decide
    const V3<float> d = y0 - xs;
    const float g = dot(N, d) / den;
    const float tol_g = 1e-3f * (sqrtf(dot(d, d)) + fabsf(g));
    if (g > eps_max + tol_g || g < -tol_g) return false;
    const V3<float> p = xs + g * ns;
    float b[3];
    bary(p, y0, y1, y2, b);
    const float lmax = sqrtf(rmax(dot(e1, e1), rmax(dot(e2, e2), dot(e2 - e1, e2 - e1))));
    const float tol_b = 1e-2f + 4.0f * tol_g * lmax / nN;
    return min3(b) >= -tol_b;
}

// FP32 pre-test of edge and point samples.  Their gap is g = n_s . (x_m -
// x_s) with x_s on the slave plane, i.e. the plane distance n_s . (y - x0)
// of a point y on the master edge [a, b] (a = b for a vertex), an affine
// mix of the end values.  False only when that distance is certainly >=
// eps_max (no sample can be active) or certainly <= 0 at both ends; the FP32
// error of each end value is below 1e-6 |y - x0|_1, the slack is ten times
// that plus tol_abs for the rounding of the FP64 gap itself (and eps_max is
// raised by 1e-6 relative for its own rounding to FP32).
__device__ __forceinline__ bool plane_gap_maybe(V3<float> ns, V3<float> a, V3<float> b, float eps_max,
                                                float tol_abs) {
    const float da = dot(ns, a), db = dot(ns, b);
    const float tol = 1e-5f * (fabsf(a.x) + fabsf(a.y) + fabsf(a.z) + fabsf(b.x) + fabsf(b.y) + fabsf(b.z)) +
                      tol_abs;
    return !(rmin(da, db) > eps_max * (1.0f + 1e-6f) + tol || rmax(da, db) < -tol);
}

// FP32 barycentric coordinates of p (relative to x0) in the slave frame
// (e1, e2 = x1 - x0, x2 - x0), with a bound on their error: Gram formula
// (as bary), each rounding 2^-24 relative; tol below exceeds 100 times the
// first-order error bound, plus 1e-3.  ok is false for a degenerate frame.
__device__ __forceinline__ void bary_f(V3<float> p, V3<float> e1, V3<float> e2, float* b, float& tol,
                                       bool& ok) {
    const float a = dot(e1, e1), bb = dot(e1, e2), c = dot(e2, e2);
    const float r1 = dot(p, e1), r2 = dot(p, e2);
    const float det = a * c - bb * bb;
    ok = det > 1e-6f * a * c;
    const float v = (c * r1 - bb * r2) / det;
    const float w = (a * r2 - bb * r1) / det;
    b[0] = 1.0f - v - w; b[1] = v; b[2] = w;
    const float mag = c * fabsf(r1) + fabsf(bb * r2) + a * fabsf(r2) + fabsf(bb * r1) +
                      (a * c + bb * bb) * (fabsf(v) + fabsf(w));
    tol = 1e-3f + 1e-5f * mag / det;
}

// squared distance between two boxes (0 when they overlap)
__device__ __forceinline__ double box_dist2(const double* alo, const double* ahi, const double* blo,
                                            const double* bhi) {
    double s = 0.0;
    for (int c = 0; c < 3; ++c) {
        double d = rmax(0.0, rmax(alo[c] - bhi[c], blo[c] - ahi[c]));
        s += d * d;
    }
    return s;
}

// Eq. (adaptive_eps): eps is eps_max whenever the rest boxes are so far apart
// that 0.9 g_ref > eps_max for any sample of the pair (g_ref >= box distance)
__device__ __forceinline__ bool rest_far(const double* slo, const double* shi, const double* mlo,
                                         const double* mhi, double eps_max) {
    const double r = eps_max * (1.2 / 0.9);
    return box_dist2(slo, shi, mlo, mhi) >= r * r;
}
// certain FP32 version: boxes rounded outward and every operation rounded
// down give a lower bound of the squared distance; r2f is the threshold
// rounded up with a 1e-6 margin (Params::far_r2_f), so true implies that
// rest_far holds in FP64 (false decides nothing)
__device__ __forceinline__ bool rest_far_f(const float* slo, const float* shi, const float* mlo, const float* mhi,
                                           float r2f) {
    float s = 0.0f;
    for (int q = 0; q < 3; ++q) {
        const float d = fmaxf(0.0f, fmaxf(__fsub_rd(mlo[q], shi[q]), __fsub_rd(slo[q], mhi[q])));
        s = __fadd_rd(s, __fmul_rd(d, d));
    }
    return s >= r2f;
}

__device__ __forceinline__ bool any_facing(const SceneView& S, const double* xm, const int32_t* tris,
                                           int n, V3<double> ns) {
    for (int i = 0; i < n; ++i) {
        const int32_t* M = S.mtri + 3 * (int64_t)tris[i];
        V3<double> y0 = ld3(xm, M[0]);
        V3<double> N = cross(ld3(xm, M[1]) - y0, ld3(xm, M[2]) - y0);
        if (dot(N, ns) < 0.0) return true;
    }
    return false;
}

template <class T>
struct Acc {
    double E;
    T G[3];
    T S[6];
    double amin;
    __device__ void zero() {
        E = 0.0; amin = INFINITY;
        for (int i = 0; i < 3; ++i) G[i] = T(0);
        for (int i = 0; i < 6; ++i) S[i] = T(0);
    }
    __device__ void add(double e, T c1, T c2, const T* b) {
        E += e;
        G[0] += c1 * b[0]; G[1] += c1 * b[1]; G[2] += c1 * b[2];
        S[0] += c2 * b[0] * b[0]; S[1] += c2 * b[0] * b[1]; S[2] += c2 * b[0] * b[2];
        S[3] += c2 * b[1] * b[1]; S[4] += c2 * b[1] * b[2]; S[5] += c2 * b[2] * b[2];
    }
};

// one sample of Eq. (gmcp_potential) and its Sec. 4.2 derivatives
template <class T>
__device__ __forceinline__ void sample_add(Acc<T>& A, double kq, double w, double gamma, double g,
                                           double eps, const double* bs) {
    T Bv, dB, d2B;
    barrier(g, eps, Bv, dB, d2B);
    T coef = (T)(kq * w * gamma);
    T b[3] = {(T)bs[0], (T)bs[1], (T)bs[2]};
    A.add((double)(coef * Bv), coef * dB, rmax(coef * d2B, T(0)), b);
}

template <class T> __device__ __forceinline__ T shfl_x(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

// slots for the lanes with pred set, one atomic for the warp (all 32 lanes call it)
__device__ __forceinline__ int warp_reserve_c(bool pred, int32_t* counter) {
    const unsigned mask = __ballot_sync(0xffffffffu, pred);
    if (mask == 0u) return 0;
    const int leader = __ffs(mask) - 1;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    return base + __popc(mask & lt);
}

// one sample of the frozen-linear potential (lagged energy of the line
// search, reading R6): g~ = g + a dg; +inf once g~ <= 0, 0 from eps on
// the change coef [B(g + a_j dg) - B(g)] of a frozen sample's barrier
// (the line search compares changes, not totals)
__device__ __forceinline__ void lag_add(double* E8, const double* al, int na, double coef, double g,
                                        double eps, double dg) {
    double e0 = 0.0;
    if (g < eps) {
        const double d = g - eps, L = log(g / eps);
        e0 = coef * (-d * d * L);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j >= na) break;
        const double gt = g + al[j] * dg;
        double e = 0.0;
        if (!(gt > 0.0)) {
            e = INFINITY;
        } else if (gt < eps) {
            const double d = gt - eps, L = log(gt / eps);
            e = coef * (-d * d * L);
        }
        E8[j] += e - e0;
    }
}

// ---------------------------------------------------------------------------
// the samples
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Outputs touched by the active triangles only.  A contact evaluation
// numbers itself (slot kSlotPass) and stamps its active triangles; the
// frame pass also lists the vertices and contact blocks of those triangles
// once each (stamps make the lists duplicate-free).  Gradient rows and
// blocks are then gathered in a fixed order over their contributing
// triangles, skipping those not active in this evaluation (their stored
// outputs are stale), so the result does not depend on the lists' order.
// The gradient is written whole (zero rows first); the Hessian blocks live
// in the context, so only the blocks listed by the previous Hessian pass and
// not by this one are cleared.  The block lists of consecutive Hessian
// passes alternate by the parity of the Hessian-pass number (kSlotHPass).
// ---------------------------------------------------------------------------
__global__ void k_pass_begin(int32_t* misc, int hess) {
    pass_dep_wait();
    const int32_t p = ++misc[kSlotPass];
    (void)p;
    misc[kSlotVCount] = 0;
    misc[kSlotItemList] = 0;
    misc[kSlotItemList2] = 0;
    misc[kSlotItemMid] = 0;
    misc[kSlotItemMid2] = 0;
    if (hess) {
        const int32_t h = ++misc[kSlotHPass];
        misc[kSlotBCount + (h & 1)] = 0;
    }
}

struct TouchArgs {
    const int32_t* misc;
    int32_t* v_stamp;
    int32_t* v_list;
    int32_t* v_count;
    int32_t* b_stamp;
    int32_t* b_list[2];
    int32_t* b_count;      // [2], by Hessian-pass parity
    const int32_t* row;    // contact BSR pattern
    const int32_t* col;
    int grad, hess;
};

// List the vertices and contact blocks of the active slave triangles once
// each (stamps), one thread per (triangle, corner a): vertex T[a] and the
// blocks (T[a], T[b]) of its row.  Runs beside the sample evaluation.
__global__ void k_touch(SceneView S, CandView C, TouchArgs A) {
    pass_dep_wait();
    const int n = 3 * *C.n_active;
    const int32_t ps = A.misc[kSlotPass], hs = A.misc[kSlotHPass];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int32_t* T = S.stri + 3 * (int64_t)C.active[idx / 3];
        const int a = idx % 3;
        const int32_t v = T[a];
        if (A.grad && atomicExch(&A.v_stamp[v], ps) != ps) A.v_list[atomicAdd(A.v_count, 1)] = v;
        if (!A.hess) continue;
        for (int b = 0; b < 3; ++b) {
            int32_t k = A.row[v];
            while (A.col[k] != T[b]) ++k;        // the pattern holds every (T[a], T[b])
            if (atomicExch(&A.b_stamp[k], hs) != hs) A.b_list[hs & 1][atomicAdd(&A.b_count[hs & 1], 1)] = k;
        }
    }
}

// Frames of the active slave triangles, one thread per triangle, so that
// the FP64 square roots and divisions run once per triangle: unit normal
// and area at x, unit normal at rest, and the absolute slack of the FP32
// plane-distance pre-tests (which covers the FP64 rounding of gaps formed
// from coordinates of this magnitude).  frame[8 i ...] belongs to active[i].
// With items != NULL it also counts the triangle's sample items (face:
// candidate x sample, edge: candidate x Gauss point, point: candidate),
// reserves a contiguous range of slots for them (items[2 i] = first slot,
// items[2 i + 1] = count; the ranges' order depends on scheduling, the
// per-triangle results do not) and adds them to *n_items.
// With tf32 != NULL (mixed path) it also writes tf32[64 i ...]: the nk face
// samples relative to the environment's grid origin in FP32 (3 nk floats,
// interpolated in FP32 from the vertices below, so within 2^-22 max|v| of
// the exact samples), the unit normal in FP32 at [48, 51) and the three
// vertices minus the origin, rounded to FP32, at [51, 60): the inputs of the
// FP32 pre-filter of the sample items.
// With tmid64 != NULL (mixed path) it also writes the middle stage's
// per-triangle inputs: tmid32[16 i ...] the unit normal, x1 - x0 and x2 - x0
// rounded to FP32 (the values the item kernels would form), a face
// sample's weight A / nk, n_s . dx_a for the three vertices (dx NULL: 0)
// and the sum of their magnitudes rounded up; tmid64[4 i ...] the same
// products and sum in FP64: once per triangle instead of once per item.
__global__ void k_tri_frame(SceneView S, CandView C, const double* __restrict__ x,
                            double* __restrict__ frame, int nk, int32_t* __restrict__ items,
                            int32_t* __restrict__ n_items, int32_t* __restrict__ tri_stamp,
                            const int32_t* __restrict__ misc, float* __restrict__ tf32, int L,
                            const double* __restrict__ dx, double* __restrict__ tmid64,
                            float* __restrict__ tmid32) {
    pass_dep_wait();
    const int n_active = *C.n_active;
    const int32_t ps = tri_stamp ? misc[kSlotPass] : 0;
    const int lane = threadIdx.x & 31;
    // whole warps iterate together (the item slots are reserved per warp),
    // interleaved across blocks: the frame is FP64 work, and a warp-wide FP64
    // instruction holds a sub-partition's narrow FP64 pipe for ~80 cycles, so
    // a few thousand active tris must spread over the SMs rather than fill
    // the first blocks
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t wslot = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5);
    for (int64_t ib = 32 * wslot; ib < n_active; ib += stride) {
        const int i = (int)(ib + lane);
        const bool valid = i < n_active;
        int n = 0;
        if (valid) {
            const int64_t t = C.active[i];
            const int32_t* Tt = S.stri + 3 * t;
            if (tri_stamp) tri_stamp[t] = ps;
            const V3<double> x0 = ld3(x, Tt[0]), x1 = ld3(x, Tt[1]), x2 = ld3(x, Tt[2]);
            const V3<double> X0 = ld3(S.X, Tt[0]), X1 = ld3(S.X, Tt[1]), X2 = ld3(S.X, Tt[2]);
            const V3<double> cr = cross(x1 - x0, x2 - x0);
            const double clen = sqrt(dot(cr, cr));
            const V3<double> cr0 = cross(X1 - X0, X2 - X0);
            const double clen0 = sqrt(dot(cr0, cr0));
            double* f = frame + 8 * (int64_t)i;
            const double ic = 1.0 / clen, ic0 = 1.0 / clen0;   // one FP64 division per normal
            f[0] = cr.x * ic; f[1] = cr.y * ic; f[2] = cr.z * ic;
            f[3] = 0.5 * clen;
            f[4] = cr0.x * ic0; f[5] = cr0.y * ic0; f[6] = cr0.z * ic0;
            f[7] = 1e-12 * (fabs(x0.x) + fabs(x0.y) + fabs(x0.z)) + 1e-30;
            if (tf32) {
                const int e = S.stri_env[t];
                const V3<double> org = {S.grid_org[3 * e], S.grid_org[3 * e + 1], S.grid_org[3 * e + 2]};
                float* o = tf32 + 64 * (int64_t)i;
                const V3<float> v0 = tof(x0 - org), v1 = tof(x1 - org), v2 = tof(x2 - org);
                for (int k = 0; k < nk; ++k) {
                    // FP32 from the rounded vertices (within 2^-22 max|v| of the exact sample)
                    const float b0 = (float)c_rule[L - 1][k][0], b1 = (float)c_rule[L - 1][k][1],
                                b2 = (float)c_rule[L - 1][k][2];
                    o[3 * k] = b0 * v0.x + b1 * v1.x + b2 * v2.x;
                    o[3 * k + 1] = b0 * v0.y + b1 * v1.y + b2 * v2.y;
                    o[3 * k + 2] = b0 * v0.z + b1 * v1.z + b2 * v2.z;
                }
                o[48] = (float)f[0]; o[49] = (float)f[1]; o[50] = (float)f[2];
                o[51] = v0.x; o[52] = v0.y; o[53] = v0.z;
                o[54] = v1.x; o[55] = v1.y; o[56] = v1.z;
                o[57] = v2.x; o[58] = v2.y; o[59] = v2.z;
            }
            if (tmid64) {
                const V3<double> ns = {f[0], f[1], f[2]};
                float* m32 = tmid32 + 16 * (int64_t)i;
                const V3<float> nf = tof(ns), e1 = tof(x1 - x0), e2 = tof(x2 - x0);
                m32[0] = nf.x; m32[1] = nf.y; m32[2] = nf.z;
                m32[3] = e1.x; m32[4] = e1.y; m32[5] = e1.z;
                m32[6] = e2.x; m32[7] = e2.y; m32[8] = e2.z;
                V3<double> d0 = {0, 0, 0}, d1 = {0, 0, 0}, d2 = {0, 0, 0};
                if (dx) { d0 = ld3(dx, Tt[0]); d1 = ld3(dx, Tt[1]); d2 = ld3(dx, Tt[2]); }
                double* m64 = tmid64 + 4 * (int64_t)i;
                const double s0 = dot(ns, d0), s1 = dot(ns, d1), s2 = dot(ns, d2);
                m64[0] = s0; m64[1] = s1; m64[2] = s2;
                m64[3] = fabs(s0) + fabs(s1) + fabs(s2);
                m32[9] = (float)(f[3] * (1.0 / (double)nk));   // nk a power of two: exact
                m32[10] = (float)s0; m32[11] = (float)s1; m32[12] = (float)s2;
                m32[13] = (float)m64[3] * 1.000001f;   // at least the sum
                m32[14] = 0.0f; m32[15] = 0.0f;
            }
            if (items) {
                const int32_t* cnt = C.count + 4 * t;
                n = min(cnt[0], C.cap_f) * nk + 2 * min(cnt[1], C.cap_e) + min(cnt[2], C.cap_p);
            }
        }
        if (items) {
            // the warp's ranges are consecutive: one atomic per warp
            int incl = n;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            int base = 0;
            if (lane == 31) base = atomicAdd(n_items, incl);
            base = __shfl_sync(0xffffffffu, base, 31);
            if (valid) {
                items[2 * i] = base + incl - n;
                items[2 * i + 1] = n;
            }
        }
    }
}

// what the slave triangle's samples share
struct TriData {
    int64_t t;
    V3<double> x0, x1, x2, X0, X1, X2, dx0, dx1, dx2, ns, ns0;
    V3<float> ns_f;
    V3<float> e1_f, e2_f;  // x1 - x0, x2 - x0 (FP64 differences, rounded)
    float w_f;             // a face sample's weight A / nk (middle stage)
    float sdxf[4];         // sdx in FP32, the sum rounded up (middle stage)
    double As;
    float tol_abs;
    const double* sb;      // rest box of the slave tri
    const float* sbf;      // the same in FP32, rounded outward
    double sdx[4];         // n_s . dx_a of the three vertices and the sum of their magnitudes (middle stage)
    int nf, ne, np;        // candidates (capped)
};

__device__ __forceinline__ TriData load_tri(const SceneView& S, const CandView& C, const double* x,
                                            const double* dx, const double* frame, int i) {
    TriData D;
    D.t = C.active[i];
    const int32_t* Tt = S.stri + 3 * D.t;
    D.x0 = ld3(x, Tt[0]); D.x1 = ld3(x, Tt[1]); D.x2 = ld3(x, Tt[2]);
    D.X0 = ld3(S.X, Tt[0]); D.X1 = ld3(S.X, Tt[1]); D.X2 = ld3(S.X, Tt[2]);
    const double* fr = frame + 8 * (int64_t)i;
    D.ns = {fr[0], fr[1], fr[2]};
    D.As = fr[3];
    D.ns0 = {fr[4], fr[5], fr[6]};
    D.tol_abs = (float)fr[7];
    D.ns_f = tof(D.ns);
    D.e1_f = tof(D.x1 - D.x0);
    D.e2_f = tof(D.x2 - D.x0);
    D.sb = S.srest_box + 6 * D.t;
    D.sbf = S.srest_box_f + 6 * D.t;
    const int32_t* cnt = C.count + 4 * D.t;
    D.nf = min(cnt[0], C.cap_f); D.ne = min(cnt[1], C.cap_e); D.np = min(cnt[2], C.cap_p);
    D.dx0 = {0, 0, 0}; D.dx1 = {0, 0, 0}; D.dx2 = {0, 0, 0};
    if (dx) { D.dx0 = ld3(dx, Tt[0]); D.dx1 = ld3(dx, Tt[1]); D.dx2 = ld3(dx, Tt[2]); }
    return D;
}
// the middle stage's view of a triangle: what it needs per item, read from
// the per-triangle values k_tri_frame stored (tri_mid32: FP32 normal and
// edges; tri_mid64: the normal's products with the vertex displacements)
// instead of being formed again from FP64 coordinates for every item
__device__ __forceinline__ TriData load_tri_mid(const SceneView& S, const CandView& C, const double* x,
                                                const double* frame, const double* tmid64,
                                                const float* tmid32, int i) {
    TriData D;
    D.t = C.active[i];
    const int32_t* Tt = S.stri + 3 * D.t;
    D.x0 = ld3(x, Tt[0]); D.x1 = ld3(x, Tt[1]); D.x2 = ld3(x, Tt[2]);
    const double* fr = frame + 8 * (int64_t)i;
    D.As = fr[3];
    D.tol_abs = (float)fr[7];
    const float* m = tmid32 + 16 * (int64_t)i;
    D.ns_f = {m[0], m[1], m[2]};
    D.e1_f = {m[3], m[4], m[5]};
    D.e2_f = {m[6], m[7], m[8]};
    D.w_f = m[9];
    for (int q = 0; q < 4; ++q) D.sdxf[q] = m[10 + q];
    const double* m64 = tmid64 + 4 * (int64_t)i;
    for (int q = 0; q < 4; ++q) D.sdx[q] = m64[q];
    D.sb = S.srest_box + 6 * D.t;
    D.sbf = S.srest_box_f + 6 * D.t;
    const int32_t* cnt = C.count + 4 * D.t;
    D.nf = min(cnt[0], C.cap_f); D.ne = min(cnt[1], C.cap_e); D.np = min(cnt[2], C.cap_p);
    return D;
}

// an active sample: kappa_q, weight w, gamma, gap g, eps, slave
// barycentrics b and the linearised gap change dg along (dx, dxm)
struct ItemOut {
    double kq, w, gamma, g, eps, dg;
    double g_step;   // the gap the step bound uses: g, or a certified lower bound of it
    double b[3];
    int32_t mv[3];   // master vertices of x_m (-1 unused) and their weights
    double bm[3];
};

// what a face sample k shares over its candidates: its position, the
// position relative to x0 in FP32 and the slave-side gap change
struct FaceSample {
    double beta[3];
    V3<double> xs;
    V3<float> xs_rel;
    double ds;
};
__device__ __forceinline__ FaceSample face_sample(const Params& P, const TriData& D, int k, bool want_dg) {
    FaceSample F;
    for (int q = 0; q < 3; ++q) F.beta[q] = c_rule[P.L - 1][k][q];
    F.xs = interp(F.beta, D.x0, D.x1, D.x2);
    F.xs_rel = tof(F.xs - D.x0);
    F.ds = want_dg ? dot(D.ns, interp(F.beta, D.dx0, D.dx1, D.dx2)) : 0.0;
    return F;
}

// FP32 pre-tests of the mixed path: false only when the exact FP64 test of
// the item certainly fails (the bounds are stated at face_maybe,
// plane_gap_maybe and bary_f)
__device__ __forceinline__ bool face_pre(const Params& P, const TriData& D, const FaceSample& F,
                                         V3<double> y0, V3<double> y1, V3<double> y2) {
    return face_maybe(F.xs_rel, D.ns_f, tof(y0 - D.x0), tof(y1 - D.x0), tof(y2 - D.x0), (float)P.dhat);
}
__device__ __forceinline__ bool edge_pre(const Params& P, const TriData& D, V3<double> ya, V3<double> yb) {
    const V3<float> da = tof(ya - D.x0), db = tof(yb - D.x0);
    if (!plane_gap_maybe(D.ns_f, da, db, (float)P.dhat, D.tol_abs)) return false;
    // the projected edge misses the slave tri when both ends are certainly
    // on the outer side of one of its edges (beta_a is affine along it)
    float fa[3], fb[3], ta, tb;
    bool oka, okb;
    bary_f(da, D.e1_f, D.e2_f, fa, ta, oka);
    bary_f(db, D.e1_f, D.e2_f, fb, tb, okb);
    if (oka && okb)
        for (int a = 0; a < 3; ++a)
            if (fa[a] < -ta && fb[a] < -tb) return false;
    return true;
}
__device__ __forceinline__ bool point_pre(const Params& P, const TriData& D, V3<double> y) {
    const V3<float> d = tof(y - D.x0);
    if (!plane_gap_maybe(D.ns_f, d, d, (float)P.dhat, D.tol_abs)) return false;
    float f[3], tf;
    bool ok;
    bary_f(d, D.e1_f, D.e2_f, f, tf, ok);
    return !(ok && min3(f) < -tf);
}

// face sample F of slave tri D against master tri m (Sec. 4.1, reading R1)
template <int NK>
__device__ __forceinline__ bool face_item(const SceneView& S, const Params& P, const TriData& D,
                                          const FaceSample& F, const double* xm, const double* dxm,
                                          int32_t m, bool pre, bool want_dg, ItemOut& o) {
    const double eps_max = P.dhat;
    const int32_t* M = S.mtri + 3 * (int64_t)m;
    const V3<double> y0 = ld3(xm, M[0]), y1 = ld3(xm, M[1]), y2 = ld3(xm, M[2]);
    if (pre && !face_pre(P, D, F, y0, y1, y2)) return false;
    double g, bm[3];
    if (!face_geom<double>(F.xs, D.ns, y0, y1, y2, g, bm)) return false;
    double eps = eps_max;
    const double* mb = S.mrest_box + 6 * (int64_t)m;
    if (!rest_far(D.sb, D.sb + 3, mb, mb + 3, eps_max)) {
        const V3<double> xs0 = interp(F.beta, D.X0, D.X1, D.X2);
        double g0, bm0[3];
        const bool ok0 = face_geom<double>(xs0, D.ns0, ld3(S.Y0, M[0]), ld3(S.Y0, M[1]), ld3(S.Y0, M[2]), g0, bm0);
        if (ok0) eps = rmin(0.9 * g0, eps_max);
    }
    if (!(g < eps)) return false;
    o.kq = P.kappa; o.w = (1.0 / (double)NK) * D.As; o.gamma = hermite(min3(bm), P.delta_T);
    o.g = g; o.g_step = g; o.eps = eps;
    for (int q = 0; q < 3; ++q) { o.b[q] = F.beta[q]; o.mv[q] = M[q]; o.bm[q] = bm[q]; }
    o.dg = 0.0;
    if (want_dg) {
        const double dm = dxm ? dot(D.ns, interp(bm, ld3(dxm, M[0]), ld3(dxm, M[1]), ld3(dxm, M[2]))) : 0.0;
        o.dg = dm - F.ds;
    }
    return true;
}

// Gauss point q of master edge me projected on slave tri D (Sec. 4.1,
// reading R3)
__device__ __forceinline__ bool edge_item(const SceneView& S, const Params& P, const TriData& D,
                                          const double* xm, const double* dxm, int32_t me, int q,
                                          bool pre, bool want_dg, ItemOut& o) {
    const double eps_max = P.dhat;
    const double gp = 1.0 / sqrt(3.0);
    const int ia = S.medge[2 * (int64_t)me], ib = S.medge[2 * (int64_t)me + 1];
    const V3<double> ya = ld3(xm, ia), yb = ld3(xm, ib);
    if (pre && !edge_pre(P, D, ya, yb)) return false;
    const int a0 = S.me_tri_off[me], a1 = S.me_tri_off[me + 1];
    if (!any_facing(S, xm, S.me_tri + a0, a1 - a0, D.ns)) return false;
    double bA[3], bB[3];
    bary(ya, D.x0, D.x1, D.x2, bA);
    bary(yb, D.x0, D.x1, D.x2, bB);
    // clip the projected edge by the slave triangle: all beta >= 0
    double lo = 0.0, hi = 1.0;
    bool empty = false;
    for (int a = 0; a < 3; ++a) {
        const double Dd = bB[a] - bA[a];
        if (Dd > 0.0) lo = rmax(lo, -bA[a] / Dd);
        else if (Dd < 0.0) hi = rmin(hi, -bA[a] / Dd);
        else if (bA[a] < 0.0) empty = true;
    }
    if (empty || !(hi > lo)) return false;
    const V3<double> tv = yb - ya;
    const double tn = dot(tv, D.ns);
    const V3<double> tp = tv - tn * D.ns;
    const double ell = (hi - lo) * sqrt(dot(tp, tp));
    const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    const double eta = q == 0 ? mid - half * gp : mid + half * gp;
    const V3<double> xmk = (1.0 - eta) * ya + eta * yb;
    double bsk[3];
    bary(xmk, D.x0, D.x1, D.x2, bsk);
    const V3<double> xs = interp(bsk, D.x0, D.x1, D.x2);
    const double g = dot(D.ns, xmk - xs);
    if (!(g > 0.0)) return false;
    double eps = eps_max;
    const V3<double> Ya = ld3(S.Y0, ia), Yb = ld3(S.Y0, ib);
    const double elo[3] = {rmin(Ya.x, Yb.x), rmin(Ya.y, Yb.y), rmin(Ya.z, Yb.z)};
    const double ehi[3] = {rmax(Ya.x, Yb.x), rmax(Ya.y, Yb.y), rmax(Ya.z, Yb.z)};
    if (!rest_far(D.sb, D.sb + 3, elo, ehi, eps_max)) {
        const V3<double> xm0 = (1.0 - eta) * Ya + eta * Yb;
        double bs0[3];
        bary(xm0, D.X0, D.X1, D.X2, bs0);
        const double g0 = dot(D.ns0, xm0 - interp(bs0, D.X0, D.X1, D.X2));
        if (min3(bs0) >= 0.0 && g0 > 0.0) eps = rmin(0.9 * g0, eps_max);
    }
    if (!(g < eps)) return false;
    o.kq = P.kappa_edge; o.w = 0.5 * ell; o.gamma = hermite(eta, P.delta_e) * hermite(1.0 - eta, P.delta_e);
    o.g = g; o.g_step = g; o.eps = eps;
    for (int c = 0; c < 3; ++c) o.b[c] = bsk[c];
    o.mv[0] = ia; o.mv[1] = ib; o.mv[2] = -1;
    o.bm[0] = 1.0 - eta; o.bm[1] = eta; o.bm[2] = 0.0;
    o.dg = 0.0;
    if (want_dg) {
        const double ds = dot(D.ns, interp(bsk, D.dx0, D.dx1, D.dx2));
        const double dm = dxm ? dot(D.ns, (1.0 - eta) * ld3(dxm, ia) + eta * ld3(dxm, ib)) : 0.0;
        o.dg = dm - ds;
    }
    return true;
}

// master vertex u projected on slave tri D (Sec. 4.1, reading R3)
__device__ __forceinline__ bool point_item(const SceneView& S, const Params& P, const TriData& D,
                                           const double* xm, const double* dxm, int32_t u, bool pre,
                                           bool want_dg, ItemOut& o) {
    const double eps_max = P.dhat;
    const V3<double> y = ld3(xm, u);
    if (pre && !point_pre(P, D, y)) return false;
    const int a0 = S.mv_tri_off[u], a1 = S.mv_tri_off[u + 1];
    if (!any_facing(S, xm, S.mv_tri + a0, a1 - a0, D.ns)) return false;
    double bs[3];
    bary(y, D.x0, D.x1, D.x2, bs);
    if (!(min3(bs) >= 0.0)) return false;
    const double g = dot(D.ns, y - interp(bs, D.x0, D.x1, D.x2));
    if (!(g > 0.0)) return false;
    double eps = eps_max;
    const V3<double> Y = ld3(S.Y0, u);
    const double yb[3] = {Y.x, Y.y, Y.z};
    if (!rest_far(D.sb, D.sb + 3, yb, yb, eps_max)) {
        double bs0[3];
        bary(Y, D.X0, D.X1, D.X2, bs0);
        const double g0 = dot(D.ns0, Y - interp(bs0, D.X0, D.X1, D.X2));
        if (min3(bs0) >= 0.0 && g0 > 0.0) eps = rmin(0.9 * g0, eps_max);
    }
    if (!(g < eps)) return false;
    o.kq = P.kappa_point; o.w = 1.0; o.gamma = 1.0;
    o.g = g; o.g_step = g; o.eps = eps;
    for (int c = 0; c < 3; ++c) o.b[c] = bs[c];
    o.mv[0] = u; o.mv[1] = -1; o.mv[2] = -1;
    o.bm[0] = 1.0; o.bm[1] = 0.0; o.bm[2] = 0.0;
    o.dg = 0.0;
    if (want_dg) {
        const double ds = dot(D.ns, interp(bs, D.dx0, D.dx1, D.dx2));
        const double dm = dxm ? dot(D.ns, ld3(dxm, u)) : 0.0;
        o.dg = dm - ds;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Certified FP32 evaluation (mixed path, contact evaluation only).
//
// The FP32 pre-tests above reject items that certainly fail; the functions
// below accept items that certainly pass and evaluate them from FP32
// geometry.  An item is taken here only when every decision of the exact
// FP64 test has a margin far above the FP32 error of the quantity it
// compares -- so the FP64 test decides the same way -- and only when its
// value is well conditioned:
//   - facing: the cast direction is within 60 degrees of the master normal
//     (face), or some adjacent master face has N.n_s <= -0.1 |N| (edge,
//     point);
//   - eps = eps_max is settled by the rest-box test (rest_far), so no rest
//     cast is needed;
//   - 0.2 eps + tol_g <= g <= 0.95 eps - tol_g: away from g = 0, where B'
//     ~ 1/g magnifies the gap's relative error, and from g = eps, where the
//     factor (g - eps) of B, B', B'' would carry it;
//   - inside with margin: min beta^m >= tol_b (face), a clipped parameter
//     range longer than its error (edge), min beta^s >= tol_b (point);
//   - a static master (dxm == NULL), so the step bound needs only the slave
//     side's gap change.
// Error bounds.  Coordinates enter as FP64 differences rounded once to FP32
// (relative error 2^-24) and pass through a few dozen FP32 operations: the
// first-order error of a gap or barycentric coordinate is below about 1e-6
// of the magnitudes involved, times the triangle's shape factor
// |e1||e2|/|N| and, for a cast, 1 / cos of its angle.  tol_g and tol_b are
// 1e-4 of the same magnitudes and factors, a hundred times that; the
// edge/point tolerances reuse those of bary_f and plane_gap_maybe, stated
// there.  Every other item goes to the FP64 test as before.  The step bound
// of a certified item uses the gap's lower bound g - tol_g and an upper
// bound of its closing rate, so it never exceeds the FP64 bound.
// ---------------------------------------------------------------------------
constexpr float kCertLo = 0.2f, kCertHi = 0.95f;

__device__ __forceinline__ float norm3f(V3<float> a) { return sqrtf(dot(a, a)); }

// barycentric coordinates of q (relative to the triangle's first vertex) in
// the frame (e1, e2), by the Gram system of Eq. (gram)
__device__ __forceinline__ void bary_rel(V3<float> q, V3<float> e1, V3<float> e2, float* b) {
    const float a = dot(e1, e1), bb = dot(e1, e2), c = dot(e2, e2);
    const float r1 = dot(q, e1), r2 = dot(q, e2);
    const float det = a * c - bb * bb;
    const float v = (c * r1 - bb * r2) / det, w = (a * r2 - bb * r1) / det;
    b[0] = 1.0f - v - w; b[1] = v; b[2] = w;
}

// master triangle m's edges y1 - y0, y2 - y0 rounded to FP32: read from
// the per-pass table (PRE, see k_mtri_e32) or formed from xm -- the same values
template <bool PRE>
__device__ __forceinline__ void mtri_edges(const SceneView& S, const double* xm, const float* mtri_e, int64_t m,
                                           V3<float>& e1, V3<float>& e2) {
    if (PRE && mtri_e) {
        const float* E = mtri_e + 8 * m;
        e1 = {E[0], E[1], E[2]};
        e2 = {E[3], E[4], E[5]};
    } else {
        const int32_t* M = S.mtri + 3 * m;
        const V3<double> y0 = ld3(xm, M[0]);
        e1 = tof(ld3(xm, M[1]) - y0);
        e2 = tof(ld3(xm, M[2]) - y0);
    }
}
// some master face of the list certainly faces n_s (N . n_s <= -0.1 |N|)
template <bool PRE = false>
__device__ __forceinline__ bool facing_cert(const SceneView& S, const double* xm, const int32_t* tris, int n,
                                            V3<float> ns, const float* mtri_e = nullptr) {
    for (int i = 0; i < n; ++i) {
        V3<float> e1, e2;
        mtri_edges<PRE>(S, xm, mtri_e, tris[i], e1, e2);
        const V3<float> N = cross(e1, e2);
        if (dot(N, ns) <= -0.1f * norm3f(N)) return true;
    }
    return false;
}

// face sample F of slave tri D against master tri m (Sec. 4.1, reading R1),
// in the master triangle's frame
template <int NK>
__device__ __forceinline__ bool face_cert(const SceneView& S, const Params& P, const TriData& D,
                                          const FaceSample& F, const double* xm, int32_t m, bool want_dg,
                                          ItemOut& o) {
    const double eps = P.dhat;
    const double* mb = S.mrest_box + 6 * (int64_t)m;
    if (!rest_far(D.sb, D.sb + 3, mb, mb + 3, eps)) return false;
    const int32_t* M = S.mtri + 3 * (int64_t)m;
    const V3<double> y0 = ld3(xm, M[0]);
    V3<float> e1, e2;
    mtri_edges<false>(S, xm, nullptr, m, e1, e2);
    const V3<float> d = tof(y0 - F.xs);
    const V3<float> N = cross(e1, e2);
    const float nN = norm3f(N);
    const float cosn = -dot(N, D.ns_f) / nN;
    if (!(cosn >= 0.5f)) return false;
    const float g = dot(N, d) / (-cosn * nN);
    const float l1 = norm3f(e1), l2 = norm3f(e2), l3 = norm3f(e2 - e1);
    const float shape = l1 * l2 / nN;
    const float tol_g = 1e-4f * (norm3f(d) + fabsf(g)) * shape / cosn;
    const float epsf = (float)eps;
    if (!(g - tol_g >= kCertLo * epsf && g + tol_g <= kCertHi * epsf)) return false;
    const V3<float> q = g * D.ns_f - d;   // hit point relative to y0
    float bm[3];
    bary_rel(q, e1, e2, bm);
    const float hmin = nN / rmax(l1, rmax(l2, l3));
    const float tol_b = 1e-4f + (tol_g + 1e-4f * norm3f(q)) * shape / hmin;
    if (!(min3(bm) >= tol_b)) return false;
    o.kq = P.kappa; o.w = (1.0 / (double)NK) * D.As; o.gamma = (double)hermite(min3(bm), (float)P.delta_T);
    o.g = (double)g; o.g_step = (double)g - (double)tol_g; o.eps = eps;
    for (int c = 0; c < 3; ++c) { o.b[c] = F.beta[c]; o.mv[c] = M[c]; o.bm[c] = (double)bm[c]; }
    o.dg = want_dg ? -F.ds : 0.0;
    return true;
}

// the slave-side closing rate of a certified edge or point item: dg =
// -n_s . sum_a b_a dx_a with b from FP32 geometry (error <= tol_b each),
// widened toward closing by tol_b sum_a |n_s . dx_a|
__device__ __forceinline__ double cert_dg(const TriData& D, const double* b, float tol_b) {
    const double s0 = dot(D.ns, D.dx0), s1 = dot(D.ns, D.dx1), s2 = dot(D.ns, D.dx2);
    const double ds = b[0] * s0 + b[1] * s1 + b[2] * s2;
    return -ds - (double)tol_b * (fabs(s0) + fabs(s1) + fabs(s2));
}

// Gauss point q of master edge me projected on slave tri D (Sec. 4.1,
// reading R3).  Barycentric coordinates are affine along the projected
// edge, so beta^s and the plane gap at a Gauss point are the ends' values
// mixed by eta.
__device__ __forceinline__ bool edge_cert(const SceneView& S, const Params& P, const TriData& D,
                                          const double* xm, int32_t me, int q, bool want_dg, ItemOut& o) {
    const double eps = P.dhat;
    const int ia = S.medge[2 * (int64_t)me], ib = S.medge[2 * (int64_t)me + 1];
    {
        const V3<double> Ya = ld3(S.Y0, ia), Yb = ld3(S.Y0, ib);
        const double elo[3] = {rmin(Ya.x, Yb.x), rmin(Ya.y, Yb.y), rmin(Ya.z, Yb.z)};
        const double ehi[3] = {rmax(Ya.x, Yb.x), rmax(Ya.y, Yb.y), rmax(Ya.z, Yb.z)};
        if (!rest_far(D.sb, D.sb + 3, elo, ehi, eps)) return false;
    }
    const int a0 = S.me_tri_off[me], a1 = S.me_tri_off[me + 1];
    if (!facing_cert<false>(S, xm, S.me_tri + a0, a1 - a0, D.ns_f)) return false;
    const V3<double> ya = ld3(xm, ia), yb = ld3(xm, ib);
    const V3<float> da = tof(ya - D.x0), db = tof(yb - D.x0);
    float bA[3], bB[3], tA, tB;
    bool okA, okB;
    bary_f(da, D.e1_f, D.e2_f, bA, tA, okA);
    bary_f(db, D.e1_f, D.e2_f, bB, tB, okB);
    if (!okA || !okB) return false;
    const float tb = tA + tB;
    // clip eta by beta_a(eta) = bA + eta (bB - bA) >= 0, with error bounds on
    // both ends of the range
    float lo = 0.0f, hi = 1.0f, elo_t = 0.0f, ehi_t = 0.0f;
    for (int a = 0; a < 3; ++a) {
        const float Dd = bB[a] - bA[a];
        if (fabsf(Dd) <= 4.0f * tb) {
            // nearly parallel to slave edge a: certain only if inside all along
            if (rmin(bA[a], bB[a]) >= tb) continue;
            return false;
        }
        const float r = -bA[a] / Dd;
        const float er = (tA + fabsf(r) * tb) / (fabsf(Dd) - tb);
        if (Dd > 0.0f) { if (r > lo) { lo = r; elo_t = er; } }
        else if (r < hi) { hi = r; ehi_t = er; }
    }
    if (!(hi - lo > 4.0f * (elo_t + ehi_t) + 1e-3f)) return false;
    const float gp = 0.57735026918962576f;   // 1 / sqrt(3)
    const float mid = 0.5f * (lo + hi), half = 0.5f * (hi - lo);
    const float eta = q == 0 ? mid - half * gp : mid + half * gp;
    const float ga = dot(D.ns_f, da), gb = dot(D.ns_f, db);
    const float g = (1.0f - eta) * ga + eta * gb;
    const float tol_g = 1e-5f * (fabsf(da.x) + fabsf(da.y) + fabsf(da.z) + fabsf(db.x) + fabsf(db.y) + fabsf(db.z)) +
                        fabsf(gb - ga) * (elo_t + ehi_t) + D.tol_abs;
    const float epsf = (float)eps;
    if (!(g - tol_g >= kCertLo * epsf && g + tol_g <= kCertHi * epsf)) return false;
    const V3<float> tv = db - da;
    const float tn = dot(tv, D.ns_f);
    const V3<float> tp = tv - tn * D.ns_f;
    const float ell = (hi - lo) * norm3f(tp);
    o.kq = P.kappa_edge; o.w = 0.5 * (double)ell;
    o.gamma = (double)(hermite(eta, (float)P.delta_e) * hermite(1.0f - eta, (float)P.delta_e));
    o.g = (double)g; o.g_step = (double)g - (double)tol_g; o.eps = eps;
    for (int c = 0; c < 3; ++c) o.b[c] = (double)((1.0f - eta) * bA[c] + eta * bB[c]);
    o.mv[0] = ia; o.mv[1] = ib; o.mv[2] = -1;
    o.bm[0] = 1.0 - (double)eta; o.bm[1] = (double)eta; o.bm[2] = 0.0;
    o.dg = want_dg ? cert_dg(D, o.b, tb) : 0.0;
    return true;
}

// master vertex u projected on slave tri D (Sec. 4.1, reading R3)
__device__ __forceinline__ bool point_cert(const SceneView& S, const Params& P, const TriData& D,
                                           const double* xm, int32_t u, bool want_dg, ItemOut& o) {
    const double eps = P.dhat;
    {
        const V3<double> Y = ld3(S.Y0, u);
        const double yb[3] = {Y.x, Y.y, Y.z};
        if (!rest_far(D.sb, D.sb + 3, yb, yb, eps)) return false;
    }
    const int a0 = S.mv_tri_off[u], a1 = S.mv_tri_off[u + 1];
    if (!facing_cert<false>(S, xm, S.mv_tri + a0, a1 - a0, D.ns_f)) return false;
    const V3<float> d = tof(ld3(xm, u) - D.x0);
    float bs[3], tb;
    bool ok;
    bary_f(d, D.e1_f, D.e2_f, bs, tb, ok);
    if (!ok || !(min3(bs) >= tb)) return false;
    const float g = dot(D.ns_f, d);
    const float tol_g = 1e-5f * (fabsf(d.x) + fabsf(d.y) + fabsf(d.z)) + D.tol_abs;
    const float epsf = (float)eps;
    if (!(g - tol_g >= kCertLo * epsf && g + tol_g <= kCertHi * epsf)) return false;
    o.kq = P.kappa_point; o.w = 1.0; o.gamma = 1.0;
    o.g = (double)g; o.g_step = (double)g - (double)tol_g; o.eps = eps;
    for (int c = 0; c < 3; ++c) o.b[c] = (double)bs[c];
    o.mv[0] = u; o.mv[1] = -1; o.mv[2] = -1;
    o.bm[0] = 1.0; o.bm[1] = 0.0; o.bm[2] = 0.0;
    o.dg = want_dg ? cert_dg(D, o.b, tb) : 0.0;
    return true;
}

// ---- certified items of the middle stage, in FP32 throughout ----------
// The same certificates as face_cert / edge_cert / point_cert (PRE), with
// the item's weight, gap, barycentrics and closing rate kept in FP32: the
// only FP64 operations left are the master positions relative to x0 (an
// FP64 difference rounded once) and the two results stored.
struct CertOut {
    float coef;      // kappa_q w gamma
    float g, gstep;  // the gap and a certified lower bound of it
    float dg;        // the linearised gap change along dx, widened toward closing (0 without dx)
    float b[3];      // slave barycentrics
};

__device__ __forceinline__ float l1f(V3<float> v) { return fabsf(v.x) + fabsf(v.y) + fabsf(v.z); }

// dg = -n_s . sum_a b_a dx_a from the frame kernel's FP32 products, widened
// toward closing by (tol_b + 2^-21) sum_a |n_s . dx_a| (tol_b the error of
// each b_a, 2^-21 that of the FP32 products and sums, b_a <= 1 + tol_b)
__device__ __forceinline__ float cert_dg_f(const TriData& D, const float* b, float tol_b) {
    const float ds = b[0] * D.sdxf[0] + b[1] * D.sdxf[1] + b[2] * D.sdxf[2];
    return -ds - (tol_b + 4.8e-7f) * D.sdxf[3];
}

// face sample k of slave tri D against master tri m.  The offset from the
// sample to y0 is (y0 - x0) rounded to FP32 minus b1 e1 + b2 e2 in FP32, so
// its error is below 2^-21 (|y0 - x0| + |e1| + |e2|) (1-norms); that bound
// enters the gap and barycentric tolerances on top of face_cert's.
template <int NK>
__device__ __forceinline__ bool face_cert_f(const SceneView& S, const Params& P, const TriData& D, int k,
                                            const double* xm, int32_t m, bool want_dg, CertOut& o,
                                            const float* mtri_e) {
    const double* mb = S.mrest_box + 6 * (int64_t)m;
    const float* mf = S.mrest_box_f + 6 * (int64_t)m;
    if (!rest_far_f(D.sbf, D.sbf + 3, mf, mf + 3, P.far_r2_f) && !rest_far(D.sb, D.sb + 3, mb, mb + 3, P.dhat))
        return false;
    const int32_t* M = S.mtri + 3 * (int64_t)m;
    const V3<float> a = tof(ld3(xm, M[0]) - D.x0);
    const float b0 = c_rule_f[P.L - 1][k][0], b1 = c_rule_f[P.L - 1][k][1], b2 = c_rule_f[P.L - 1][k][2];
    const V3<float> d = a - (b1 * D.e1_f + b2 * D.e2_f);
    const float dd = 4.8e-7f * (l1f(a) + l1f(D.e1_f) + l1f(D.e2_f));
    V3<float> e1, e2;
    mtri_edges<true>(S, xm, mtri_e, m, e1, e2);
    const V3<float> N = cross(e1, e2);
    const float nN = norm3f(N);
    const float cosn = -dot(N, D.ns_f) / nN;
    if (!(cosn >= 0.5f)) return false;
    const float g = dot(N, d) / (-cosn * nN);
    const float l1 = norm3f(e1), l2 = norm3f(e2), l3 = norm3f(e2 - e1);
    const float shape = l1 * l2 / nN;
    const float tol_g = (1e-4f * (norm3f(d) + fabsf(g)) + dd) * shape / cosn;
    if (!(g - tol_g >= kCertLo * P.dhat_hi && g + tol_g <= kCertHi * P.dhat_hi)) return false;
    const V3<float> q = g * D.ns_f - d;   // hit point relative to y0
    float bm[3];
    bary_rel(q, e1, e2, bm);
    const float hmin = nN / rmax(l1, rmax(l2, l3));
    const float tol_b = 1e-4f + (tol_g + 1e-4f * norm3f(q) + dd) * shape / hmin;
    if (!(min3(bm) >= tol_b)) return false;
    o.coef = P.kappa_f * D.w_f * hermite(min3(bm), P.delta_T_f);
    o.g = g;
    o.gstep = g - tol_g;
    o.b[0] = b0; o.b[1] = b1; o.b[2] = b2;
    o.dg = want_dg ? cert_dg_f(D, o.b, 0.0f) : 0.0f;
    return true;
}

// Gauss point q of master edge me on slave tri D: edge_cert's certificate
// (its FP32 geometry and tolerances unchanged), the item kept in FP32
__device__ __forceinline__ bool edge_cert_f(const SceneView& S, const Params& P, const TriData& D,
                                            const double* xm, int32_t me, int q, bool want_dg, CertOut& o,
                                            const float* mtri_e) {
    const int ia = S.medge[2 * (int64_t)me], ib = S.medge[2 * (int64_t)me + 1];
    {
        const float* va = S.mvrest_box_f + 6 * (int64_t)ia;
        const float* vb = S.mvrest_box_f + 6 * (int64_t)ib;
        const float flo[3] = {fminf(va[0], vb[0]), fminf(va[1], vb[1]), fminf(va[2], vb[2])};
        const float fhi[3] = {fmaxf(va[3], vb[3]), fmaxf(va[4], vb[4]), fmaxf(va[5], vb[5])};
        if (!rest_far_f(D.sbf, D.sbf + 3, flo, fhi, P.far_r2_f)) {
            const V3<double> Ya = ld3(S.Y0, ia), Yb = ld3(S.Y0, ib);
            const double elo[3] = {rmin(Ya.x, Yb.x), rmin(Ya.y, Yb.y), rmin(Ya.z, Yb.z)};
            const double ehi[3] = {rmax(Ya.x, Yb.x), rmax(Ya.y, Yb.y), rmax(Ya.z, Yb.z)};
            if (!rest_far(D.sb, D.sb + 3, elo, ehi, P.dhat)) return false;
        }
    }
    const int a0 = S.me_tri_off[me], a1 = S.me_tri_off[me + 1];
    if (!facing_cert<true>(S, xm, S.me_tri + a0, a1 - a0, D.ns_f, mtri_e)) return false;
    const V3<float> da = tof(ld3(xm, ia) - D.x0), db = tof(ld3(xm, ib) - D.x0);
    float bA[3], bB[3], tA, tB;
    bool okA, okB;
    bary_f(da, D.e1_f, D.e2_f, bA, tA, okA);
    bary_f(db, D.e1_f, D.e2_f, bB, tB, okB);
    if (!okA || !okB) return false;
    const float tb = tA + tB;
    float lo = 0.0f, hi = 1.0f, elo_t = 0.0f, ehi_t = 0.0f;
    for (int a = 0; a < 3; ++a) {
        const float Dd = bB[a] - bA[a];
        if (fabsf(Dd) <= 4.0f * tb) {
            if (rmin(bA[a], bB[a]) >= tb) continue;
            return false;
        }
        const float r = -bA[a] / Dd;
        const float er = (tA + fabsf(r) * tb) / (fabsf(Dd) - tb);
        if (Dd > 0.0f) { if (r > lo) { lo = r; elo_t = er; } }
        else if (r < hi) { hi = r; ehi_t = er; }
    }
    if (!(hi - lo > 4.0f * (elo_t + ehi_t) + 1e-3f)) return false;
    const float gp = 0.57735026918962576f;   // 1 / sqrt(3)
    const float mid = 0.5f * (lo + hi), half = 0.5f * (hi - lo);
    const float eta = q == 0 ? mid - half * gp : mid + half * gp;
    const float ga = dot(D.ns_f, da), gb = dot(D.ns_f, db);
    const float g = (1.0f - eta) * ga + eta * gb;
    const float tol_g = 1e-5f * (l1f(da) + l1f(db)) + fabsf(gb - ga) * (elo_t + ehi_t) + D.tol_abs;
    if (!(g - tol_g >= kCertLo * P.dhat_hi && g + tol_g <= kCertHi * P.dhat_hi)) return false;
    const V3<float> tv = db - da;
    const float tn = dot(tv, D.ns_f);
    const V3<float> tp = tv - tn * D.ns_f;
    const float ell = (hi - lo) * norm3f(tp);
    o.coef = P.kappa_edge_f * (0.5f * ell) * (hermite(eta, P.delta_e_f) * hermite(1.0f - eta, P.delta_e_f));
    o.g = g;
    o.gstep = g - tol_g;
    for (int c = 0; c < 3; ++c) o.b[c] = (1.0f - eta) * bA[c] + eta * bB[c];
    o.dg = want_dg ? cert_dg_f(D, o.b, tb) : 0.0f;
    return true;
}

// master vertex u on slave tri D: point_cert's certificate, kept in FP32
__device__ __forceinline__ bool point_cert_f(const SceneView& S, const Params& P, const TriData& D,
                                             const double* xm, int32_t u, bool want_dg, CertOut& o,
                                             const float* mtri_e) {
    {
        const float* vu = S.mvrest_box_f + 6 * (int64_t)u;
        if (!rest_far_f(D.sbf, D.sbf + 3, vu, vu + 3, P.far_r2_f)) {
            const V3<double> Y = ld3(S.Y0, u);
            const double yb[3] = {Y.x, Y.y, Y.z};
            if (!rest_far(D.sb, D.sb + 3, yb, yb, P.dhat)) return false;
        }
    }
    const int a0 = S.mv_tri_off[u], a1 = S.mv_tri_off[u + 1];
    if (!facing_cert<true>(S, xm, S.mv_tri + a0, a1 - a0, D.ns_f, mtri_e)) return false;
    const V3<float> d = tof(ld3(xm, u) - D.x0);
    float bs[3], tb;
    bool ok;
    bary_f(d, D.e1_f, D.e2_f, bs, tb, ok);
    if (!ok || !(min3(bs) >= tb)) return false;
    const float g = dot(D.ns_f, d);
    const float tol_g = 1e-5f * l1f(d) + D.tol_abs;
    if (!(g - tol_g >= kCertLo * P.dhat_hi && g + tol_g <= kCertHi * P.dhat_hi)) return false;
    o.coef = P.kappa_point_f;
    o.g = g;
    o.gstep = g - tol_g;
    for (int c = 0; c < 3; ++c) o.b[c] = bs[c];
    o.dg = want_dg ? cert_dg_f(D, o.b, tb) : 0.0f;
    return true;
}

// value of a certified FP32 item (eps = dhat): the barrier's B, B' and B''
// (as barrier() forms them) in FP32, with d = g - dhat formed against
// dhat's FP32 pair (exact where g is within a factor two of dhat) and
// d / dhat as a product with 1 / dhat, and the step bound 0.9 gstep / (-dg)
// in FP32 lowered by 2e-6 (more than its rounding), so it stays at or
// below the FP64 path's
__device__ __forceinline__ void item_value_cert_f(const CertOut& o, bool want_dg, const Params& P, double& e,
                                                  double& amin, float& c1, float& c2, float* b) {
    const float d = (o.g - P.dhat_hi) - P.dhat_lo;
    const float L = log1pf(d * P.inv_dhat_f);
    const float r = d / o.g;
    const float Bv = -d * d * L;
    const float dB = -2.0f * d * L - d * r;
    const float d2B = -2.0f * L - 4.0f * r + r * r;
    e = (double)(o.coef * Bv);
    c1 = o.coef * dB;
    c2 = rmax(o.coef * d2B, 0.0f);
    for (int cc = 0; cc < 3; ++cc) b[cc] = o.b[cc];
    amin = INFINITY;
    if (want_dg && o.dg < 0.0f) amin = (double)(0.9f * o.gstep / (-o.dg) * (1.0f - 2e-6f));
}

// the value of an item for the evaluation: energy, c1, c2, slave
// barycentrics and its step bound (the arithmetic of sample_add)
template <class T>
__device__ __forceinline__ void item_value(const ItemOut& o, bool want_dg, double& e, double& amin, T& c1, T& c2,
                                           T* b) {
    T Bv, dB, d2B;
    barrier(o.g, o.eps, Bv, dB, d2B);
    const T coef = (T)(o.kq * o.w * o.gamma);
    e = (double)(coef * Bv);
    c1 = coef * dB;
    c2 = rmax(coef * d2B, T(0));
    for (int cc = 0; cc < 3; ++cc) b[cc] = (T)o.b[cc];
    amin = INFINITY;
    if (want_dg && o.dg < 0.0) amin = 0.9 * o.g_step / (-o.dg);
}
// The paper's clipped-overlap face samples of slave tri D against master
// tri m (Sec. 4.1 "Face samples", ipc_params.face_sampler = 1): the pair
// counts when the master triangle faces the slave (N . n_s < 0); each clip
// sample (fclip::clip_samples) is active when 0 < g < eps, eps from the same
// slave point at rest cast onto the rest master (Eq. adaptive_eps, reading
// R5), with weight w = its Gauss weight (area / 3) and gamma =
// H(min beta^m, delta_T) (Eq. gamma).  emit(o) is called for each.
template <class Emit>
__device__ __forceinline__ int face_clip_items(const SceneView& S, const Params& P, const TriData& D,
                                               const double* xm, const double* dxm, int32_t m, bool want_dg,
                                               Emit&& emit) {
    const int32_t* M = S.mtri + 3 * (int64_t)m;
    const V3<double> y0 = ld3(xm, M[0]), y1 = ld3(xm, M[1]), y2 = ld3(xm, M[2]);
    if (!(dot(cross(y1 - y0, y2 - y0), D.ns) < 0.0)) return 0;
    const double* mb = S.mrest_box + 6 * (int64_t)m;
    const bool far0 = rest_far(D.sb, D.sb + 3, mb, mb + 3, P.dhat);
    auto p3 = [](V3<double> v) { return fclip::P3{v.x, v.y, v.z}; };
    return fclip::clip_samples(p3(D.x0), p3(D.x1), p3(D.x2), p3(y0), p3(y1), p3(y2),
                               [&](const double* bs, const double* bm, double g, double w) {
        if (!(g > 0.0)) return;
        double eps = P.dhat;
        if (!far0) {
            const V3<double> xs0 = interp(bs, D.X0, D.X1, D.X2);
            double g0, bm0[3];
            if (face_geom<double>(xs0, D.ns0, ld3(S.Y0, M[0]), ld3(S.Y0, M[1]), ld3(S.Y0, M[2]), g0, bm0))
                eps = rmin(0.9 * g0, P.dhat);
        }
        if (!(g < eps)) return;
        ItemOut o;
        o.kq = P.kappa; o.w = w; o.gamma = hermite(min3(bm), P.delta_T);
        o.g = g; o.g_step = g; o.eps = eps;
        for (int c = 0; c < 3; ++c) { o.b[c] = bs[c]; o.mv[c] = M[c]; o.bm[c] = bm[c]; }
        o.dg = 0.0;
        if (want_dg) {
            const double ds = dot(D.ns, interp(bs, D.dx0, D.dx1, D.dx2));
            const double dm = dxm ? dot(D.ns, interp(bm, ld3(dxm, M[0]), ld3(dxm, M[1]), ld3(dxm, M[2]))) : 0.0;
            o.dg = dm - ds;
        }
        emit(o);
    });
}

// Warp per active triangle (persistent grid).  Used for the step bound and
// the lagged energies of the line search, and for the contact evaluation
// when the item buffer is too small (then run_if_over selects it).
__device__ void put_block(const ModeArgs& LG, int32_t r, int32_t c, double coef, const V3<double>& n) {
    const unsigned long long at = atomicAdd(LG.h_count, 1ull);
    if ((int64_t)at >= LG.h_cap) return;
    LG.h_ij[2 * at] = r; LG.h_ij[2 * at + 1] = c;
    double* b = LG.h_blk + 9 * at;
    const double nn[3] = {n.x, n.y, n.z};
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) b[3 * p + q] = coef * nn[p] * nn[q];
}

// the sample's gap gradient is (-beta_a n_s) on its slave vertices Ts[a] and
// (bm_j n_s) on its master vertices; its Gauss-Newton block between two of
// them is max(kappa w gamma B''(g), 0) w_u w_v n_s n_s^T
__device__ void master_blocks(const ModeArgs& LG, const ItemOut& o, const int32_t* Ts, const V3<double>& ns) {
    double Bv, dB, d2B;
    barrier(o.g, o.eps, Bv, dB, d2B);
    const double c2 = rmax(o.kq * o.w * o.gamma * d2B, 0.0);
    const double c1 = o.kq * o.w * o.gamma * dB;
    for (int j = 0; j < 3; ++j) {
        if (o.mv[j] < 0) continue;
        const int32_t cj = LG.m_off + o.mv[j];
        if (LG.h_rows) {
            const unsigned long long at = atomicAdd(LG.h_count, 1ull);
            if ((int64_t)at < LG.h_cap) {
                LG.h_ij[2 * at] = cj; LG.h_ij[2 * at + 1] = -1;
                double* b = LG.h_blk + 9 * at;
                const double f = c1 * o.bm[j];
                b[0] = f * ns.x; b[1] = f * ns.y; b[2] = f * ns.z;
                for (int q = 3; q < 9; ++q) b[q] = 0.0;
            }
        }
        if (!LG.h_blocks) continue;
        for (int a = 0; a < 3; ++a) put_block(LG, Ts[a], cj, -c2 * o.b[a] * o.bm[j], ns);
        for (int i = 0; i < 3; ++i)
            if (o.mv[i] >= 0) put_block(LG, LG.m_off + o.mv[i], cj, c2 * o.bm[i] * o.bm[j], ns);
    }
}

template <int NK, class T, int MODE, bool CLIP = false>
__global__ void __launch_bounds__(256)
k_samples(SceneView S, Params P, CandView C, const double* __restrict__ x,
          const double* __restrict__ xm, double* __restrict__ triE, T* __restrict__ triG,
          T* __restrict__ triS, T* __restrict__ triN, long long* counters,
          const double* __restrict__ dx, const double* __restrict__ dxm,
          unsigned long long* alpha_bits, ModeArgs LG, const double* __restrict__ frame,
          const int32_t* __restrict__ run_if_over, int64_t item_cap) {
    pass_dep_wait();
    if (run_if_over && (int64_t)*run_if_over <= item_cap) return;
    const int lane = threadIdx.x & 31;
    const int n_active = *C.n_active;
    long long cnt_f = 0, cnt_e = 0, cnt_p = 0, cnt_eval = 0;
    double al8[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) al8[j] = (MODE == MODE_LAGGED && j < LG.na) ? LG.alphas[j] : 0.0;
    const bool pre = P.precision == IPC_PREC_MIXED;   // FP32 pre-tests (exact decisions unchanged)
    const bool want_dg = dx != nullptr;
    const bool want_alpha = MODE != MODE_LAGGED && want_dg;
    const bool cert = pre && MODE == MODE_EVAL && dxm == nullptr;   // certified FP32 items
    for (int i = next_item(C.work, lane); i < n_active; i = next_item(C.work, lane)) {
        const TriData D = load_tri(S, C, x, dx, frame, i);
        if (MODE == MODE_LAGGED && LG.alphas_stride > 0) {
            const double* ae = LG.alphas + (int64_t)LG.alphas_stride * S.stri_env[D.t];
#pragma unroll
            for (int j = 0; j < 8; ++j) al8[j] = j < LG.na ? ae[j] : 0.0;
        }
        Acc<T> A;
        A.zero();
        double E8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) E8[j] = 0.0;
        auto consume = [&](const ItemOut& o) {
            if (MODE == MODE_EVAL) sample_add<T>(A, o.kq, o.w, o.gamma, o.g, o.eps, o.b);
            if (MODE == MODE_MASTER_HESS) master_blocks(LG, o, S.stri + 3 * D.t, D.ns);
            if (want_dg) {
                if (want_alpha && o.dg < 0.0) A.amin = rmin(A.amin, 0.9 * o.g_step / (-o.dg));
                if (MODE == MODE_LAGGED) lag_add(E8, al8, LG.na, o.kq * o.w * o.gamma, o.g, o.eps, o.dg);
            }
        };
        // face items (lane, lane + 32, ...): 32 is a multiple of NK, so each
        // lane keeps one sample
        if (CLIP) {
            // clipped-overlap samples: one lane per candidate pair
            const int32_t* Lf = C.face + D.t * C.cap_f;
            for (int j = lane; j < D.nf; j += 32)
                cnt_eval += face_clip_items(S, P, D, xm, dxm, Lf[j], want_dg, [&](const ItemOut& o) {
                    ++cnt_f;
                    consume(o);
                });
        } else {
            const FaceSample F = face_sample(P, D, lane % NK, want_dg);
            const int32_t* Lf = C.face + D.t * C.cap_f;
            for (int it = lane; it < D.nf * NK; it += 32) {
                ++cnt_eval;
                ItemOut o;
                if (!(cert && face_cert<NK>(S, P, D, F, xm, Lf[it / NK], want_dg, o)) &&
                    !face_item<NK>(S, P, D, F, xm, dxm, Lf[it / NK], pre, want_dg, o))
                    continue;
                ++cnt_f;
                consume(o);
            }
        }
        {
            const int32_t* Le = C.edge + D.t * C.cap_e;
            for (int it = lane; it < D.ne * 2; it += 32) {
                ItemOut o;
                if (!(cert && edge_cert(S, P, D, xm, Le[it >> 1], it & 1, want_dg, o)) &&
                    !edge_item(S, P, D, xm, dxm, Le[it >> 1], it & 1, pre, want_dg, o))
                    continue;
                ++cnt_e;
                consume(o);
            }
        }
        {
            const int32_t* Lp = C.point + D.t * C.cap_p;
            for (int it = lane; it < D.np; it += 32) {
                ItemOut o;
                if (!(cert && point_cert(S, P, D, xm, Lp[it], want_dg, o)) &&
                    !point_item(S, P, D, xm, dxm, Lp[it], pre, want_dg, o))
                    continue;
                ++cnt_p;
                consume(o);
            }
        }
        // ---------------- fixed-order warp reduction ----------------
        if (MODE == MODE_EVAL) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                A.E += shfl_x(A.E, o);
#pragma unroll
                for (int q = 0; q < 3; ++q) A.G[q] += shfl_x(A.G[q], o);
#pragma unroll
                for (int q = 0; q < 6; ++q) A.S[q] += shfl_x(A.S[q], o);
            }
            if (lane == 0) {
                const int64_t t = D.t;
                triE[t] = A.E;
                for (int q = 0; q < 3; ++q) triG[3 * t + q] = A.G[q];
                for (int q = 0; q < 6; ++q) triS[6 * t + q] = A.S[q];
                triN[3 * t + 0] = (T)D.ns.x; triN[3 * t + 1] = (T)D.ns.y; triN[3 * t + 2] = (T)D.ns.z;
            }
        }
        if (MODE == MODE_LAGGED) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) E8[j] += shfl_x(E8[j], o);
            if (lane == 0)
                for (int j = 0; j < LG.na; ++j) LG.triE8[(int64_t)j * LG.ns + D.t] = E8[j];
        }
        if (want_alpha) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) A.amin = rmin(A.amin, shfl_x(A.amin, o));
            if (lane == 0 && A.amin < INFINITY)
                atomicMin(alpha_bits + (int64_t)LG.alpha_stride * S.stri_env[D.t],
                          (unsigned long long)__double_as_longlong(A.amin));
        }
    }
    // counters (integers: order does not matter)
    if (counters) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt_f += shfl_x(cnt_f, o); cnt_e += shfl_x(cnt_e, o);
            cnt_p += shfl_x(cnt_p, o); cnt_eval += shfl_x(cnt_eval, o);
        }
        if (lane == 0 && (cnt_f | cnt_e | cnt_p | cnt_eval)) {
            atomic_add_ll(&counters[0], cnt_f); atomic_add_ll(&counters[1], cnt_e);
            atomic_add_ll(&counters[2], cnt_p); atomic_add_ll(&counters[3], cnt_eval);
        }
    }
}

// ---------------------------------------------------------------------------
// the contact evaluation, one thread per sample item
//
// The warp-per-triangle kernel leaves most lanes idle when a triangle has
// few candidates and hides little latency.  Here k_fill_owner maps every
// item slot to its triangle, k_items evaluates one item per thread and
// stores its contribution (energy, c1, c2, slave barycentrics, step bound),
// and k_tri_reduce sums each triangle's items with exactly the lane
// assignment and shuffle tree of the warp-per-triangle kernel, so the
// results are bitwise the same.
// ---------------------------------------------------------------------------
struct ItemBufs {
    int32_t* owner;      // [cap] active index of the slot's triangle
    double* rd;          // [cap][2] energy, step bound
    void* rt;            // [cap][5] c1, c2, b0, b1, b2 (T)
    const int32_t* n;    // items requested
    int64_t cap;
    uint32_t* mask;      // [cap / 32 + 1] bit set: the slot holds a record (else it contributes nothing)
};

// master vertices minus their environment's grid origin, rounded to FP32
// (w = 0): the master side of the face items' FP32 pre-filter
__global__ void k_master_f32(SceneView S, const double* __restrict__ xm, float4* __restrict__ ym32) {
    pass_dep_wait();
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= S.nmv) return;
    const int e = S.mvert_env[u];
    ym32[u] = make_float4((float)(xm[3 * u] - S.grid_org[3 * e]), (float)(xm[3 * u + 1] - S.grid_org[3 * e + 1]),
                          (float)(xm[3 * u + 2] - S.grid_org[3 * e + 2]), 0.0f);
}

// What the FP32 face pre-filter needs of a master triangle, once per pass
// from the FP32 master vertices (the same operations face_reject_f32 would
// run per item): [24 m ...] = y0 (3), e1 = y1 - y0 (3), e2 = y2 - y0 (3),
// N = e1 x e2 (3), |N|, |e1|, |e2|, |e2 - e1|, max |coordinate| of the
// three vertices, e1.e1, e1.e2, e2.e2, their Gram determinant, 3 unused.
constexpr int kMtriPre = 24;
__global__ void k_mtri_pre(SceneView S, const float4* __restrict__ ym32, float* __restrict__ out) {
    pass_dep_wait();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= S.nmt) return;
    const int32_t* M = S.mtri + 3 * m;
    const float4 A = ym32[M[0]], B4 = ym32[M[1]], C4 = ym32[M[2]];
    const V3<float> y0 = {A.x, A.y, A.z}, y1 = {B4.x, B4.y, B4.z}, y2 = {C4.x, C4.y, C4.z};
    const V3<float> e1 = y1 - y0, e2 = y2 - y0, N = cross(e1, e2);
    float* o = out + kMtriPre * m;
    o[0] = y0.x; o[1] = y0.y; o[2] = y0.z;
    o[3] = e1.x; o[4] = e1.y; o[5] = e1.z;
    o[6] = e2.x; o[7] = e2.y; o[8] = e2.z;
    o[9] = N.x; o[10] = N.y; o[11] = N.z;
    o[12] = sqrtf(dot(N, N));
    o[13] = sqrtf(dot(e1, e1));
    o[14] = sqrtf(dot(e2, e2));
    o[15] = sqrtf(dot(e2 - e1, e2 - e1));
    o[16] = rmax(rmax(fabsf(y0.x), rmax(fabsf(y0.y), fabsf(y0.z))),
                 rmax(rmax(fabsf(y1.x), rmax(fabsf(y1.y), fabsf(y1.z))), rmax(fabsf(y2.x), rmax(fabsf(y2.y), fabsf(y2.z)))));
    const float a = dot(e1, e1), bb = dot(e1, e2), c = dot(e2, e2);
    o[17] = a; o[18] = bb; o[19] = c;
    o[20] = a * c - bb * bb;
    o[21] = 0.0f; o[22] = 0.0f; o[23] = 0.0f;
}

// FP32 pre-filter of a face item in its environment's frame (coordinates
// relative to the grid origin: master vertices rounded once from FP64, the
// sample interpolated in FP32 from rounded slave vertices): true only when
// the exact FP64 test (face_geom<double> with g < eps <= eps_max) certainly
// fails.  A master coordinate is within 2^-24 of its magnitude of the exact
// value and a sample coordinate within 2^-22 max|v|, so the differences
// below carry at most del = 2^-21 max|v|.  From there (first order, then
// widened):
//   N = e1 x e2 is within rel_N |N| of the exact normal, rel_N = 8 del
//   (l1 + l2) / |N| + 1e-5;
//   a cast with N.n_s >= (rel_N + 1e-3) |N| certainly faces away; one with
//   N.n_s > -(rel_N + 0.05) |N| is left to the later tests;
//   the gap g = N.d / N.n_s is within tol_g = (2 rel_N (|d| + |g|) + 8 del)
//   / cos + 1e-4 (|d| + |g|), cos = -N.n_s / |N|;
//   the hit point's barycentric coordinates are within tol_b = 0.02 +
//   4 (tol_g + 4 del) / h_min, h_min the triangle's smallest height.
// the per-sample part of the face pre-filter, given the master triangle's
// part: y0, its edges e1, e2, N = e1 x e2 and |N|, the edge lengths, the
// largest coordinate magnitude Rm of its vertices and the Gram terms a =
// e1.e1, bb = e1.e2, c = e2.e2, det = a c - bb^2.  Quotients by fast division
// and |d| by the reciprocal square root: their few-ulp errors are far inside
// the test's tolerances (1e-4 relative in g, 2^-21 R per coordinate, 0.02
// in the barycentrics), so a rejection stays certain.
__device__ __forceinline__ bool face_reject_core(V3<float> xs, V3<float> ns, V3<float> y0, V3<float> e1,
                                                 V3<float> e2, V3<float> N, float nN, float l1, float l2, float l3,
                                                 float Rm, float a, float bb, float c, float det, float eps_max) {
    const float R = rmax(rmax(fabsf(xs.x), rmax(fabsf(xs.y), fabsf(xs.z))), Rm);
    const float del = 4.7683716e-7f * R;   // 2^-21 R
    if (!(nN > 0.0f)) return false;
    const float inv_nN = __fdividef(1.0f, nN);
    const float rel_N = 8.0f * del * (l1 + l2) * inv_nN + 1e-5f;
    const float den = dot(N, ns);
    if (den >= (rel_N + 1e-3f) * nN) return true;           // faces away
    if (den > -(rel_N + 0.05f) * nN) return false;           // near grazing: later tests decide
    const float cosn = -den * inv_nN;
    const V3<float> d = y0 - xs;
    const float g = __fdividef(dot(N, d), den);
    const float dd = dot(d, d);
    const float dn = dd > 0.0f ? dd * rsqrtf(dd) : 0.0f;
    const float tol_g = __fdividef(2.0f * rel_N * (dn + fabsf(g)) + 8.0f * del, cosn) + 1e-4f * (dn + fabsf(g));
    if (g > eps_max * (1.0f + 1e-6f) + tol_g || g < -tol_g) return true;
    const V3<float> q = g * ns - d;    // hit point relative to y0
    const float r1 = dot(q, e1), r2 = dot(q, e2);
    const float inv_det = __fdividef(1.0f, det);
    const float v = (c * r1 - bb * r2) * inv_det, w = (a * r2 - bb * r1) * inv_det;
    const float hmin = nN * __fdividef(1.0f, rmax(l1, rmax(l2, l3)));
    const float tol_b = 0.02f + 4.0f * (tol_g + 4.0f * del) * __fdividef(1.0f, hmin);
    return rmin(1.0f - v - w, rmin(v, w)) < -tol_b;
}
__device__ __forceinline__ bool face_reject_f32(V3<float> xs, V3<float> ns, V3<float> y0, V3<float> y1, V3<float> y2,
                                                float eps_max) {
    const float Rm = rmax(rmax(fabsf(y0.x), rmax(fabsf(y0.y), fabsf(y0.z))),
                          rmax(rmax(fabsf(y1.x), rmax(fabsf(y1.y), fabsf(y1.z))),
                               rmax(fabsf(y2.x), rmax(fabsf(y2.y), fabsf(y2.z)))));
    const V3<float> e1 = y1 - y0, e2 = y2 - y0, N = cross(e1, e2);
    const float nN = sqrtf(dot(N, N));
    const float l1 = sqrtf(dot(e1, e1)), l2 = sqrtf(dot(e2, e2)), l3 = sqrtf(dot(e2 - e1, e2 - e1));
    const float a = dot(e1, e1), bb = dot(e1, e2), c = dot(e2, e2);
    return face_reject_core(xs, ns, y0, e1, e2, N, nN, l1, l2, l3, Rm, a, bb, c, a * c - bb * bb, eps_max);
}

// the same test with the master triangle's part read from its k_mtri_pre
// record: the same operations on the same values, so the same decisions
__device__ __forceinline__ bool face_reject_f32_rec(V3<float> xs, V3<float> ns, const float* rec, float eps_max) {
    const float4* r4 = reinterpret_cast<const float4*>(rec);
    const float4 q0 = r4[0], q1 = r4[1], q2 = r4[2], q3 = r4[3], q4 = r4[4], q5 = r4[5];
    const V3<float> y0 = {q0.x, q0.y, q0.z}, e1 = {q0.w, q1.x, q1.y}, e2 = {q1.z, q1.w, q2.x};
    const V3<float> N = {q2.y, q2.z, q2.w};
    return face_reject_core(xs, ns, y0, e1, e2, N, q3.x, q3.y, q3.z, q3.w, q4.x, q4.y, q4.z, q4.w, q5.x, eps_max);
}

__global__ void k_fill_owner(CandView C, const int32_t* __restrict__ items, ItemBufs B) {
    pass_dep_wait();
    if ((int64_t)*B.n > B.cap) return;
    const int lane = threadIdx.x & 31;
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    const int n_active = *C.n_active;
    for (int i = warp; i < n_active; i += nwarps) {
        const int off = items[2 * i], n = items[2 * i + 1];
        for (int q = lane; q < n; q += 32) B.owner[off + q] = i;
    }
}

// where item slot s of active triangle i points: kind 0 face (candidate j,
// sample k), 1 edge (candidate j, Gauss point k), 2 point (candidate j)
struct ItemRef { int kind, j, k; };
template <int NK>
__device__ __forceinline__ ItemRef item_ref(const TriData& D, int q) {
    if (q < D.nf * NK) return ItemRef{0, q / NK, q % NK};
    const int r = q - D.nf * NK;
    if (r < 2 * D.ne) return ItemRef{1, r >> 1, r & 1};
    return ItemRef{2, r - 2 * D.ne, 0};
}

template <class T>
__device__ __forceinline__ void item_store(const ItemBufs& B, int64_t s, double e, double amin, T c1, T c2,
                                           const T* b) {
    T* rt = (T*)B.rt;
    B.rd[2 * s] = e;
    B.rd[2 * s + 1] = amin;
    rt[5 * s] = c1; rt[5 * s + 1] = c2;
    rt[5 * s + 2] = b[0]; rt[5 * s + 3] = b[1]; rt[5 * s + 4] = b[2];
}

// FP32 pre-filter of an edge or point item in the environment's frame: true
// only when the exact FP64 test certainly fails.  An edge (a != b) or a
// master vertex (a == b) has no active sample when the plane distances
// n_s . (y - x0) of both ends are certainly above eps_max or below 0
// (plane_gap_maybe's bound plus 8 del for the frame's rounding, del =
// 2^-23 max|v|), or when both ends are certainly outside one edge of the
// slave triangle (bary_f's bound plus 16 del / h for the frame's rounding,
// h the slave triangle's smallest height); for a vertex, when it is
// certainly outside any slave edge.
__device__ __forceinline__ bool edge_reject_f32(V3<float> x0, V3<float> x1, V3<float> x2, V3<float> ns,
                                                V3<float> ya, V3<float> yb, float eps_max) {
    float R = 0.0f;
    for (const V3<float>& v : {x0, x1, x2, ya, yb}) R = rmax(R, rmax(fabsf(v.x), rmax(fabsf(v.y), fabsf(v.z))));
    const float del = 1.1920929e-7f * R;
    const V3<float> da = ya - x0, db = yb - x0;
    if (!plane_gap_maybe(ns, da, db, eps_max, 8.0f * del)) return true;
    const V3<float> e1 = x1 - x0, e2 = x2 - x0;
    float fa[3], fb[3], ta, tb;
    bool oka, okb;
    bary_f(da, e1, e2, fa, ta, oka);
    bary_f(db, e1, e2, fb, tb, okb);
    if (!(oka && okb)) return false;
    const V3<float> N = cross(e1, e2);
    const float l1 = sqrtf(dot(e1, e1)), l2 = sqrtf(dot(e2, e2)), l3 = sqrtf(dot(e2 - e1, e2 - e1));
    const float hmin = sqrtf(dot(N, N)) / rmax(l1, rmax(l2, l3));
    const float slack = 16.0f * del / hmin;
    for (int a = 0; a < 3; ++a)
        if (fa[a] < -(ta + slack) && fb[a] < -(tb + slack)) return true;
    return false;
}

// Phase 1, one thread per item slot: the FP32 pre-filter of the face items
// in the environment's frame (face_reject_f32; no FP64 arithmetic), which
// most face candidates of dense contact fail.  Items that fail it hold no
// record (their mask bit stays clear and they contribute nothing); every
// other item gets its mask bit and is listed for phase 1b.
template <int NK>
__global__ void __launch_bounds__(256)
k_items_pre(SceneView S, Params P, CandView C, const int32_t* __restrict__ items, ItemBufs B,
            int32_t* __restrict__ mid, int32_t* __restrict__ n_mid, int32_t* __restrict__ n_mid2,
            long long* counters, const float* __restrict__ tf32, const float4* __restrict__ ym32,
            const float* __restrict__ mtri_pre) {
    pass_dep_wait();
    const int64_t n = *B.n;
    if (n > B.cap) return;
    long long cnt_eval = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together (mask words and list appends are per warp)
    for (int64_t sb = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); sb < n; sb += stride) {
        const int64_t s = sb + (threadIdx.x & 31);
        bool pass = false, face = false;
        if (s < n) {
            const int i = B.owner[s];
            const int q = (int)(s - items[2 * i]);
            const int64_t t = C.active[i];
            const int nf = min(C.count[4 * t], C.cap_f), ne = min(C.count[4 * t + 1], C.cap_e);
            pass = true;
            const float* tf = tf32 ? tf32 + 64 * (int64_t)i : nullptr;
            if (q < nf * NK) {
                ++cnt_eval;
                face = true;
                if (tf) {
                    const int k = q % NK;
                    const int64_t m = C.face[t * C.cap_f + q / NK];
                    if (mtri_pre) {
                        pass = !face_reject_f32_rec({tf[3 * k], tf[3 * k + 1], tf[3 * k + 2]},
                                                    {tf[48], tf[49], tf[50]}, mtri_pre + kMtriPre * m, (float)P.dhat);
                    } else {
                        const int32_t* M = S.mtri + 3 * m;
                        const float4 a = ym32[M[0]], b = ym32[M[1]], c = ym32[M[2]];
                        pass = !face_reject_f32({tf[3 * k], tf[3 * k + 1], tf[3 * k + 2]}, {tf[48], tf[49], tf[50]},
                                                {a.x, a.y, a.z}, {b.x, b.y, b.z}, {c.x, c.y, c.z}, (float)P.dhat);
                    }
                }
            } else if (tf) {
                // an edge (either Gauss point) or a master vertex
                const int r = q - nf * NK;
                int32_t ia, ib;
                if (r < 2 * ne) {
                    const int32_t me = C.edge[t * C.cap_e + (r >> 1)];
                    ia = S.medge[2 * (int64_t)me]; ib = S.medge[2 * (int64_t)me + 1];
                } else {
                    ia = ib = C.point[t * C.cap_p + (r - 2 * ne)];
                }
                const float4 a = ym32[ia], b = ym32[ib];
                pass = !edge_reject_f32({tf[51], tf[52], tf[53]}, {tf[54], tf[55], tf[56]}, {tf[57], tf[58], tf[59]},
                                        {tf[48], tf[49], tf[50]}, {a.x, a.y, a.z}, {b.x, b.y, b.z}, (float)P.dhat);
            }
        }
        // one mask word per 32 slots (the warp's slots start at a multiple of 32)
        const unsigned word = __ballot_sync(0xffffffffu, pass);
        if ((threadIdx.x & 31) == 0 && sb < n) B.mask[sb >> 5] = word;
        // faces from the front of the list, edges and points from the back
        const int at_f = warp_reserve_c(pass && face, n_mid);
        const int at_o = warp_reserve_c(pass && !face, n_mid2);
        if (pass) mid[face ? (int64_t)at_f : B.cap - 1 - at_o] = (int32_t)s;
    }
    if (counters) {
        for (int o = 16; o > 0; o >>= 1) cnt_eval += shfl_x(cnt_eval, o);
        if ((threadIdx.x & 31) == 0 && cnt_eval) atomic_add_ll(&counters[3], cnt_eval);
    }
}

// Phase 1b, one thread per item past the pre-filter (full warps): the
// local-frame FP32 pre-tests of the mixed path (face_pre, edge_pre,
// point_pre), which reject; then, for the evaluation with a static master,
// the certified FP32 evaluation (face_cert, edge_cert, point_cert), which
// stores the item's record.  Rejected items get an empty record; the others
// are listed for phase 2 (faces from the front of the list, edges and points
// from the back, so that phase 2 runs warps of one kind).  The FP64 path
// lists every item.
// master triangles' edges y1 - y0, y2 - y0 rounded to FP32, once per pass
// (the certified tests read them per item)
__global__ void k_mtri_e32(SceneView S, const double* __restrict__ xm, float* __restrict__ out) {
    pass_dep_wait();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= S.nmt) return;
    const int32_t* M = S.mtri + 3 * m;
    const V3<double> y0 = ld3(xm, M[0]);
    const V3<float> e1 = tof(ld3(xm, M[1]) - y0), e2 = tof(ld3(xm, M[2]) - y0);
    float* o = out + 8 * m;
    o[0] = e1.x; o[1] = e1.y; o[2] = e1.z;
    o[3] = e2.x; o[4] = e2.y; o[5] = e2.z;
    o[6] = 0.0f; o[7] = 0.0f;
}

template <int NK, class T>
__global__ void __launch_bounds__(256)
k_items_mid(SceneView S, Params P, CandView C, const double* __restrict__ x, const double* __restrict__ xm,
            const double* __restrict__ dx, const double* __restrict__ frame, const int32_t* __restrict__ items,
            ItemBufs B, const int32_t* __restrict__ mid, const int32_t* __restrict__ n_mid,
            const int32_t* __restrict__ n_mid2, int32_t* __restrict__ list, int32_t* __restrict__ n_list,
            int32_t* __restrict__ n_list2, long long* counters, bool cert, const double* __restrict__ tmid64,
            const float* __restrict__ tmid32, const float* __restrict__ mtri_e) {
    pass_dep_wait();
    if ((int64_t)*B.n > B.cap) return;
    // faces (the front of the list) first, then edges and points (the back):
    // only the warp at the boundary holds both kinds
    const int nmf = *n_mid;
    const int nm = nmf + *n_mid2;
    const bool pre = P.precision == IPC_PREC_MIXED && tmid64 != nullptr;
    const bool want_dg = dx != nullptr;
    long long cnt_f = 0, cnt_e = 0, cnt_p = 0;
    const int stride = gridDim.x * blockDim.x;
    for (int cb = blockIdx.x * blockDim.x + (threadIdx.x & ~31); cb < nm; cb += stride) {
        const int c = cb + (threadIdx.x & 31);
        const bool faces = c < nmf;
        bool keep = false, face = faces;
        int64_t s = 0;
        if (c < nm) {
            s = faces ? mid[c] : mid[B.cap - 1 - (c - nmf)];
            keep = true;
            if (pre) {
                const int i = B.owner[s];
                const int q = (int)(s - items[2 * i]);
                const TriData D = load_tri_mid(S, C, x, frame, tmid64, tmid32, i);
                const ItemRef R = item_ref<NK>(D, q);
                bool certified = false;
                CertOut o;
                // the certified evaluation first (most items past the pre-filter
                // are active, and it runs in FP32), then the local reject
                // tests for the rest
                if (faces) {
                    const int32_t m = C.face[D.t * C.cap_f + R.j];
                    certified = cert && face_cert_f<NK>(S, P, D, R.k, xm, m, want_dg, o, mtri_e);
                    if (!certified) {
                        FaceSample F;
                        for (int a = 0; a < 3; ++a) F.beta[a] = c_rule[P.L - 1][R.k][a];
                        F.xs = interp(F.beta, D.x0, D.x1, D.x2);
                        F.xs_rel = tof(F.xs - D.x0);
                        const int32_t* M = S.mtri + 3 * (int64_t)m;
                        keep = face_pre(P, D, F, ld3(xm, M[0]), ld3(xm, M[1]), ld3(xm, M[2]));
                    }
                    cnt_f += certified;
                } else if (R.kind == 1) {
                    const int32_t me = C.edge[D.t * C.cap_e + R.j];
                    certified = cert && edge_cert_f(S, P, D, xm, me, R.k, want_dg, o, mtri_e);
                    if (!certified)
                        keep = edge_pre(P, D, ld3(xm, S.medge[2 * (int64_t)me]), ld3(xm, S.medge[2 * (int64_t)me + 1]));
                    cnt_e += certified;
                } else {
                    const int32_t u = C.point[D.t * C.cap_p + R.j];
                    certified = cert && point_cert_f(S, P, D, xm, u, want_dg, o, mtri_e);
                    if (!certified) keep = point_pre(P, D, ld3(xm, u));
                    cnt_p += certified;
                }
                if (certified) {
                    // an active item evaluated from certified FP32 geometry
                    double e, amin;
                    float c1, c2, bf[3];
                    item_value_cert_f(o, want_dg, P, e, amin, c1, c2, bf);
                    const T bt[3] = {(T)bf[0], (T)bf[1], (T)bf[2]};
                    item_store<T>(B, s, e, amin, (T)c1, (T)c2, bt);
                    keep = false;
                } else if (!keep) {
                    const T z[3] = {T(0), T(0), T(0)};
                    item_store<T>(B, s, 0.0, INFINITY, T(0), T(0), z);
                }
            }
        }
        const int at_f = warp_reserve_c(keep && face, n_list);
        const int at_o = warp_reserve_c(keep && !face, n_list2);
        if (keep) list[face ? (int64_t)at_f : B.cap - 1 - at_o] = (int32_t)s;
    }
    if (counters) {
        for (int o = 16; o > 0; o >>= 1) {
            cnt_f += shfl_x(cnt_f, o); cnt_e += shfl_x(cnt_e, o); cnt_p += shfl_x(cnt_p, o);
        }
        if ((threadIdx.x & 31) == 0 && (cnt_f | cnt_e | cnt_p)) {
            atomic_add_ll(&counters[0], cnt_f); atomic_add_ll(&counters[1], cnt_e);
            atomic_add_ll(&counters[2], cnt_p);
        }
    }
}

// Phase 2, one thread per listed item: the exact FP64 geometry and the
// contribution (the arithmetic of sample_add).
template <int NK, class T, int MODE = MODE_EVAL>
__global__ void __launch_bounds__(64, 6)
k_items(SceneView S, Params P, CandView C, const double* __restrict__ x, const double* __restrict__ xm,
        const double* __restrict__ dx, const double* __restrict__ dxm, const double* __restrict__ frame,
        const int32_t* __restrict__ items, ItemBufs B, const int32_t* __restrict__ list,
        const int32_t* __restrict__ n_list, const int32_t* __restrict__ n_list2, long long* counters,
        ModeArgs LG = ModeArgs()) {
    pass_dep_wait();
    if ((int64_t)*B.n > B.cap) return;
    const int nf = *n_list;
    const int n = nf + *n_list2;
    const bool want_dg = dx != nullptr;
    long long cnt_f = 0, cnt_e = 0, cnt_p = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int64_t s = c < nf ? list[c] : list[B.cap - 1 - (c - nf)];
        const int i = B.owner[s];
        const int q = (int)(s - items[2 * i]);
        const TriData D = load_tri(S, C, x, dx, frame, i);
        const ItemRef R = item_ref<NK>(D, q);
        ItemOut o;
        bool on;
        if (R.kind == 0) {
            const FaceSample F = face_sample(P, D, R.k, want_dg);
            on = face_item<NK>(S, P, D, F, xm, dxm, C.face[D.t * C.cap_f + R.j], false, want_dg, o);
            cnt_f += on;
        } else if (R.kind == 1) {
            on = edge_item(S, P, D, xm, dxm, C.edge[D.t * C.cap_e + R.j], R.k, false, want_dg, o);
            cnt_e += on;
        } else {
            on = point_item(S, P, D, xm, dxm, C.point[D.t * C.cap_p + R.j], false, want_dg, o);
            cnt_p += on;
        }
        if (MODE == MODE_MASTER_HESS) {
            if (on) master_blocks(LG, o, S.stri + 3 * D.t, D.ns);
            continue;
        }
        double e = 0.0, amin = INFINITY;
        T c1 = T(0), c2 = T(0), b[3] = {T(0), T(0), T(0)};
        if (on) item_value<T>(o, want_dg, e, amin, c1, c2, b);
        item_store<T>(B, s, e, amin, c1, c2, b);
    }
    if (counters) {
        for (int o = 16; o > 0; o >>= 1) {
            cnt_f += shfl_x(cnt_f, o); cnt_e += shfl_x(cnt_e, o); cnt_p += shfl_x(cnt_p, o);
        }
        if ((threadIdx.x & 31) == 0 && (cnt_f | cnt_e | cnt_p)) {
            atomic_add_ll(&counters[0], cnt_f); atomic_add_ll(&counters[1], cnt_e);
            atomic_add_ll(&counters[2], cnt_p);
        }
    }
}

template <int NK, class T>
__global__ void __launch_bounds__(256)
k_tri_reduce(CandView C, const double* __restrict__ frame, const int32_t* __restrict__ items, ItemBufs B,
             double* __restrict__ triE, T* __restrict__ triG, T* __restrict__ triS, T* __restrict__ triN,
             unsigned long long* alpha_bits) {
    pass_dep_wait();
    if ((int64_t)*B.n > B.cap) return;
    const int lane = threadIdx.x & 31;
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    const int n_active = *C.n_active;
    const T* rt = (const T*)B.rt;
    for (int i = warp; i < n_active; i += nwarps) {
        const int64_t t = C.active[i];
        const int32_t* cnt = C.count + 4 * t;
        const int nf = min(cnt[0], C.cap_f), ne = min(cnt[1], C.cap_e), np = min(cnt[2], C.cap_p);
        const int64_t off = items[2 * i];
        Acc<T> A;
        A.zero();
        auto take = [&](int64_t s) {
            if (!((B.mask[s >> 5] >> (s & 31)) & 1u)) return;   // contributes nothing
            const T b[3] = {rt[5 * s + 2], rt[5 * s + 3], rt[5 * s + 4]};
            A.add(B.rd[2 * s], rt[5 * s], rt[5 * s + 1], b);
            A.amin = rmin(A.amin, B.rd[2 * s + 1]);
        };
        for (int it = lane; it < nf * NK; it += 32) take(off + it);
        for (int it = lane; it < ne * 2; it += 32) take(off + nf * NK + it);
        for (int it = lane; it < np; it += 32) take(off + nf * NK + 2 * ne + it);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            A.E += shfl_x(A.E, o);
#pragma unroll
            for (int q = 0; q < 3; ++q) A.G[q] += shfl_x(A.G[q], o);
#pragma unroll
            for (int q = 0; q < 6; ++q) A.S[q] += shfl_x(A.S[q], o);
            A.amin = rmin(A.amin, shfl_x(A.amin, o));
        }
        if (lane == 0) {
            const double* fr = frame + 8 * (int64_t)i;
            triE[t] = A.E;
            for (int q = 0; q < 3; ++q) triG[3 * t + q] = A.G[q];
            for (int q = 0; q < 6; ++q) triS[6 * t + q] = A.S[q];
            triN[3 * t + 0] = (T)fr[0]; triN[3 * t + 1] = (T)fr[1]; triN[3 * t + 2] = (T)fr[2];
            if (alpha_bits && A.amin < INFINITY)
                atomicMin(alpha_bits, (unsigned long long)__double_as_longlong(A.amin));
        }
    }
}

// ---------------------------------------------------------------------------
// deterministic gathers
// ---------------------------------------------------------------------------
template <class T, class TO>
__global__ void k_gather_grad(const int32_t* __restrict__ off, const int32_t* __restrict__ ent,
                              const T* __restrict__ triG, const T* __restrict__ triN,
                              const int32_t* __restrict__ tri_stamp, const int32_t* __restrict__ misc,
                              const int32_t* __restrict__ v_list, TO* __restrict__ out) {
    pass_dep_wait();
    const int n = misc[kSlotVCount];
    const int32_t ps = misc[kSlotPass];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t v = v_list[i];
        T g0 = T(0), g1 = T(0), g2 = T(0);
        for (int k = off[v]; k < off[v + 1]; ++k) {
            const int e = ent[k];
            const int64_t t = e >> 2;
            if (tri_stamp[t] != ps) continue;
            const int a = e & 3;
            const T c = triG[3 * t + a];
            g0 -= c * triN[3 * t]; g1 -= c * triN[3 * t + 1]; g2 -= c * triN[3 * t + 2];
        }
        out[3 * v] = (TO)g0; out[3 * v + 1] = (TO)g1; out[3 * v + 2] = (TO)g2;
    }
}

__device__ __forceinline__ int sym_idx(int a, int b) {
    // 00 01 02 11 12 22
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

template <class T>
__global__ void k_gather_hess(const int32_t* __restrict__ off, const int32_t* __restrict__ ent,
                              const T* __restrict__ triS, const T* __restrict__ triN,
                              const int32_t* __restrict__ tri_stamp, const int32_t* __restrict__ misc,
                              int32_t* const* __restrict__ b_list, const int32_t* __restrict__ b_stamp,
                              T* __restrict__ out) {
    pass_dep_wait();
    const int32_t ps = misc[kSlotPass], hs = misc[kSlotHPass];
    const int n_cur = misc[kSlotBCount + (hs & 1)], n_prev = misc[kSlotBCount + ((hs + 1) & 1)];
    const int32_t* cur = b_list[hs & 1];
    const int32_t* prev = b_list[(hs + 1) & 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cur + n_prev; i += gridDim.x * blockDim.x) {
        if (i >= n_cur) {
            // listed by the previous Hessian pass: clear it unless this pass listed it too
            const int64_t b = prev[i - n_cur];
            if (b_stamp[b] != hs)
                for (int q = 0; q < 9; ++q) out[9 * b + q] = T(0);
            continue;
        }
        const int64_t b = cur[i];
        T h[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) h[q] = T(0);
        for (int k = off[b]; k < off[b + 1]; ++k) {
            const int e = ent[k];
            const int64_t t = e >> 4;
            if (tri_stamp[t] != ps) continue;
            const int a = (e >> 2) & 3, c = e & 3;
            const T sv = triS[6 * t + sym_idx(a, c)];
            const T nn[3] = {triN[3 * t], triN[3 * t + 1], triN[3 * t + 2]};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) h[3 * p + q] += sv * nn[p] * nn[q];
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) out[9 * b + q] = h[q];
    }
}

// two-pass fixed-order sum of n doubles
constexpr int kRedThreads = 256;
constexpr int kRedPer = 8;
// (with stamp: only the entries whose stamp equals *pass count)
__global__ void k_reduce_partial(const double* __restrict__ in, int64_t n, double* __restrict__ part,
                                 const int32_t* __restrict__ stamp, const int32_t* __restrict__ pass) {
    pass_dep_wait();
    __shared__ double sh[kRedThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kRedThreads * kRedPer;
    const int32_t ps = pass ? *pass : 0;
    double s = 0.0;
    for (int i = 0; i < kRedPer; ++i) {
        const int64_t k = base + (int64_t)i * kRedThreads + threadIdx.x;
        if (k < n && (!stamp || stamp[k] == ps)) s += in[k];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}
__global__ void k_reduce_final(const double* __restrict__ part, int64_t n, double* __restrict__ out) {
    pass_dep_wait();
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += 1024) s += part[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = sh[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *out = v;
    }
}

}  // namespace

// the master's FP32 tables of the mixed path (vertices in the environment's
// frame, triangle edges, the face pre-filter's per-triangle part), from xm,
// on stream s
cudaError_t master_tables(Ctx& c, const double* xm, cudaStream_t s) {
    GMCP_CUDA_TRY(c.ym32.ensure(4 * (size_t)c.nmv + 4));
    if (c.use_mtri_e32) GMCP_CUDA_TRY(c.mtri_e32.ensure(8 * (size_t)c.nmt + 8));
    if (c.use_mtri_pre) GMCP_CUDA_TRY(c.mtri_pre.ensure((size_t)kMtriPre * c.nmt + kMtriPre));
    if (c.nmv == 0) return cudaSuccess;
    launch_dep(k_master_f32, (unsigned)((c.nmv + 255) / 256), 256, 0, s, c.view(), xm, (float4*)c.ym32.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    if (c.nmt == 0) return cudaSuccess;
    if (c.use_mtri_e32) {
        launch_dep(k_mtri_e32, (unsigned)((c.nmt + 255) / 256), 256, 0, s, c.view(), xm, c.mtri_e32.p);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    // the face pre-filter's per-triangle table pays only when most master
    // triangles take many face items (see Ctx::use_mtri_pre)
    if (!c.use_mtri_pre) return cudaSuccess;
    launch_dep(k_mtri_pre, (unsigned)((c.nmt + 255) / 256), 256, 0, s, c.view(), (const float4*)c.ym32.p, c.mtri_pre.p);
    return cudaGetLastError();
}

namespace {

template <int NK, class T, int MODE>
cudaError_t launch_samples(Ctx& c, const double* x, const double* xm, T* G, T* Sm, T* N,
                           long long* counters, const double* dx, const double* dxm,
                           unsigned long long* alpha_bits, ModeArgs LG = ModeArgs()) {
    const int threads = 256;
    const int sms = sm_count(c.device);
    const int blocks = sms * c.tune_samples_bpsm;
    // the warp-per-triangle kernel, instantiated for the face rule in use
    auto launch_k_samples = [&](auto... a) {
        if (c.P.face_clip) launch_dep(k_samples<NK, T, MODE, true>, blocks, threads, 0, c.stream, a...);
        else launch_dep(k_samples<NK, T, MODE, false>, blocks, threads, 0, c.stream, a...);
    };
    GMCP_CUDA_TRY(c.tri_frame.ensure(8 * (size_t)c.ns + 8));
    constexpr bool kMaster = MODE == MODE_MASTER_HESS;
    if (MODE != MODE_EVAL && !kMaster) {
        launch_dep(k_tri_frame, sms * 4, 256, 0, c.stream, c.view(), c.cand(), x, c.tri_frame.p, NK, nullptr, nullptr,
                   nullptr, nullptr, nullptr, 1, nullptr, nullptr, nullptr);
        GMCP_CUDA_TRY(cudaGetLastError());
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + 4, 0, sizeof(int32_t), c.stream));
        launch_k_samples(
            c.view(), c.P, c.cand(), x, xm, c.tri_E.p, G, Sm, N, counters, dx, dxm, alpha_bits, LG,
            c.tri_frame.p, nullptr, 0);
        return cudaGetLastError();
    }
    if (MODE == MODE_EVAL && c.P.face_clip) {
        // clipped-overlap face samples: a variable number per pair, evaluated
        // by the warp-per-triangle kernel (the items' fixed slots do not apply)
        launch_dep(k_tri_frame, sms * 4, 256, 0, c.stream, c.view(), c.cand(), x, c.tri_frame.p, NK, nullptr, nullptr,
                   c.tri_stamp.p, c.misc_i32.p, nullptr, 1, nullptr, nullptr, nullptr);
        GMCP_CUDA_TRY(cudaGetLastError());
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + 4, 0, sizeof(int32_t), c.stream));
        launch_k_samples(
            c.view(), c.P, c.cand(), x, xm, c.tri_E.p, G, Sm, N, counters, dx, dxm, alpha_bits, LG,
            c.tri_frame.p, nullptr, 0);
        return cudaGetLastError();
    }
    // contact evaluation: one thread per sample item, and the warp-per-
    // triangle kernel only when the items do not fit the buffer (the
    // count is known on the device alone; the caller grows the buffer)
    if (c.cap_items == 0) c.cap_items = std::max<int64_t>((int64_t)1 << 20, c.ns);
    GMCP_CUDA_TRY(c.tri_items.ensure(2 * (size_t)c.ns + 2));
    GMCP_CUDA_TRY(c.item_owner.ensure((size_t)c.cap_items));
    GMCP_CUDA_TRY(c.item_rd.ensure(2 * (size_t)c.cap_items));
    GMCP_CUDA_TRY(c.item_rt.ensure(5 * sizeof(T) * (size_t)c.cap_items));
    GMCP_CUDA_TRY(c.item_list.ensure((size_t)c.cap_items));
    GMCP_CUDA_TRY(c.item_mask.ensure((size_t)c.cap_items / 32 + 2));
    GMCP_CUDA_TRY(c.item_mid.ensure((size_t)c.cap_items));
    int32_t* n_items = c.misc_i32.p + 16;
    GMCP_CUDA_TRY(cudaMemsetAsync(n_items, 0, sizeof(int32_t), c.stream));
    if (kMaster) {
        // outside a contact pass: fresh item lists, and no pass stamps
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + kSlotItemList, 0, sizeof(int32_t), c.stream));
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + kSlotItemList2, 0, sizeof(int32_t), c.stream));
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + kSlotItemMid, 0, 2 * sizeof(int32_t), c.stream));
    }
    // the FP32 face pre-filter's inputs (mixed path): samples per active
    // triangle and master vertices, both in the environment's frame
    const bool f32pre = c.P.precision == IPC_PREC_MIXED && c.nmv > 0;
    if (f32pre) {
        GMCP_CUDA_TRY(c.tri_f32.ensure(64 * (size_t)c.ns + 64));
        GMCP_CUDA_TRY(c.ym32.ensure(4 * (size_t)c.nmv + 4));
        GMCP_CUDA_TRY(c.tri_mid64.ensure(4 * (size_t)c.ns + 8));
        GMCP_CUDA_TRY(c.tri_mid32.ensure(16 * (size_t)c.ns + 16));
        if (c.use_mtri_e32) GMCP_CUDA_TRY(c.mtri_e32.ensure(8 * (size_t)c.nmt + 8));
        if (c.use_mtri_pre) GMCP_CUDA_TRY(c.mtri_pre.ensure((size_t)kMtriPre * c.nmt + kMtriPre));
        // the master's FP32 tables depend on xm alone: already enqueued at
        // the start of a contact pass (c.master_pre), else beside the frame
        // kernel on the side stream when the pass has forked one
        if (!c.master_pre) {
            cudaStream_t ms = c.side_master ? c.aux_stream : c.stream;
            GMCP_CUDA_TRY(master_tables(c, xm, ms));
            if (c.side_master) GMCP_CUDA_TRY(cudaEventRecord(c.ev_master, c.aux_stream));
        }
    }
    // certified FP32 items: mixed path, evaluation, static master (the
    // middle stage then reads dx's products with the normals from the frame
    // kernel's table)
    const bool cert = !kMaster && c.P.precision == IPC_PREC_MIXED && dxm == nullptr;
    launch_dep(k_tri_frame, sms * 4, 256, 0, c.stream, c.view(), c.cand(), x, c.tri_frame.p, NK, c.tri_items.p, n_items,
                                               kMaster ? nullptr : c.tri_stamp.p, c.misc_i32.p,
                                               f32pre ? c.tri_f32.p : nullptr, c.P.L, cert ? dx : nullptr,
                                               f32pre ? c.tri_mid64.p : nullptr, f32pre ? c.tri_mid32.p : nullptr);
    GMCP_CUDA_TRY(cudaGetLastError());
    ItemBufs B{c.item_owner.p, c.item_rd.p, (void*)c.item_rt.p, n_items, c.cap_items, c.item_mask.p};
    launch_dep(k_fill_owner, sms * 8, 256, 0, c.stream, c.cand(), c.tri_items.p, B);
    GMCP_CUDA_TRY(cudaGetLastError());
    if (f32pre && (c.side_master || c.master_pre)) GMCP_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.ev_master, 0));
    int32_t* n_list = c.misc_i32.p + kSlotItemList;
    int32_t* n_list2 = c.misc_i32.p + kSlotItemList2;
    int32_t* n_mid = c.misc_i32.p + kSlotItemMid;
    int32_t* n_mid2 = c.misc_i32.p + kSlotItemMid2;
    launch_dep(k_items_pre<NK>, sms * 16, 256, 0, c.stream, c.view(), c.P, c.cand(), c.tri_items.p, B, c.item_mid.p, n_mid,
                                                    n_mid2, counters, f32pre ? c.tri_f32.p : nullptr,
                                                    f32pre ? (const float4*)c.ym32.p : nullptr,
                                                    f32pre && c.use_mtri_pre ? c.mtri_pre.p : nullptr);
    GMCP_CUDA_TRY(cudaGetLastError());
    launch_dep(k_items_mid<NK, T>, sms * 8, 256, 0, c.stream, c.view(), c.P, c.cand(), x, xm, dx, c.tri_frame.p,
                                                      c.tri_items.p, B, c.item_mid.p, n_mid, n_mid2, c.item_list.p,
                                                      n_list, n_list2, counters, cert,
                                                      f32pre ? c.tri_mid64.p : nullptr,
                                                      f32pre ? c.tri_mid32.p : nullptr,
                                                      f32pre && c.use_mtri_e32 ? c.mtri_e32.p : nullptr);
    GMCP_CUDA_TRY(cudaGetLastError());
    if (kMaster) {
        launch_dep(k_items<NK, T, MODE>, sms * 64, 64, 0, c.stream, c.view(), c.P, c.cand(), x, xm, dx, dxm, c.tri_frame.p,
                                                             c.tri_items.p, B, c.item_list.p, n_list, n_list2,
                                                             counters, LG);
        GMCP_CUDA_TRY(cudaGetLastError());
        // oversized item sets: the warp-per-triangle kernel instead
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + 4, 0, sizeof(int32_t), c.stream));
        launch_k_samples(
            c.view(), c.P, c.cand(), x, xm, c.tri_E.p, G, Sm, N, counters, dx, dxm, alpha_bits, LG,
            c.tri_frame.p, n_items, c.cap_items);
        return cudaGetLastError();
    }
    {
        ProfScope pi(c.prof, c.stream, "items");
        // 64-thread blocks, at most 168 registers a thread: 12 warps fit an
        // SM (8 with 256-thread blocks)
        launch_dep(k_items<NK, T>, sms * 64, 64, 0, c.stream, c.view(), c.P, c.cand(), x, xm, dx, dxm, c.tri_frame.p,
                   c.tri_items.p, B, c.item_list.p, n_list, n_list2, counters, ModeArgs());
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    launch_dep(k_tri_reduce<NK, T>, sms * 8, 256, 0, c.stream, c.cand(), c.tri_frame.p, c.tri_items.p, B, c.tri_E.p,
                                                        G, Sm, N, alpha_bits);
    GMCP_CUDA_TRY(cudaGetLastError());
    GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + 4, 0, sizeof(int32_t), c.stream));
    launch_k_samples(
        c.view(), c.P, c.cand(), x, xm, c.tri_E.p, G, Sm, N, counters, dx, dxm, alpha_bits, LG,
        c.tri_frame.p, n_items, c.cap_items);
    return cudaGetLastError();
}

}  // namespace

cudaError_t contact_init_constants(const double* rule_l1l2) {
    float rf[2 * 16 * 3];
    for (int q = 0; q < 2 * 16 * 3; ++q) rf[q] = (float)rule_l1l2[q];
    GMCP_CUDA_TRY(cudaMemcpyToSymbol(c_rule_f, rf, sizeof(rf)));
    return cudaMemcpyToSymbol(c_rule, rule_l1l2, sizeof(double) * 2 * 16 * 3);
}

int sm_count(int device) {
    static int cached[64] = {0};
    if (device >= 0 && device < 64 && cached[device]) return cached[device];
    int n = 148;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
    if (device >= 0 && device < 64) cached[device] = n;
    return n;
}

cudaError_t reduce_sum(Ctx& c, const double* in, int64_t n, double* out, const int32_t* stamp,
                       const int32_t* pass) {
    const int64_t per = (int64_t)kRedThreads * kRedPer;
    const int64_t nb = (n + per - 1) / per;
    GMCP_CUDA_TRY(c.red_tmp.ensure((size_t)nb + 2));
    if (nb > 0) {
        launch_dep(k_reduce_partial, (unsigned)nb, kRedThreads, 0, c.stream, in, n, c.red_tmp.p, stamp, pass);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    launch_dep(k_reduce_final, 1, 1024, 0, c.stream, c.red_tmp.p, nb, out);
    return cudaGetLastError();
}

cudaError_t contact_eval(Ctx& c, const double* x, const double* xm, double* energy_dev,
                         void* grad_dev, bool want_hess, long long* counters, const double* dx,
                         const double* dxm, unsigned long long* alpha_bits) {
    const bool f32 = c.P.precision == IPC_PREC_MIXED;
    const bool grad = grad_dev != nullptr, hess = want_hess && c.cb_nnzb > 0;
    const int sms = sm_count(c.device);
    const unsigned flat = (unsigned)(sms * 8);
    int32_t* misc = c.misc_i32.p;
    launch_dep(k_pass_begin, 1, 1, 0, c.stream, misc, hess ? 1 : 0);
    GMCP_CUDA_TRY(cudaGetLastError());
    // The touched vertices and blocks depend on the active list alone: they
    // are listed on a third stream beside the sample evaluation (the
    // profiler keeps one stream) and joined before the gathers.
    const bool fork = (grad || hess) && !c.prof.on;
    if (grad || hess) {
        const TouchArgs TA{misc, c.v_stamp.p, c.v_list.p, misc + kSlotVCount, c.b_stamp.p,
                           {c.b_list0.p, c.b_list1.p}, misc + kSlotBCount, c.cb_row.p, c.cb_col.p,
                           grad ? 1 : 0, hess ? 1 : 0};
        cudaStream_t ts = c.stream;
        if (fork) {
            if (!c.aux_stream) GMCP_CUDA_TRY(cudaStreamCreateWithFlags(&c.aux_stream, cudaStreamNonBlocking));
            if (!c.ev_touch0) GMCP_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_touch0, cudaEventDisableTiming));
            if (!c.ev_touch1) GMCP_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_touch1, cudaEventDisableTiming));
            if (!c.ev_samples) GMCP_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_samples, cudaEventDisableTiming));
            GMCP_CUDA_TRY(cudaEventRecord(c.ev_touch0, c.stream));
            GMCP_CUDA_TRY(cudaStreamWaitEvent(c.aux_stream, c.ev_touch0, 0));
            ts = c.aux_stream;
        }
        launch_dep(k_touch, flat, 256, 0, ts, c.view(), c.cand(), TA);
        GMCP_CUDA_TRY(cudaGetLastError());
        if (fork) GMCP_CUDA_TRY(cudaEventRecord(c.ev_touch1, c.aux_stream));
    }
    // the sample stage may put the master's FP32 tables on the side stream
    if (fork && !c.ev_master) GMCP_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_master, cudaEventDisableTiming));
    struct SideFlag { bool& f; SideFlag(bool& r, bool v) : f(r) { f = v; } ~SideFlag() { f = false; } };
    SideFlag side_flag(c.side_master, fork);
    {
        ProfScope ps(c.prof, c.stream, "samples");
        if (f32) {
            if (c.P.nk == 4)
                GMCP_CUDA_TRY((launch_samples<4, float, MODE_EVAL>(c, x, xm, c.tri_G32.p, c.tri_S32.p, c.tri_n32.p, counters, dx, dxm, alpha_bits)));
            else
                GMCP_CUDA_TRY((launch_samples<16, float, MODE_EVAL>(c, x, xm, c.tri_G32.p, c.tri_S32.p, c.tri_n32.p, counters, dx, dxm, alpha_bits)));
        } else {
            if (c.P.nk == 4)
                GMCP_CUDA_TRY((launch_samples<4, double, MODE_EVAL>(c, x, xm, c.tri_G64.p, c.tri_S64.p, c.tri_n64.p, counters, dx, dxm, alpha_bits)));
            else
                GMCP_CUDA_TRY((launch_samples<16, double, MODE_EVAL>(c, x, xm, c.tri_G64.p, c.tri_S64.p, c.tri_n64.p, counters, dx, dxm, alpha_bits)));
        }
    }
    // After the samples: the gradient gather on the main stream, the Hessian
    // gather and the energy sum on the third stream (behind the touch lists),
    // joined at the end.
    cudaStream_t hs_stream = c.stream;
    if (fork) {
        GMCP_CUDA_TRY(cudaEventRecord(c.ev_samples, c.stream));
        GMCP_CUDA_TRY(cudaStreamWaitEvent(c.aux_stream, c.ev_samples, 0));
        GMCP_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.ev_touch1, 0));
        hs_stream = c.aux_stream;
    }
    if (grad) {
        ProfScope ps(c.prof, c.stream, "gather_grad");
        GMCP_CUDA_TRY(cudaMemsetAsync(grad_dev, 0, (f32 ? sizeof(float) : sizeof(double)) * 3 * (size_t)c.nv,
                                      c.stream));
        if (f32)
            launch_dep(k_gather_grad<float, float>, flat, 256, 0, c.stream, c.vt_off.p, c.vt_ent.p, c.tri_G32.p, c.tri_n32.p,
                                                                 c.tri_stamp.p, misc, c.v_list.p, (float*)grad_dev);
        else
            launch_dep(k_gather_grad<double, double>, flat, 256, 0, c.stream, c.vt_off.p, c.vt_ent.p, c.tri_G64.p,
                                                                   c.tri_n64.p, c.tri_stamp.p, misc, c.v_list.p,
                                                                   (double*)grad_dev);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    if (hess) {
        ProfScope ps(c.prof, hs_stream, "gather_hess");
        int32_t* const* lists = c.b_lists.p;
        if (f32)
            launch_dep(k_gather_hess<float>, flat, 256, 0, hs_stream, c.cb_src_off.p, c.cb_src.p, c.tri_S32.p, c.tri_n32.p,
                                                              c.tri_stamp.p, misc, lists, c.b_stamp.p, c.cb_val32.p);
        else
            launch_dep(k_gather_hess<double>, flat, 256, 0, hs_stream, c.cb_src_off.p, c.cb_src.p, c.tri_S64.p, c.tri_n64.p,
                                                               c.tri_stamp.p, misc, lists, c.b_stamp.p, c.cb_val64.p);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    if (energy_dev) {
        ProfScope ps(c.prof, hs_stream, "reduce");
        cudaStream_t main = c.stream;
        c.stream = hs_stream;
        const cudaError_t e = reduce_sum(c, c.tri_E.p, c.ns, energy_dev, c.tri_stamp.p, misc + kSlotPass);
        c.stream = main;
        GMCP_CUDA_TRY(e);
    }
    if (fork) {
        GMCP_CUDA_TRY(cudaEventRecord(c.ev_touch1, c.aux_stream));
        GMCP_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.ev_touch1, 0));
    }
    return cudaSuccess;
}

cudaError_t contact_alpha_lin(Ctx& c, const double* x, const double* xm, const double* dx,
                              const double* dxm, unsigned long long* alpha_bits, int alpha_stride) {
    ProfScope ps(c.prof, c.stream, "alpha_lin");
    ModeArgs LG;
    LG.alpha_stride = alpha_stride;
    // the step bound always uses FP64 geometry
    if (c.P.nk == 4)
        return launch_samples<4, double, MODE_ALPHA>(c, x, xm, nullptr, nullptr, nullptr, nullptr, dx, dxm,
                                                     alpha_bits, LG);
    return launch_samples<16, double, MODE_ALPHA>(c, x, xm, nullptr, nullptr, nullptr, nullptr, dx, dxm,
                                                  alpha_bits, LG);
}

cudaError_t contact_master_hess(Ctx& c, const double* x, const double* xm, int32_t* ij, double* blk,
                                int64_t cap, unsigned long long* count, bool rows, bool blocks) {
    ProfScope ps(c.prof, c.stream, "master_hess");
    GMCP_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned long long), c.stream));
    ModeArgs LG;
    LG.h_ij = ij; LG.h_blk = blk; LG.h_count = count; LG.h_cap = cap; LG.m_off = (int32_t)c.nv;
    LG.h_rows = rows; LG.h_blocks = blocks;
    if (c.P.nk == 4)
        return launch_samples<4, double, MODE_MASTER_HESS>(c, x, xm, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                            nullptr, nullptr, LG);
    return launch_samples<16, double, MODE_MASTER_HESS>(c, x, xm, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                         nullptr, nullptr, LG);
}

cudaError_t contact_lagged(Ctx& c, const double* x, const double* xm, const double* p,
                           const double* alphas_dev, int na, double* triE8, double* energies_dev,
                           int alphas_stride, const double* pm) {
    ProfScope ps(c.prof, c.stream, "lagged");
    if (na < 1 || na > 8) return cudaErrorInvalidValue;
    GMCP_CUDA_TRY(cudaMemsetAsync(triE8, 0, sizeof(double) * (size_t)na * (size_t)c.ns, c.stream));
    ModeArgs LG;
    LG.alphas = alphas_dev; LG.na = na; LG.triE8 = triE8; LG.ns = c.ns; LG.alphas_stride = alphas_stride;
    if (c.P.nk == 4)
        GMCP_CUDA_TRY((launch_samples<4, double, MODE_LAGGED>(c, x, xm, nullptr, nullptr, nullptr, nullptr, p, pm, nullptr, LG)));
    else
        GMCP_CUDA_TRY((launch_samples<16, double, MODE_LAGGED>(c, x, xm, nullptr, nullptr, nullptr, nullptr, p, pm, nullptr, LG)));
    if (energies_dev)
        for (int j = 0; j < na; ++j) GMCP_CUDA_TRY(reduce_sum(c, triE8 + (int64_t)j * c.ns, c.ns, energies_dev + j));
    return cudaSuccess;
}

}  // namespace gmcp

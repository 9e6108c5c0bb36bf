// broadphase.cu -- spatial-hash broad phase and additive CCD (FP64).
//
// Compiled with -fmad=false: every product and sum is rounded separately, so
// the candidate predicates (boxes grown by dhat, face-sample positions
// ((b0 x0 + b1 x1) + b2 x2)) and the additive-CCD iteration give the same
// bits as a plain IEEE evaluation in the same order.  That makes candidate
// sets exact and the CCD step reproducible.
//
// Grid: one dense box of cells per environment, sized at context creation
// from the rest geometry; cell coordinates are clamped to the box, which
// keeps the cell map monotone (so overlapping boxes always share a cell).
// Cell ranges are conservative FP32 ranges (see cell_range_f); the exact
// FP64 tests decide every pair.
// Master triangles are counting-sorted into cells (atomic integer counts,
// exclusive scan, atomic integer cursors).  A query visits the cells of its
// box and reports a master triangle only in the first cell common to both
// boxes, so every pair is seen once; per-triangle lists are then sorted,
// which removes any dependence on the order of the cell entries.
//
// Candidate kinds (Sec. 4.1's features, within eps_max = dhat):
//   face  (slave tri, master tri): a face sample of the slave tri lies in the
//         master tri's box grown by dhat
//   edge  (slave tri, master edge): slave vertex box vs edge box grown by dhat
//   point (slave tri, master vertex): slave vertex box vs vertex grown by dhat
// Edges and vertices are found through the master triangle that owns them
// (the lowest-numbered adjacent triangle), whose box contains theirs.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "gmcp_internal.cuh"

namespace gmcp {
namespace {

struct I3 { int x, y, z; };

__device__ __forceinline__ double dmin_(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ double dmax_(double a, double b) { return a > b ? a : b; }

__device__ __forceinline__ int64_t cell_id(const SceneView& S, int e, int ix, int iy, int iz) {
    const int* d = S.grid_dim + 3 * e;
    return S.grid_off[e] + (int64_t)ix + (int64_t)d[0] * ((int64_t)iy + (int64_t)d[1] * iz);
}

// ---------------------------------------------------------------------------
// Conservative cell ranges without the FP64 pipe.
//
// B300 issues FP64 at 1/64 of the FP32 rate, and the per-triangle box and
// cell arithmetic of the filters and the grid build kept that pipe ~75% busy.
// Cell ranges only have to CONTAIN the cells the exact FP64 map gives: a
// wider range visits more cells but changes no result, because the exact
// FP64 box tests decide every pair, and the "first common cell" rule that
// reports a pair once is evaluated on the same (wider) ranges that are
// visited.  So the ranges are computed in FP32 from truncated copies of the
// coordinates, widened by a bound on every rounding involved.
// ---------------------------------------------------------------------------

// v truncated toward zero to FP32 from its bits (integer pipe only):
// |result - v| <= 2^-23 |v| for 2^-126 <= |v| < 2^128; +-0 below that (the
// absolute slack of the cell ranges covers it); +-inf above it; NaN stays NaN.
__device__ __forceinline__ float trunc_f32(double v) {
    const unsigned hi = (unsigned)__double2hiint(v);
    const unsigned lo = (unsigned)__double2loint(v);
    const unsigned sgn = hi & 0x80000000u;
    const unsigned ex = (hi >> 20) & 0x7FFu;
    if (ex < 897u) return __uint_as_float(sgn);
    if (ex > 1150u) {
        const bool nan = ex == 0x7FFu && ((hi & 0xFFFFFu) | lo) != 0u;
        return __uint_as_float(sgn | (nan ? 0x7FC00000u : 0x7F800000u));
    }
    return __uint_as_float(sgn | ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// cell index bounds from an FP32 cell coordinate that already includes its
// slack: NaN and out-of-grid values go to the widest admissible cell
__device__ __forceinline__ int cell_lo_f(float u, int dim) {
    if (!(u >= 0.0f)) return 0;
    if (u >= (float)(dim - 1)) return dim - 1;
    return (int)u;
}
__device__ __forceinline__ int cell_hi_f(float u, int dim) {
    if (!(u < (float)(dim - 1))) return dim - 1;
    if (u < 0.0f) return 0;
    return (int)u;
}

// Cell range of env e that contains the cells (p - org) * inv (real
// arithmetic) of every box whose corners differ from lo/hi (FP32) by at most
// 2^-21 * mag per axis, where mag bounds the sum of the magnitudes of all
// values combined into the box (vertex coordinates, displacements, growth).
// With the FP32 rounding of org, inv, the difference and the product, the
// FP32 cell coordinate is off by at most ~2^-20 (mag + |org|) inv cells; the
// slack is twice that plus 1e-3 cell, which also covers values flushed to
// zero by trunc_f32.  Ranges computed this way for two boxes that overlap
// always share a cell.
__device__ __forceinline__ void cell_range_f(const SceneView& S, int e, const float* lo, const float* hi,
                                             const float* mag, I3& a, I3& b) {
    const float inv = S.grid_inv_f[e];
    int ra[3], rb[3];
    for (int q = 0; q < 3; ++q) {
        const float o = S.grid_org_f[3 * e + q];
        const int dim = S.grid_dim[3 * e + q];
        const float sl = (mag[q] + fabsf(o)) * inv * 2e-6f + 1e-3f;
        ra[q] = cell_lo_f((lo[q] - o) * inv - sl, dim);
        rb[q] = cell_hi_f((hi[q] - o) * inv + sl, dim);
    }
    a = I3{ra[0], ra[1], ra[2]};
    b = I3{rb[0], rb[1], rb[2]};
}

// Exact minimum / maximum of doubles by integer comparison of their ordered
// bit patterns (negative values have their magnitude bits flipped), which
// keeps the FP64 pipe free.  For non-NaN inputs the result is the IEEE
// minimum / maximum, except that -0 orders below +0; no box test can tell
// the two zeros apart.
__device__ __forceinline__ long long ord_key(double v) {
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double kmin3(double a, double b, double c) {
    const long long ka = ord_key(a), kb = ord_key(b), kc = ord_key(c);
    return ka <= kb ? (ka <= kc ? a : c) : (kb <= kc ? b : c);
}
__device__ __forceinline__ double kmax3(double a, double b, double c) {
    const long long ka = ord_key(a), kb = ord_key(b), kc = ord_key(c);
    return ka >= kb ? (ka >= kc ? a : c) : (kb >= kc ? b : c);
}

// Conservative FP32 bounds of a double: lo_f32(v) <= v <= hi_f32(v), within
// ~2^-21 |v| + 1e-30 of v, from trunc_f32 and FP32 arithmetic with directed
// rounding (no FP64 instruction).  Each bound keeps a slack of at least
// ~2^-23 |v| beyond the truncation error, which also covers the FP64
// rounding of a sum of two such values (2^-53 of their magnitudes).
__device__ __forceinline__ float f32_slack(float t) { return __fadd_ru(fabsf(t) * 0x1p-22f, 1e-30f); }
__device__ __forceinline__ float lo_f32(double v) {
    const float t = trunc_f32(v);
    return __fsub_rd(t, f32_slack(t));
}
__device__ __forceinline__ float hi_f32(double v) {
    const float t = trunc_f32(v);
    return __fadd_ru(t, f32_slack(t));
}
// FP32 box test that keeps a pair unless the boxes are certainly apart
// (NaN compares false, so it keeps)
__device__ __forceinline__ bool overlap_keep(const float* alo, const float* ahi, const float* blo,
                                             const float* bhi) {
    return !(alo[0] > bhi[0] || blo[0] > ahi[0] || alo[1] > bhi[1] || blo[1] > ahi[1] ||
             alo[2] > bhi[2] || blo[2] > ahi[2]);
}
// conservative FP32 box of a vertex swept from p to p + d (d may be NULL);
// contains the FP64 box of swept_vert
__device__ __forceinline__ void swept_vert_f(const double* P, const double* D, int64_t v, float* lo,
                                             float* hi) {
    for (int c = 0; c < 3; ++c) {
        const double a = P[3 * v + c];
        float l = lo_f32(a), h = hi_f32(a);
        if (D) {
            const double b = D[3 * v + c];
            l = fminf(l, __fadd_rd(l, lo_f32(b)));
            h = fmaxf(h, __fadd_ru(h, hi_f32(b)));
        }
        lo[c] = l; hi[c] = h;
    }
}

__device__ __forceinline__ void load3(const double* p, int64_t i, double* o) {
    o[0] = p[3 * i]; o[1] = p[3 * i + 1]; o[2] = p[3 * i + 2];
}

// face-rule barycentrics per level (index L-1), filled at context creation
// with the exact quotients (3i+1)/(3n), (3i+2)/(3n) of the fixed rule
__constant__ double c_rule[2][16][3];
// FP32 brackets of the same values: [l][k][0..2] <= c_rule[l][k][0..2] <= [l][k][3..5]
__constant__ float c_rule_f[2][16][6];

// ---------------------------------------------------------------------------
// grid build
// ---------------------------------------------------------------------------
__global__ void k_mtri_box_count(SceneView S, const double* __restrict__ xm,
                                 const double* __restrict__ dxm, float* __restrict__ mboxf,
                                 int4* __restrict__ mcell, int32_t* __restrict__ cnt,
                                 float* __restrict__ mboxf_in) {
    pass_dep_wait();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= S.nmt) return;
    const int32_t* T = S.mtri + 3 * m;
    double lo[3], hi[3];
    float flo[3], fhi[3], mag[3];
    if (dxm) {
        // swept box: the corners p + dp are FP64 sums
        for (int c = 0; c < 3; ++c) { lo[c] = DBL_MAX; hi[c] = -DBL_MAX; }
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) {
                double p = xm[3 * (int64_t)T[a] + c];
                double q = p + dxm[3 * (int64_t)T[a] + c];
                lo[c] = dmin_(lo[c], dmin_(p, q));
                hi[c] = dmax_(hi[c], dmax_(p, q));
            }
    } else {
        double v[3][3];
        for (int a = 0; a < 3; ++a) load3(xm, T[a], v[a]);
        for (int c = 0; c < 3; ++c) {
            lo[c] = kmin3(v[0][c], v[1][c], v[2][c]);
            hi[c] = kmax3(v[0][c], v[1][c], v[2][c]);
        }
    }
    // conservative FP32 bounds of the exact FP64 box (the exact box itself is
    // formed again, from the vertices, for the few pairs the exact tests see)
    for (int c = 0; c < 3; ++c) {
        flo[c] = lo_f32(lo[c]); fhi[c] = hi_f32(hi[c]);
        mag[c] = fabsf(flo[c]) + fabsf(fhi[c]);
        mboxf[6 * m + c] = flo[c]; mboxf[6 * m + 3 + c] = fhi[c];
        // FP32 bounds inside the exact static box (empty for a swept box,
        // which is not the box the exact face test uses)
        mboxf_in[6 * m + c] = dxm ? INFINITY : __double2float_ru(lo[c]);
        mboxf_in[6 * m + 3 + c] = dxm ? -INFINITY : __double2float_rd(hi[c]);
    }
    const int e = S.mtri_env[m];
    I3 a, b;
    cell_range_f(S, e, flo, fhi, mag, a, b);
    mcell[m] = make_int4(a.x, a.y, a.z, e);
    for (int iz = a.z; iz <= b.z; ++iz)
        for (int iy = a.y; iy <= b.y; ++iy)
            for (int ix = a.x; ix <= b.x; ++ix) atomicAdd(&cnt[cell_id(S, e, ix, iy, iz)], 1);
}

// Fill: the same cell range as the count (recomputed from the same FP32
// box), each entry at the next free position of its cell.  cur holds the
// exclusive scan of the counts and is advanced in place, so that afterwards
// cur[c] is the end of cell c; the cell start array is cur shifted by one
// (start[0] = 0, start[c + 1] = cur[c]).
__global__ void k_mtri_fill(SceneView S, const float* __restrict__ mboxf, const int4* __restrict__ mcell,
                            int32_t* __restrict__ cur, int32_t* __restrict__ ent, int64_t cap,
                            int32_t* __restrict__ overflow) {
    pass_dep_wait();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= S.nmt) return;
    const int e = mcell[m].w;
    float flo[3], fhi[3], mag[3];
    for (int c = 0; c < 3; ++c) {
        flo[c] = mboxf[6 * m + c]; fhi[c] = mboxf[6 * m + 3 + c];
        mag[c] = fabsf(flo[c]) + fabsf(fhi[c]);
    }
    I3 a, b;
    cell_range_f(S, e, flo, fhi, mag, a, b);
    for (int iz = a.z; iz <= b.z; ++iz)
        for (int iy = a.y; iy <= b.y; ++iy)
            for (int ix = a.x; ix <= b.x; ++ix) {
                const int pos = atomicAdd(&cur[cell_id(S, e, ix, iy, iz)], 1);
                if (pos < cap) ent[pos] = (int32_t)m;
                else atomicMax(overflow, 1);
            }
}

__device__ __forceinline__ void swept_vert(const double* P, const double* D, int64_t v, double* lo,
                                           double* hi) {
    for (int c = 0; c < 3; ++c) {
        double a = P[3 * v + c];
        double b = D ? a + D[3 * v + c] : a;
        lo[c] = dmin_(a, b); hi[c] = dmax_(a, b);
    }
}
__device__ __forceinline__ void grow_box(double* lo, double* hi, const double* l2, const double* h2) {
    for (int c = 0; c < 3; ++c) { lo[c] = dmin_(lo[c], l2[c]); hi[c] = dmax_(hi[c], h2[c]); }
}
// exact FP64 box of master tri m: of its vertices, or of their motion from
// xm to xm + dxm when dxm is given (the box the grid build bounds in FP32)
__device__ __forceinline__ void exact_mbox(const SceneView& S, const double* xm, const double* dxm,
                                           int64_t m, double* lo, double* hi) {
    const int32_t* T = S.mtri + 3 * m;
    if (dxm) {
        double l2[3], h2[3];
        swept_vert(xm, dxm, T[0], lo, hi);
        swept_vert(xm, dxm, T[1], l2, h2);
        grow_box(lo, hi, l2, h2);
        swept_vert(xm, dxm, T[2], l2, h2);
        grow_box(lo, hi, l2, h2);
    } else {
        double v[3][3];
        for (int a = 0; a < 3; ++a) load3(xm, T[a], v[a]);
        for (int c = 0; c < 3; ++c) {
            lo[c] = kmin3(v[0][c], v[1][c], v[2][c]);
            hi[c] = kmax3(v[0][c], v[1][c], v[2][c]);
        }
    }
}

// insertion sort of a short list held in global memory
__device__ void sort_small(int32_t* a, int n) {
    for (int i = 1; i < n; ++i) {
        int32_t v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
        a[j + 1] = v;
    }
}

// ---------------------------------------------------------------------------
// contact candidate query: one warp per slave triangle
//
// The warp visits the cells of the slave triangle's box; the entries of each
// non-empty cell are spread over the lanes, each lane runs the exact tests
// for its master triangle and the lanes append their hits with a ballot.
// Every list is sorted at the end, so the output does not depend on the
// order in which cells or lanes found the pairs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Slots for the lanes with pred set, reserved by one atomic for the whole
// warp (a counter that every thread bumps serialises at its L2 slice).
// All 32 lanes must call it.
__device__ __forceinline__ int warp_reserve(bool pred, int32_t* counter) {
    const unsigned mask = __ballot_sync(0xffffffffu, pred);
    if (mask == 0u) return 0;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(mask & lanemask_lt());
}

// ascending sort of the first n entries of L by the warp (entries are
// distinct ids).  n <= 32: bitonic network in registers; n <= 128: each
// lane ranks up to four entries against all n and stores them at their
// ranks; longer lists (rare): lane 0 insertion sort.
__device__ void warp_sort(int32_t* L, int n, int lane) {
    if (n <= 1) return;
    if (n <= 32) {
        int32_t v = lane < n ? L[lane] : INT32_MAX;
        for (int k = 2; k <= 32; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                const int32_t o = __shfl_xor_sync(0xffffffffu, v, j);
                const bool up = (lane & k) == 0;
                const bool lower = (lane & j) == 0;
                const int32_t lo = v < o ? v : o, hi = v < o ? o : v;
                v = (lower == up) ? lo : hi;
            }
        if (lane < n) L[lane] = v;
        __syncwarp();
        return;
    }
    __syncwarp();
    if (n <= 128) {
        int32_t v[4];
        int r[4];
        for (int q = 0; q < 4; ++q) {
            const int j = lane + 32 * q;
            v[q] = j < n ? L[j] : 0;
            r[q] = 0;
        }
        for (int i = 0; i < n; ++i) {
            const int32_t w = L[i];
            for (int q = 0; q < 4; ++q) r[q] += w < v[q];
        }
        __syncwarp();
        for (int q = 0; q < 4; ++q)
            if (lane + 32 * q < n) L[r[q]] = v[q];
        __syncwarp();
        return;
    }
    if (lane == 0) sort_small(L, n);
    __syncwarp();
}

// Phase 1 of both queries (one thread per slave triangle): the triangle's
// box (static: vertex box grown by dhat; swept: box of the vertices at x and
// x + dx), its cell range, and whether any of those cells holds a master
// triangle.  Contact mode zeroes every triangle's candidate counts; the
// triangles that reach a non-empty cell are appended, with their boxes and
// cell range, to the list that the later launches work through.
struct QueryList {
    int32_t* n;        // scalar
    int32_t* tri;      // [ns]
    float* boxf;       // [ns][6]: query box lo/hi (conservative FP32: contains the exact grown box)
    float* vboxf;      // [ns][3][6]: conservative FP32 box of each corner (swept: of its motion)
    double* box;       // [ns][6]: exact slave tri box lo/hi (contact query only)
    int32_t* cell;     // [ns][6]: first and last cell (x, y, z)
    int32_t* work;     // work counter of the persistent query (reset before each launch)
};

// Per-vertex conservative FP32 bounds for the query filter, once per slave
// vertex instead of once per triangle corner (a vertex is shared by about
// six triangles).  Contact, [nv][8]: lo_f32 and hi_f32 of the position.
// Swept, [nv][12]: the swept corner box (lo xyz, hi xyz) and the two
// magnitude terms of each axis (position, displacement).  The filter combines
// them in the same order as it would per corner, so its results are
// unchanged.
template <bool SWEPT>
__global__ void k_vert_bounds(int64_t n, const int32_t* __restrict__ svert, const double* __restrict__ x,
                              const double* __restrict__ dx, float* __restrict__ out) {
    pass_dep_wait();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t v = svert[k];
    float pl[3], ph[3];
    for (int c = 0; c < 3; ++c) {
        const double p = x[3 * v + c];
        pl[c] = lo_f32(p);
        ph[c] = hi_f32(p);
    }
    if (!SWEPT) {
        float4* o = reinterpret_cast<float4*>(out + 8 * v);
        o[0] = make_float4(pl[0], pl[1], pl[2], 0.f);
        o[1] = make_float4(ph[0], ph[1], ph[2], 0.f);
        return;
    }
    float l[3], h[3], tx[3], td[3];
    for (int c = 0; c < 3; ++c) {
        const double d = dx[3 * v + c];
        const float dl = lo_f32(d), dh = hi_f32(d);
        tx[c] = fmaxf(fabsf(pl[c]), fabsf(ph[c]));
        td[c] = fmaxf(fabsf(dl), fabsf(dh));
        l[c] = fminf(pl[c], __fadd_rd(pl[c], dl));
        h[c] = fmaxf(ph[c], __fadd_ru(ph[c], dh));
    }
    float4* o = reinterpret_cast<float4*>(out + 12 * v);
    o[0] = make_float4(l[0], l[1], l[2], h[0]);
    o[1] = make_float4(h[1], h[2], tx[0], tx[1]);
    o[2] = make_float4(tx[2], td[0], td[1], td[2]);
}

template <bool SWEPT>
__global__ void __launch_bounds__(256)
k_query_filter(SceneView S, Params P, const double* __restrict__ x, const float* __restrict__ vb_in,
               const int32_t* __restrict__ start, QueryList Q, int32_t* __restrict__ count) {
    pass_dep_wait();
    // every lane runs to the warp-wide append at the end (lanes past the last
    // triangle work on triangle 0 and append nothing)
    const int64_t t_raw = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t_raw < S.ns;
    const int64_t t = valid ? t_raw : 0;
    const int32_t* T = S.stri + 3 * t;
    // The decision (does the grown box reach a non-empty cell?) and the
    // coarse box of the second phase are conservative FP32 bounds; no FP64
    // instruction runs here except the exact slave box of contact survivors.
    // the corners' bounds from the per-vertex pass (k_vert_bounds)
    constexpr int VS = SWEPT ? 12 : 8;
    float r[3][VS];
    for (int a = 0; a < 3; ++a) {
        const float4* src = reinterpret_cast<const float4*>(vb_in + VS * (int64_t)T[a]);
        for (int q = 0; q < VS / 4; ++q) {
            const float4 u = __ldg(src + q);
            r[a][4 * q] = u.x; r[a][4 * q + 1] = u.y; r[a][4 * q + 2] = u.z; r[a][4 * q + 3] = u.w;
        }
    }
    const double grow = SWEPT ? S.margin : P.dhat + S.margin;
    const float grow_up = __double2float_ru(grow);
    float flo[3], fhi[3], mag[3];
    float vb[3][6];        // conservative FP32 box of each corner (swept: as swept_vert_f)
    for (int c = 0; c < 3; ++c) {
        float lo_c = INFINITY, hi_c = -INFINITY, m_c = grow_up;
        for (int a = 0; a < 3; ++a) {
            float pl, ph;
            if (SWEPT) {
                pl = r[a][c]; ph = r[a][3 + c];
                m_c += r[a][6 + c];   // position term
                m_c += r[a][9 + c];   // displacement term
            } else {
                pl = r[a][c]; ph = r[a][4 + c];
                m_c += fmaxf(fabsf(pl), fabsf(ph));
            }
            vb[a][c] = pl; vb[a][3 + c] = ph;
            lo_c = fminf(lo_c, pl); hi_c = fmaxf(hi_c, ph);
        }
        flo[c] = __fsub_rd(lo_c, grow_up); fhi[c] = __fadd_ru(hi_c, grow_up); mag[c] = m_c;
    }
    const int e = S.stri_env[t];
    I3 ca, cb;
    cell_range_f(S, e, flo, fhi, mag, ca, cb);
    bool any = false;
    for (int iz = ca.z; iz <= cb.z && !any; ++iz)
        for (int iy = ca.y; iy <= cb.y && !any; ++iy) {
            const int64_t c0 = cell_id(S, e, ca.x, iy, iz);
            any = start[c0 + (cb.x - ca.x) + 1] > start[c0];   // cells of a row are contiguous
        }
    if (!SWEPT && valid) {
        // the candidate counts start at zero (the exact tests append to them)
        *reinterpret_cast<int4*>(count + 4 * t) = make_int4(0, 0, 0, 0);
    }
    any = any && valid;
    // one atomic per warp for the survivors' slots
    const int idx = warp_reserve(any, Q.n);
    if (any) {
        Q.tri[idx] = (int32_t)t;
        float* bf = Q.boxf + 6 * (int64_t)idx;
        for (int c = 0; c < 3; ++c) { bf[c] = flo[c]; bf[3 + c] = fhi[c]; }
        float* w = Q.vboxf + 18 * (int64_t)idx;
        for (int a = 0; a < 3; ++a)
            for (int q = 0; q < 6; ++q) w[6 * a + q] = vb[a][q];
        if (!SWEPT) {
            // exact slave box for the edge and point tests
            double v[3][3];
            for (int a = 0; a < 3; ++a) load3(x, T[a], v[a]);
            double* b = Q.box + 6 * (int64_t)idx;
            for (int c = 0; c < 3; ++c) {
                b[c] = kmin3(v[0][c], v[1][c], v[2][c]);
                b[3 + c] = kmax3(v[0][c], v[1][c], v[2][c]);
            }
        }
        int32_t* cl = Q.cell + 6 * (int64_t)idx;
        cl[0] = ca.x; cl[1] = ca.y; cl[2] = ca.z; cl[3] = cb.x; cl[4] = cb.y; cl[5] = cb.z;
    }
}

// Entries of the cells in one x-row of the query range are contiguous in the
// cell lists (cells of a row are consecutive and the lists are a prefix sum
// over cells), so the warp walks each row's entries 32 at a time whatever
// the cells' occupancy.  A pair is kept only in the first cell common to the
// two cell ranges: in row (iy, iz) that is the entry at position k of cell
// cx = max(ca.x, mc.x) when start[cx] <= k < start[cx + 1].
__device__ __forceinline__ bool first_common_cell(const SceneView& S, const int32_t* __restrict__ start,
                                                  int e, I3 ca, int4 mc, int iy, int iz, int k) {
    if (max(ca.y, mc.y) != iy || max(ca.z, mc.z) != iz) return false;
    const int64_t cell = cell_id(S, e, max(ca.x, mc.x), iy, iz);
    return start[cell] <= k && k < start[cell + 1];
}

// Walk over the rows (iy, iz) of a cell range, 32 entries at a time.  While
// more() holds, [kb, kb + 32) intersected with [kb, k1) is the current chunk
// of row (iy, iz); empty rows are skipped.
struct RowWalk {
    const int32_t* __restrict__ start;
    int64_t off;           // first cell of the env
    int dx, dy;            // env grid dimensions in x and y
    int x0, nx, y0, y1, z1;
    int iy, iz, kb, k1;
    __device__ RowWalk(const SceneView& S, const int32_t* __restrict__ st, int e, I3 ca, I3 cb)
        : start(st), off(S.grid_off[e]), dx(S.grid_dim[3 * e]), dy(S.grid_dim[3 * e + 1]),
          x0(ca.x), nx(cb.x - ca.x + 1), y0(ca.y), y1(cb.y), z1(cb.z), iy(ca.y), iz(ca.z) {
        load_row();
        skip_empty();
    }
    __device__ void load_row() {
        const int64_t c0 = off + (int64_t)x0 + (int64_t)dx * ((int64_t)iy + (int64_t)dy * iz);
        kb = start[c0];
        k1 = start[c0 + nx];
    }
    __device__ void skip_empty() {
        while (kb >= k1) {
            if (++iy > y1) { iy = y0; ++iz; }
            if (iz > z1) return;
            load_row();
        }
    }
    __device__ bool more() const { return iz <= z1; }
    __device__ void next() { kb += 32; skip_empty(); }
};

// Primitive or (triangle, master) pairs passed between the launches of a
// query: p[i] = (x, y), n = pairs emitted (may exceed cap), overflow = the
// capacity needed when it does.
struct PairList {
    int2* p;
    int32_t* n;
    int32_t* overflow;
    int32_t cap;
};

// Walk of the cell entries of the filtered slave triangles (warp per
// triangle): emits (query-list index, master) for every entry that passes
// the coarse test on conservative FP32 boxes and the first-common-cell
// rule.  Shared by the contact and the swept query.
__global__ void __launch_bounds__(256)
k_query_walk(SceneView S, QueryList Q, const float* __restrict__ mboxf, const int4* __restrict__ mcell,
             const int32_t* __restrict__ start, const int32_t* __restrict__ ent, PairList L) {
    pass_dep_wait();
    // pairs are staged per warp in shared memory and written out kWalkStage
    // at a time, one atomic per batch (a counter bumped per chunk serialises)
    constexpr int kWalkStage = 128;
    __shared__ int2 s_stage[8][kWalkStage];
    const int lane = threadIdx.x & 31;
    int2* stage = s_stage[threadIdx.x >> 5];
    int ns = 0;
    auto flush = [&]() {
        int base = 0;
        if (lane == 0) {
            base = atomicAdd(L.n, ns);
            if (base + ns > L.cap) atomicMax(L.overflow, base + ns);
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        __syncwarp();
        for (int j = lane; j < ns; j += 32)
            if (base + j < L.cap) L.p[base + j] = stage[j];
        __syncwarp();
        ns = 0;
    };
    const int n_list = *Q.n;
    // Items per atomic on the shared work counter: one while the list is
    // short against the grid (balance matters), up to 16 for long lists (a
    // counter bumped millions of times serialises).
    const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    const int grab = max(1, min(16, n_list / (16 * nwarps)));
    for (int lb = next_items(Q.work, lane, grab); lb < n_list; lb = next_items(Q.work, lane, grab))
    for (int li = lb; li < min(lb + grab, n_list); ++li) {
        const float* qf = Q.boxf + 6 * (int64_t)li;
        const float qlo[3] = {qf[0], qf[1], qf[2]}, qhi[3] = {qf[3], qf[4], qf[5]};
        const int32_t* ql = Q.cell + 6 * (int64_t)li;
        const I3 ca = {ql[0], ql[1], ql[2]}, cb = {ql[3], ql[4], ql[5]};
        const int e = S.stri_env[Q.tri[li]];
        const int nx = cb.x - ca.x + 1, ny = cb.y - ca.y + 1;
        const int nrows = ny * (cb.z - ca.z + 1);
        const int64_t off = S.grid_off[e];
        const int dx = S.grid_dim[3 * e], dy = S.grid_dim[3 * e + 1];
        // rows (iy, iz) in batches of 32, one per lane: their entry ranges,
        // then their entries as one flat range walked 32 at a time
        for (int rb = 0; rb < nrows; rb += 32) {
            const int r = rb + lane;
            int k0 = 0, len = 0, iy = 0, iz = 0;
            if (r < nrows) {
                iy = ca.y + r % ny; iz = ca.z + r / ny;
                const int64_t c0 = off + (int64_t)ca.x + (int64_t)dx * ((int64_t)iy + (int64_t)dy * iz);
                k0 = start[c0];
                len = start[c0 + nx] - k0;
            }
            int incl = len;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int excl = incl - len;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int jb = 0; jb < total; jb += 32) {
                const int j = jb + lane;
                // the row holding flat entry j: the last lane whose prefix is
                // <= j (empty rows share the next row's prefix); every lane
                // searches, so the shuffles stay convergent
                int lo = 0;
                for (int step = 16; step > 0; step >>= 1) {
                    const int probe = __shfl_sync(0xffffffffu, excl, (lo + step) & 31);
                    if (lo + step < 32 && probe <= j) lo += step;
                }
                const int rk0 = __shfl_sync(0xffffffffu, k0, lo);
                const int rex = __shfl_sync(0xffffffffu, excl, lo);
                const int riy = __shfl_sync(0xffffffffu, iy, lo);
                const int riz = __shfl_sync(0xffffffffu, iz, lo);
                bool take = false;
                int32_t m = 0;
                if (j < total) {
                    const int k = rk0 + (j - rex);
                    m = ent[k];
                    const float* B = mboxf + 6 * (int64_t)m;
                    take = overlap_keep(qlo, qhi, B, B + 3) &&
                           first_common_cell(S, start, e, ca, mcell[m], riy, riz, k);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                if (bal == 0u) continue;
                if (ns + __popc(bal) > kWalkStage) flush();
                if (take) stage[ns + __popc(bal & lanemask_lt())] = make_int2(li, m);
                ns += __popc(bal);
            }
        }
    }
    if (ns > 0) flush();
}

// append v to the list of kind q of slave tri t (counts may exceed the
// capacity; the finishing pass flags that)
__device__ __forceinline__ void cand_append(const CandView& C, int64_t t, int q, int32_t v) {
    const int pos = atomicAdd(&C.count[4 * t + q], 1);
    const int cap = q == 0 ? C.cap_f : (q == 1 ? C.cap_e : C.cap_p);
    int32_t* L = q == 0 ? C.face : (q == 1 ? C.edge : C.point);
    if (pos < cap) L[t * cap + pos] = v;
}

// Exact candidate tests of one (filtered slave triangle, master triangle)
// pair: face (some sample ((b0 x0 + b1 x1) + b2 x2) inside the master box
// grown by eps), owned master edges and vertices (slave tri box vs their
// boxes grown by eps; FP32 pre-test on conservative boxes first).
template <int NK>
__global__ void __launch_bounds__(256)
k_contact_exact(SceneView S, Params P, CandView C, QueryList Q, PairList W,
                const double* __restrict__ x, const double* __restrict__ xm,
                const float* __restrict__ mboxf, const float* __restrict__ mboxf_in) {
    pass_dep_wait();
    const int n = min(*W.n, W.cap);
    const double eps = P.dhat;
    // eps rounded up, with a relative slack that covers the FP64 rounding of
    // the grown master box
    const float eps_up = __double2float_ru(eps * (1.0 + 0x1p-20));
    // and rounded down with the same slack: a sample bound inside the inner
    // FP32 box grown by eps_dn is inside the FP64 grown box, whose bounds
    // (lo - eps, hi + eps, one rounding each) are closer to the exact box
    // than eps 2^-20
    const float eps_dn = __double2float_rd(eps * (1.0 - 0x1p-20));
    const double (*rule)[3] = c_rule[P.L - 1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int2 pr = W.p[i];
        const int li = pr.x;
        const int32_t m = pr.y;
        // everything that depends only on the pair, loaded up front
        const int64_t t = Q.tri[li];
        const float* qf = Q.boxf + 6 * (int64_t)li;      // contains the slave box grown by eps
        const float* vb = Q.vboxf + 18 * (int64_t)li;
        const float* Bf = mboxf + 6 * (int64_t)m;
        int32_t own_e[3], own_v[3];
        for (int j = 0; j < 3; ++j) {
            own_e[j] = S.mtri_own_edge[3 * (int64_t)m + j];
            own_v[j] = S.mtri_own_vert[3 * (int64_t)m + j];
        }
        const int32_t* T = S.stri + 3 * t;
        // face: FP32 tests on conservative sample bounds -- certainly outside
        // every grown box (no pair), certainly inside one (a pair) -- then
        // the exact test for the rest
        bool maybe = false, sure = false;
        if (P.face_clip) {
            // clipped-overlap samples: the slave tri's box meets the master
            // tri's box grown by eps (exact FP64 boxes, as for edges)
            const double* qb = Q.box + 6 * (int64_t)li;
            double B[6];
            exact_mbox(S, xm, nullptr, m, B, B + 3);
            bool ok = true;
            for (int c = 0; c < 3 && ok; ++c) {
                const double lo = B[c] - eps, hi = B[3 + c] + eps;
                ok = qb[c] <= hi && lo <= qb[3 + c];
            }
            sure = ok;
        } else {
            const float* Bi = mboxf_in + 6 * (int64_t)m;
            float L[3], H[3], Li[3], Hi[3];
            for (int c = 0; c < 3; ++c) {
                L[c] = __fsub_rd(Bf[c], eps_up); H[c] = __fadd_ru(Bf[3 + c], eps_up);
                Li[c] = __fsub_ru(Bi[c], eps_dn); Hi[c] = __fadd_rd(Bi[3 + c], eps_dn);
            }
            const float (*rf)[6] = c_rule_f[P.L - 1];
            for (int q = 0; q < NK && !sure; ++q) {
                bool in = true, inside = true;
                for (int c = 0; c < 3 && in; ++c) {
                    // bounds of ((b0 x0 + b1 x1) + b2 x2) with b >= 0
                    float lo = 0.0f, hi = 0.0f;
                    for (int a = 0; a < 3; ++a) {
                        const float xl = vb[6 * a + c], xh = vb[6 * a + 3 + c];
                        lo = __fadd_rd(lo, __fmul_rd(xl >= 0.0f ? rf[q][a] : rf[q][3 + a], xl));
                        hi = __fadd_ru(hi, __fmul_ru(xh >= 0.0f ? rf[q][3 + a] : rf[q][a], xh));
                    }
                    in = !(hi < L[c] || lo > H[c]);
                    inside = inside && lo >= Li[c] && hi <= Hi[c];
                }
                maybe = maybe || in;
                sure = in && inside;
            }
        }
        if (sure) {
            cand_append(C, t, 0, m);
        } else if (maybe) {
            double x0[3], x1[3], x2[3];
            load3(x, T[0], x0); load3(x, T[1], x1); load3(x, T[2], x2);
            double B[6];
            exact_mbox(S, xm, nullptr, m, B, B + 3);
            const double l0 = B[0] - eps, l1 = B[1] - eps, l2 = B[2] - eps;
            const double h0 = B[3] + eps, h1 = B[4] + eps, h2 = B[5] + eps;
            bool hit = false;
            for (int q = 0; q < NK && !hit; ++q) {
                const double b0 = rule[q][0], b1 = rule[q][1], b2 = rule[q][2];
                const double sxq = b0 * x0[0] + b1 * x1[0] + b2 * x2[0];
                if (!(l0 <= sxq && sxq <= h0)) continue;
                const double syq = b0 * x0[1] + b1 * x1[1] + b2 * x2[1];
                if (!(l1 <= syq && syq <= h1)) continue;
                const double szq = b0 * x0[2] + b1 * x1[2] + b2 * x2[2];
                hit = l2 <= szq && szq <= h2;
            }
            if (hit) cand_append(C, t, 0, m);
        }
        const double* qb = Q.box + 6 * (int64_t)li;       // exact slave box
        for (int j = 0; j < 3; ++j) {
            const int32_t me = own_e[j];
            if (me < 0) continue;
            const int32_t ia = S.medge[2 * (int64_t)me], ib = S.medge[2 * (int64_t)me + 1];
            double ya[3], yb[3];
            load3(xm, ia, ya);
            load3(xm, ib, yb);
            float flo[3], fhi[3];
            for (int c = 0; c < 3; ++c) {
                flo[c] = fminf(lo_f32(ya[c]), lo_f32(yb[c]));
                fhi[c] = fmaxf(hi_f32(ya[c]), hi_f32(yb[c]));
            }
            if (!overlap_keep(qf, qf + 3, flo, fhi)) continue;
            bool ok = true;
            for (int c = 0; c < 3 && ok; ++c) {
                const double lo = dmin_(ya[c], yb[c]) - eps, hi = dmax_(ya[c], yb[c]) + eps;
                ok = qb[c] <= hi && lo <= qb[3 + c];
            }
            if (ok) cand_append(C, t, 1, me);
        }
        for (int j = 0; j < 3; ++j) {
            const int32_t u = own_v[j];
            if (u < 0) continue;
            double y[3];
            load3(xm, u, y);
            float flo[3], fhi[3];
            for (int c = 0; c < 3; ++c) { flo[c] = lo_f32(y[c]); fhi[c] = hi_f32(y[c]); }
            if (!overlap_keep(qf, qf + 3, flo, fhi)) continue;
            bool ok = true;
            for (int c = 0; c < 3 && ok; ++c) ok = qb[c] <= y[c] + eps && y[c] - eps <= qb[3 + c];
            if (ok) cand_append(C, t, 2, u);
        }
    }
}

// Finishing pass of the contact query (warp per filtered slave triangle):
// sort each list (the order of the appends depends on scheduling), flag
// overflowing lists, add the triangle to the active list or zero its
// outputs.
__global__ void __launch_bounds__(256)
k_contact_finish(CandView C, QueryList Q) {
    pass_dep_wait();
    const int lane = threadIdx.x & 31;
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    const int n_list = *Q.n;
    // one triangle at a time per warp; the triangles with candidates wait in
    // a lane register (lane j holds the j-th) and join the active list 32 at
    // a time, one atomic each time
    int32_t held = 0;
    int nheld = 0;
    auto flush = [&]() {
        int base = 0;
        if (lane == 0) base = atomicAdd(C.n_active, nheld);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane < nheld) C.active[base + lane] = held;
        nheld = 0;
    };
    for (int li = warp; li < n_list; li += nwarps) {
        const int64_t t = Q.tri[li];
        const int4 cn = *reinterpret_cast<const int4*>(C.count + 4 * t);
        const int nf = cn.x, ne = cn.y, np = cn.z;
        warp_sort(C.face + t * C.cap_f, min(nf, C.cap_f), lane);
        warp_sort(C.edge + t * C.cap_e, min(ne, C.cap_e), lane);
        warp_sort(C.point + t * C.cap_p, min(np, C.cap_p), lane);
        if (lane == 0) {
            if (nf > C.cap_f) atomicMax(&C.overflow[0], nf);
            if (ne > C.cap_e) atomicMax(&C.overflow[1], ne);
            if (np > C.cap_p) atomicMax(&C.overflow[2], np);
        }
        // triangles without candidates are not stamped by the evaluation, so
        // their stored outputs are never read
        if (nf + ne + np > 0) {
            if (lane == nheld) held = (int32_t)t;
            if (++nheld == 32) flush();
        }
    }
    if (nheld > 0) flush();
}

// ---------------------------------------------------------------------------
// additive CCD (Li, Kaufman, Jiang 2021, Alg. 1), thickness 0
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sub3(const double* a, const double* b, double* o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ double ps_dist2(const double* p, const double* a, const double* b) {
    double ab[3], ap[3], q[3], d[3];
    sub3(b, a, ab); sub3(p, a, ap);
    double t = dot3(ap, ab) / dot3(ab, ab);
    t = dmin_(dmax_(t, 0.0), 1.0);
    for (int c = 0; c < 3; ++c) q[c] = a[c] + t * ab[c];
    sub3(p, q, d);
    return dot3(d, d);
}

// point-triangle: plane distance when the projection is inside, else the
// nearest edge
__device__ double pt_dist2(const double* p, const double* t0, const double* t1, const double* t2) {
    double e1[3], e2[3], d[3];
    sub3(t1, t0, e1); sub3(t2, t0, e2); sub3(p, t0, d);
    double a = dot3(e1, e1), bb = dot3(e1, e2), c = dot3(e2, e2);
    double r1 = dot3(d, e1), r2 = dot3(d, e2);
    double det = a * c - bb * bb;
    double v = (c * r1 - bb * r2) / det;
    double w = (a * r2 - bb * r1) / det;
    double u = 1.0 - v - w;
    if (u >= 0.0 && v >= 0.0 && w >= 0.0) {
        double e1b[3], e2b[3], n[3], db[3];
        sub3(t1, t0, e1b); sub3(t2, t0, e2b); cross3(e1b, e2b, n); sub3(p, t0, db);
        double h = dot3(db, n);
        return h * h / dot3(n, n);
    }
    return dmin_(ps_dist2(p, t0, t1), dmin_(ps_dist2(p, t1, t2), ps_dist2(p, t2, t0)));
}

// segment-segment: four endpoint-segment distances and the line-line
// distance when both closest-point parameters fall inside the segments
__device__ double ee_dist2(const double* a0, const double* a1, const double* b0, const double* b1) {
    double d = dmin_(dmin_(ps_dist2(a0, b0, b1), ps_dist2(a1, b0, b1)),
                     dmin_(ps_dist2(b0, a0, a1), ps_dist2(b1, a0, a1)));
    double u[3], v[3], w[3];
    sub3(a1, a0, u); sub3(b1, b0, v); sub3(a0, b0, w);
    double A = dot3(u, u), B = dot3(u, v), Cc = dot3(v, v), D = dot3(u, w), E = dot3(v, w);
    double den = A * Cc - B * B;
    if (den > 1e-14 * A * Cc) {
        double sc = (B * E - Cc * D) / den, tc = (A * E - B * D) / den;
        if (sc > 0.0 && sc < 1.0 && tc > 0.0 && tc < 1.0) {
            double n[3];
            cross3(u, v, n);
            double h = dot3(w, n);
            d = dmin_(d, h * h / dot3(n, n));
        }
    }
    return d;
}

// x[12], p[12] (modified); type 0 point-triangle, 1 edge-edge.  Returns the
// largest safe fraction found in [0, tc] (tc when nothing closes in time).
__device__ __noinline__ double accd(int type, double* x, double* p, double s, double tc, int max_iter,
                       int* iters) {
    double pbar[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 4; ++i)
        for (int c = 0; c < 3; ++c) pbar[c] += p[3 * i + c];
    for (int c = 0; c < 3; ++c) pbar[c] = pbar[c] / 4.0;
    for (int i = 0; i < 4; ++i)
        for (int c = 0; c < 3; ++c) p[3 * i + c] -= pbar[c];
    double n[4];
    for (int i = 0; i < 4; ++i) n[i] = sqrt(dot3(p + 3 * i, p + 3 * i));
    double lp = type == 0 ? n[0] + dmax_(n[1], dmax_(n[2], n[3])) : dmax_(n[0], n[1]) + dmax_(n[2], n[3]);
    *iters = 0;
    if (lp == 0.0) return tc;
    // The first advance is tl = (1-s) d / lp and the iteration returns tc as
    // soon as t = tl exceeds tc, whatever the distance after the advance.  A
    // lower bound of d (the distance between the two primitives' boxes), with
    // a relative margin far above rounding, settles that case without the
    // exact distance; either way the result equals the full iteration's.
    {
        double lo0[3], hi0[3], lo1[3], hi1[3];
        const int na = type == 0 ? 1 : 2;
        for (int c = 0; c < 3; ++c) {
            lo0[c] = hi0[c] = x[c];
            lo1[c] = hi1[c] = x[3 * na + c];
        }
        for (int i = 1; i < na; ++i)
            for (int c = 0; c < 3; ++c) { lo0[c] = dmin_(lo0[c], x[3 * i + c]); hi0[c] = dmax_(hi0[c], x[3 * i + c]); }
        for (int i = na + 1; i < 4; ++i)
            for (int c = 0; c < 3; ++c) { lo1[c] = dmin_(lo1[c], x[3 * i + c]); hi1[c] = dmax_(hi1[c], x[3 * i + c]); }
        double g2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double gap = dmax_(0.0, dmax_(lo0[c] - hi1[c], lo1[c] - hi0[c]));
            g2 += gap * gap;
        }
        if ((1.0 - s) * sqrt(g2) * (1.0 - 1e-9) > tc * lp) { *iters = 1; return tc; }
    }
    double d2 = type == 0 ? pt_dist2(x, x + 3, x + 6, x + 9) : ee_dist2(x, x + 3, x + 6, x + 9);
    double d = sqrt(d2);
    if (d == 0.0) return 0.0;
    double gstop = s * d;
    double t = 0.0;
    double tl = (1.0 - s) * d / lp;
    if (tl > tc) { *iters = 1; return tc; }
    for (int it = 0; it < max_iter; ++it) {
        *iters = it + 1;
        for (int i = 0; i < 12; ++i) x[i] = x[i] + tl * p[i];
        d2 = type == 0 ? pt_dist2(x, x + 3, x + 6, x + 9) : ee_dist2(x, x + 3, x + 6, x + 9);
        d = sqrt(d2);
        if (t > 0.0 && d < gstop) return t;
        t = t + tl;
        if (t > tc) return tc;
        tl = 0.9 * d / lp;
    }
    return t;
}

__device__ __forceinline__ bool overlap(const double* alo, const double* ahi, const double* blo,
                                        const double* bhi) {
    return alo[0] <= bhi[0] && blo[0] <= ahi[0] && alo[1] <= bhi[1] && blo[1] <= ahi[1] &&
           alo[2] <= bhi[2] && blo[2] <= ahi[2];
}

// atomic minimum of a non-negative double via its bit pattern
__device__ __forceinline__ void atomic_min_pos(unsigned long long* dst, double v) {
    atomicMin(dst, (unsigned long long)__double_as_longlong(v));
}

// Primitive pairs that ACCD must test (PairList), emitted by k_ccd_exact
// and consumed by k_accd_pairs: x = first id | kind << 30, y = second id.
// Kinds: 0 slave vertex / master tri, 1 master vertex / slave tri, 2 slave
// edge / master edge.
__device__ __forceinline__ void emit_pair(const PairList& L, int kind, int32_t a, int32_t b) {
    const int pos = atomicAdd(L.n, 1);
    if (pos < L.cap) L.p[pos] = make_int2(a | (kind << 30), b);
    else atomicMax(L.overflow, pos + 1);
}

// Swept query, in three launches so that each stays light: the walk over
// cell entries (k_query_walk) emits the (triangle, master) pairs that pass
// the coarse test on conservative FP32 boxes and the first-common-cell
// rule; k_ccd_exact (thread per such pair) tests the owned primitives,
// first on FP32 boxes, then, for the pairs that pass, on their exact FP64
// boxes, and emits the primitive pairs that overlap; k_accd_pairs runs ACCD
// on those.  The primitive pairs are exactly those of the plain FP64 box
// tests.

// corner of slave tri T holding vertex v (v is one of T's vertices)
__device__ __forceinline__ int corner_of(const int32_t* T, int32_t v) {
    return T[0] == v ? 0 : (T[1] == v ? 1 : 2);
}

// the exact primitive tests of one (filtered slave triangle, master) pair
__global__ void __launch_bounds__(256)
k_ccd_exact(SceneView S, QueryList Q, PairList C, const double* __restrict__ x,
            const double* __restrict__ dx, const double* __restrict__ xm0,
            const double* __restrict__ dxm, const float* __restrict__ mboxf, PairList L) {
    pass_dep_wait();
    const int n = min(*C.n, C.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int2 pr = C.p[i];
        const int li = pr.x;
        const int32_t m = pr.y;
        const int64_t t = Q.tri[li];
        const int32_t* T = S.stri + 3 * t;
        const float* vb = Q.vboxf + 18 * (int64_t)li;     // swept boxes of T's corners
        const float* qf = Q.boxf + 6 * (int64_t)li;
        const float* Bf = mboxf + 6 * (int64_t)m;
        // slave vertices owned by t vs master triangle m
        for (int j = 0; j < 3; ++j) {
            const int32_t v = S.stri_own_vert[3 * t + j];
            if (v < 0) continue;
            const float* b = vb + 6 * corner_of(T, v);
            if (!overlap_keep(b, b + 3, Bf, Bf + 3)) continue;
            double vlo[3], vhi[3], B[6];
            swept_vert(x, dx, v, vlo, vhi);
            exact_mbox(S, xm0, dxm, m, B, B + 3);
            if (overlap(vlo, vhi, B, B + 3)) emit_pair(L, 0, v, m);
        }
        // master vertices owned by m vs slave triangle t
        for (int j = 0; j < 3; ++j) {
            const int32_t u = S.mtri_own_vert[3 * (int64_t)m + j];
            if (u < 0) continue;
            float uf_lo[3], uf_hi[3];
            swept_vert_f(xm0, dxm, u, uf_lo, uf_hi);
            if (!overlap_keep(uf_lo, uf_hi, qf, qf + 3)) continue;
            double ulo[3], uhi[3], tlo[3], thi[3], l2[3], h2[3];
            swept_vert(xm0, dxm, u, ulo, uhi);
            swept_vert(x, dx, T[0], tlo, thi);
            swept_vert(x, dx, T[1], l2, h2);
            grow_box(tlo, thi, l2, h2);
            swept_vert(x, dx, T[2], l2, h2);
            grow_box(tlo, thi, l2, h2);
            if (overlap(ulo, uhi, tlo, thi)) emit_pair(L, 1, u, (int32_t)t);
        }
        // slave edges owned by t vs master edges owned by m
        float se_lo[3][3], se_hi[3][3];
        int32_t se[3];
        for (int j = 0; j < 3; ++j) {
            se[j] = S.stri_own_edge[3 * t + j];
            if (se[j] < 0) continue;
            const float* b0 = vb + 6 * corner_of(T, S.sedge[2 * (int64_t)se[j]]);
            const float* b1 = vb + 6 * corner_of(T, S.sedge[2 * (int64_t)se[j] + 1]);
            for (int c = 0; c < 3; ++c) {
                se_lo[j][c] = fminf(b0[c], b1[c]);
                se_hi[j][c] = fmaxf(b0[3 + c], b1[3 + c]);
            }
        }
        for (int q = 0; q < 3; ++q) {
            const int32_t em = S.mtri_own_edge[3 * (int64_t)m + q];
            if (em < 0) continue;
            const int32_t m0 = S.medge[2 * (int64_t)em], m1 = S.medge[2 * (int64_t)em + 1];
            float bf_lo[3], bf_hi[3], fl2[3], fh2[3];
            swept_vert_f(xm0, dxm, m0, bf_lo, bf_hi);
            swept_vert_f(xm0, dxm, m1, fl2, fh2);
            for (int c = 0; c < 3; ++c) { bf_lo[c] = fminf(bf_lo[c], fl2[c]); bf_hi[c] = fmaxf(bf_hi[c], fh2[c]); }
            for (int j = 0; j < 3; ++j) {
                if (se[j] < 0) continue;
                if (!overlap_keep(se_lo[j], se_hi[j], bf_lo, bf_hi)) continue;
                const int32_t sa = S.sedge[2 * (int64_t)se[j]], sb = S.sedge[2 * (int64_t)se[j] + 1];
                double alo[3], ahi[3], blo[3], bhi[3], l2[3], h2[3];
                swept_vert(x, dx, sa, alo, ahi);
                swept_vert(x, dx, sb, l2, h2);
                grow_box(alo, ahi, l2, h2);
                swept_vert(xm0, dxm, m0, blo, bhi);
                swept_vert(xm0, dxm, m1, l2, h2);
                grow_box(blo, bhi, l2, h2);
                if (overlap(alo, ahi, blo, bhi)) emit_pair(L, 2, se[j], em);
            }
        }
    }
}

// ACCD of the emitted pairs, one thread per pair; the minimum and the
// counters do not depend on the order (exact minimum, integer sums).
__global__ void __launch_bounds__(256)
k_accd_pairs(SceneView S, Params P, PairList L, const double* __restrict__ x,
             const double* __restrict__ dx, const double* __restrict__ xm0,
             const double* __restrict__ dxm, unsigned long long* alpha_bits, long long* counters,
             int alpha_stride) {
    pass_dep_wait();
    const int n = min(*L.n, L.cap);
    double best = 1.0;
    long long n_pt = 0, n_ee = 0;
    int cap_hit = 0;
    // alpha_stride > 0: one bound per environment at alpha_bits[alpha_stride
    // * env]; a thread keeps the minimum of its current environment and
    // publishes it when the environment changes (the minimum is exact)
    int env = -1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int2 pr = L.p[i];
        const int kind = (int)((unsigned)pr.x >> 30);
        const int32_t a = pr.x & 0x3FFFFFFF, b = pr.y;
        if (alpha_stride > 0) {
            const int e = kind == 0 ? S.mtri_env[b] : kind == 1 ? S.stri_env[b] : S.mvert_env[S.medge[2 * (int64_t)b]];
            if (e != env) {
                if (env >= 0 && best < 1.0) atomic_min_pos(alpha_bits + (int64_t)alpha_stride * env, best);
                env = e;
                best = 1.0;
            }
        }
        double X12[12], P12[12];
        int32_t va[4];          // the four vertices: first primitive's, then the second's
        bool first_slave;
        if (kind == 0) {        // slave vertex a, master tri b
            const int32_t* M = S.mtri + 3 * (int64_t)b;
            va[0] = a; va[1] = M[0]; va[2] = M[1]; va[3] = M[2];
            first_slave = true;
        } else if (kind == 1) { // master vertex a, slave tri b
            const int32_t* T = S.stri + 3 * (int64_t)b;
            va[0] = a; va[1] = T[0]; va[2] = T[1]; va[3] = T[2];
            first_slave = false;
        } else {                // slave edge a, master edge b
            va[0] = S.sedge[2 * (int64_t)a]; va[1] = S.sedge[2 * (int64_t)a + 1];
            va[2] = S.medge[2 * (int64_t)b]; va[3] = S.medge[2 * (int64_t)b + 1];
            first_slave = true;
        }
        const int n_first = kind == 2 ? 2 : 1;
        for (int q = 0; q < 4; ++q) {
            const bool slave = (q < n_first) == first_slave;
            const double* Px = slave ? x : xm0;
            const double* Pd = slave ? dx : dxm;
            for (int c = 0; c < 3; ++c) {
                X12[3 * q + c] = Px[3 * (int64_t)va[q] + c];
                P12[3 * q + c] = Pd ? Pd[3 * (int64_t)va[q] + c] : 0.0;
            }
        }
        // ACCD's tc: the smallest bound known so far, this thread's or one
        // published by any thread (alpha_bits only ever holds pair results or
        // its initial 1).  A pair whose time of impact lies above tc stops as
        // soon as its advance passes tc and returns tc, which cannot lower the
        // minimum; a pair whose result lies below tc runs exactly as with
        // tc = 1 (its advances never pass tc), so the minimum is bitwise that
        // of running every pair to tc = 1.
        unsigned long long* pub = alpha_stride > 0 ? alpha_bits + (int64_t)alpha_stride * env : alpha_bits;
        const double known = __longlong_as_double((long long)*reinterpret_cast<volatile unsigned long long*>(pub));
        const double tc = dmin_(best, dmin_(known, 1.0));
        int it;
        const double r = accd(kind == 2 ? 1 : 0, X12, P12, P.ccd_slack, tc, P.ccd_max_iter, &it);
        if (kind == 2) ++n_ee; else ++n_pt;
        cap_hit |= it >= P.ccd_max_iter;
        if (r < best) {
            best = r;
            if (r < known) atomic_min_pos(pub, r);   // let the other threads stop early too
        }
    }
    if (alpha_stride > 0 && env >= 0 && best < 1.0) atomic_min_pos(alpha_bits + (int64_t)alpha_stride * env, best);
    if (alpha_stride > 0) best = 1.0;
    // warp reductions (min is exact; counters are integers)
    for (int o = 16; o > 0; o >>= 1) {
        best = dmin_(best, __shfl_xor_sync(0xffffffffu, best, o));
        n_pt += __shfl_xor_sync(0xffffffffu, n_pt, o);
        n_ee += __shfl_xor_sync(0xffffffffu, n_ee, o);
        cap_hit |= __shfl_xor_sync(0xffffffffu, cap_hit, o);
    }
    if ((threadIdx.x & 31) != 0) return;
    if (best < 1.0) atomic_min_pos(alpha_bits, best);
    if (n_pt) atomic_add_ll(&counters[0], n_pt);
    if (n_ee) atomic_add_ll(&counters[1], n_ee);
    if (cap_hit) atomicMax(&counters[2], 1LL);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t bp_init_constants(const double* rule_l1l2) {
    // FP32 brackets of the rule's barycentrics: lo <= b <= hi
    float f[2][16][6];
    for (int l = 0; l < 2; ++l)
        for (int k = 0; k < 16; ++k)
            for (int a = 0; a < 3; ++a) {
                const double b = rule_l1l2[(l * 16 + k) * 3 + a];
                const float r = (float)b;
                f[l][k][a] = (double)r > b ? std::nextafter(r, -INFINITY) : r;
                f[l][k][3 + a] = (double)r < b ? std::nextafter(r, INFINITY) : r;
            }
    GMCP_CUDA_TRY(cudaMemcpyToSymbol(c_rule_f, f, sizeof(f)));
    return cudaMemcpyToSymbol(c_rule, rule_l1l2, sizeof(double) * 2 * 16 * 3);
}

cudaError_t bp_build_grid(Ctx& c, const double* xm, const double* dxm, bool swept, bool lazy) {
    ProfScope ps(c.prof, c.stream, "grid");
    SceneView S = c.view();
    cudaStream_t s = c.stream;
    GMCP_CUDA_TRY(c.mcell.ensure((size_t)c.nmt + 1));
    GMCP_CUDA_TRY(c.mboxf.ensure(6 * (size_t)c.nmt + 6));
    GMCP_CUDA_TRY(c.mboxf_in.ensure(6 * (size_t)c.nmt + 6));
    GMCP_CUDA_TRY(c.cell_cnt.ensure((size_t)c.n_cells + 1));
    GMCP_CUDA_TRY(c.cell_start.ensure((size_t)c.n_cells + 2));
    GMCP_CUDA_TRY(c.scan_tmp.ensure(2 * scan_tmp_size(c.n_cells)));
    GMCP_CUDA_TRY(cudaMemsetAsync(c.cell_cnt.p, 0, sizeof(int32_t) * (c.n_cells + 1), s));
    const int B = 256;
    const unsigned g = (unsigned)((c.nmt + B - 1) / B);
    if (c.nmt > 0) {
        launch_dep(k_mtri_box_count, g, B, 0, s, S, xm, swept ? dxm : nullptr, c.mboxf.p, c.mcell.p, c.cell_cnt.p,
                                         c.mboxf_in.p);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    // scan into start + 1 (start[0] = 0), which the fill advances in place
    GMCP_CUDA_TRY(cudaMemsetAsync(c.cell_start.p, 0, sizeof(int32_t), s));
    GMCP_CUDA_TRY(exclusive_scan_i32(c.cell_cnt.p, c.cell_start.p + 1, c.n_cells, c.scan_tmp.p,
                                     c.scan_tmp.n, s));
    if (lazy) {
        // Cells are at least the mean master extent, so a triangle spans a few
        // cells per axis and 27 entries per triangle is ample on average; the
        // fill flags any overflow, which the caller checks when it
        // synchronises and then redoes the pass with a larger list.
        GMCP_CUDA_TRY(c.cell_ent.ensure(std::max<size_t>(27 * (size_t)c.nmt + 1, c.cell_ent.n)));
    } else {
        int32_t total = 0;
        GMCP_CUDA_TRY(cudaMemcpyAsync(&total, c.cell_start.p + 1 + c.n_cells, sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, s));
        GMCP_CUDA_TRY(cudaStreamSynchronize(s));
        GMCP_CUDA_TRY(c.cell_ent.ensure((size_t)total + 1));
    }
    if (c.nmt > 0) {
        launch_dep(k_mtri_fill, g, B, 0, s, S, c.mboxf.p, c.mcell.p, c.cell_start.p + 1, c.cell_ent.p,
                                    (int64_t)c.cell_ent.n, c.misc_i32.p + 12);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

// the contact and swept queries share the list buffers but keep their
// lengths apart (slots 8 and 9), so both survive a pass for the statistics
// The contact and the swept query keep separate lists, counters and work
// counters (slots 8 / 5 and 9 / 7), so that the two can run concurrently.
static QueryList query_list(Ctx& c, bool swept) {
    QueryBufs& B = swept ? c.qswept : c.qcontact;
    QueryList Q;
    Q.n = c.misc_i32.p + (swept ? 9 : 8);
    Q.work = c.misc_i32.p + (swept ? 7 : 5);
    Q.tri = B.tri.p;
    Q.box = B.box.p;
    Q.boxf = B.boxf.p;
    Q.vboxf = B.vboxf.p;
    Q.cell = B.cell.p;
    return Q;
}

static cudaError_t ensure_query_list(Ctx& c, bool swept) {
    QueryBufs& B = swept ? c.qswept : c.qcontact;
    GMCP_CUDA_TRY(B.tri.ensure((size_t)c.ns + 1));
    if (!swept) GMCP_CUDA_TRY(B.box.ensure(6 * (size_t)c.ns + 6));
    GMCP_CUDA_TRY(B.boxf.ensure(6 * (size_t)c.ns + 6));
    GMCP_CUDA_TRY(B.vboxf.ensure(18 * (size_t)c.ns + 18));
    GMCP_CUDA_TRY(B.cell.ensure(6 * (size_t)c.ns + 6));
    return cudaSuccess;
}

static unsigned persistent_blocks(Ctx& c) { return (unsigned)(sm_count(c.device) * c.tune_query_bpsm); }

cudaError_t bp_query_contact(Ctx& c, const double* x, const double* xm, bool lazy) {
    ProfScope ps(c.prof, c.stream, "query");
    SceneView S = c.view();
    Params P = c.P;
    cudaStream_t s = c.stream;
    CandView C = c.cand();
    GMCP_CUDA_TRY(ensure_query_list(c, false));
    QueryList Q = query_list(c, false);
    GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p, 0, sizeof(int32_t) * 12, s));
    if (c.ns == 0) return cudaSuccess;
    launch_dep(k_vert_bounds<false>, (unsigned)((c.n_svert + 255) / 256), 256, 0, s, c.n_svert, c.svert.p, x, nullptr,
                                                                           c.vbound_c.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    launch_dep(k_query_filter<false>, (unsigned)((c.ns + 255) / 256), 256, 0, s, 
        S, P, x, c.vbound_c.p, c.cell_start.p, Q, c.cand_count.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    if (c.cap_coarse == 0) c.cap_coarse = (int32_t)std::min<int64_t>((1 << 16) + 2 * c.ns, 1 << 30);
    const unsigned flat = (unsigned)(sm_count(c.device) * 8);
    for (int attempt = 0;; ++attempt) {
        GMCP_CUDA_TRY(c.coarse_pairs.ensure((size_t)c.cap_coarse));
        // (triangle, master) pairs: count in slot 6, needed capacity in slot 15
        PairList W{c.coarse_pairs.p, c.misc_i32.p + 6, c.misc_i32.p + 15, c.cap_coarse};
        GMCP_CUDA_TRY(cudaMemsetAsync(W.n, 0, sizeof(int32_t), s));
        GMCP_CUDA_TRY(cudaMemsetAsync(W.overflow, 0, sizeof(int32_t), s));
        GMCP_CUDA_TRY(cudaMemsetAsync(Q.work, 0, sizeof(int32_t), s));
        launch_dep(k_query_walk, persistent_blocks(c), 256, 0, s, S, Q, c.mboxf.p, c.mcell.p, c.cell_start.p,
                                                          c.cell_ent.p, W);
        GMCP_CUDA_TRY(cudaGetLastError());
        if (P.nk == 4)
            launch_dep(k_contact_exact<4>, flat, 256, 0, s, S, P, C, Q, W, x, xm, c.mboxf.p, c.mboxf_in.p);
        else
            launch_dep(k_contact_exact<16>, flat, 256, 0, s, S, P, C, Q, W, x, xm, c.mboxf.p, c.mboxf_in.p);
        GMCP_CUDA_TRY(cudaGetLastError());
        if (lazy) break;   // the caller reads the overflow slot after it synchronises
        int32_t need = 0;
        GMCP_CUDA_TRY(cudaMemcpyAsync(&need, W.overflow, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        GMCP_CUDA_TRY(cudaStreamSynchronize(s));
        if (need == 0) break;
        if (attempt >= 4) return cudaErrorInvalidValue;
        c.cap_coarse = std::max(c.cap_coarse, need);
        // the lists restart empty
        GMCP_CUDA_TRY(cudaMemsetAsync(c.cand_count.p, 0, sizeof(int32_t) * 4 * c.ns, s));
    }
    launch_dep(k_contact_finish, persistent_blocks(c), 256, 0, s, C, Q);
    return cudaGetLastError();
}

cudaError_t bp_ccd_accd(Ctx& c, const double* x, const double* dx, const double* xm0,
                        const double* dxm, unsigned long long* alpha_bits, long long* counters,
                        bool reuse_grid, bool lazy, int alpha_stride) {
    if (!(reuse_grid && dxm == nullptr)) GMCP_CUDA_TRY(bp_build_grid(c, xm0, dxm, true, lazy));
    ProfScope ps(c.prof, c.stream, "accd");
    if (c.ns == 0) return cudaSuccess;
    SceneView S = c.view();
    GMCP_CUDA_TRY(ensure_query_list(c, true));
    QueryList Q = query_list(c, true);
    GMCP_CUDA_TRY(cudaMemsetAsync(Q.n, 0, sizeof(int32_t), c.stream));
    launch_dep(k_vert_bounds<true>, (unsigned)((c.n_svert + 255) / 256), 256, 0, c.stream, c.n_svert, c.svert.p, x, dx,
                                                                                 c.vbound_s.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    launch_dep(k_query_filter<true>, (unsigned)((c.ns + 255) / 256), 256, 0, c.stream, 
        S, c.P, x, c.vbound_s.p, c.cell_start.p, Q, nullptr);
    GMCP_CUDA_TRY(cudaGetLastError());
    if (c.cap_ccd == 0) c.cap_ccd = (int32_t)std::min<int64_t>((1 << 16) + c.ns / 4, 1 << 30);
    if (c.cap_coarse_swept == 0) c.cap_coarse_swept = (int32_t)std::min<int64_t>((1 << 16) + 2 * c.ns, 1 << 30);
    const unsigned flat = (unsigned)(sm_count(c.device) * 8);
    for (int attempt = 0;; ++attempt) {
        GMCP_CUDA_TRY(c.ccd_pairs.ensure((size_t)c.cap_ccd));
        GMCP_CUDA_TRY(c.coarse_swept.ensure((size_t)c.cap_coarse_swept));
        // coarse pairs: count in slot 11, needed capacity in slot 14;
        // primitive pairs: count in slot 10, needed capacity in slot 13
        PairList C{c.coarse_swept.p, c.misc_i32.p + 11, c.misc_i32.p + 14, c.cap_coarse_swept};
        PairList L{c.ccd_pairs.p, c.misc_i32.p + 10, c.misc_i32.p + 13, c.cap_ccd};
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + 10, 0, 2 * sizeof(int32_t), c.stream));
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + 13, 0, 2 * sizeof(int32_t), c.stream));
        GMCP_CUDA_TRY(cudaMemsetAsync(Q.work, 0, sizeof(int32_t), c.stream));
        launch_dep(k_query_walk, persistent_blocks(c), 256, 0, c.stream, S, Q, c.mboxf.p, c.mcell.p, c.cell_start.p,
                                                               c.cell_ent.p, C);
        GMCP_CUDA_TRY(cudaGetLastError());
        launch_dep(k_ccd_exact, flat, 256, 0, c.stream, S, Q, C, x, dx, xm0, dxm, c.mboxf.p, L);
        GMCP_CUDA_TRY(cudaGetLastError());
        launch_dep(k_accd_pairs, flat, 256, 0, c.stream, S, c.P, L, x, dx, xm0, dxm, alpha_bits, counters, alpha_stride);
        GMCP_CUDA_TRY(cudaGetLastError());
        // a lazy caller reads the overflow slots after it synchronises and redoes the pass
        if (lazy) return cudaSuccess;
        int32_t need[2] = {0, 0};
        GMCP_CUDA_TRY(cudaMemcpyAsync(need, c.misc_i32.p + 13, sizeof(need), cudaMemcpyDeviceToHost, c.stream));
        GMCP_CUDA_TRY(cudaStreamSynchronize(c.stream));
        if (need[0] == 0 && need[1] == 0) return cudaSuccess;
        if (attempt >= 4) return cudaErrorInvalidValue;
        // the minimum over the pairs seen so far stays valid; the counters restart
        c.cap_ccd = std::max(c.cap_ccd, need[0]);
        c.cap_coarse_swept = std::max(c.cap_coarse_swept, need[1]);
        GMCP_CUDA_TRY(cudaMemsetAsync(counters, 0, 3 * sizeof(long long), c.stream));
    }
}

}  // namespace gmcp

// ===========================================================================
// Allocation-free additive-CCD minimum (ipc_accd_min_noalloc).
//
// Some callers must not allocate device memory once they are running: a
// robot controller's real-time loop cannot afford cudaMalloc, which may block
// and synchronise the whole device, and some host frameworks route every
// device allocation through their own pool and forbid direct cudaMalloc.
// This entry point gives such callers the additive-CCD step bound over a
// context created beforehand without touching any allocator: its only
// scratch (the minimum's bit pattern, three counters and, for a moving
// master, the master displacement) lives in the file-scope array below,
// 4 MiB that every GPU which loads the library keeps until the process
// exits.  The pairs are enumerated by brute force (every slave triangle
// against every master triangle of its environment) with the same owned-
// primitive rules, swept-box filters and ACCD routine as k_query_ccd, so the
// result equals the alpha_accd of ipc_ccd_max_step bit for bit; the cost is
// O(slave tris x master tris), meant for small scenes.
// ===========================================================================
namespace gmcp {
Ctx& ctx_of(ipc_ctx* h);   // api.cu
}

static constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;
static constexpr size_t kNoAllocHeaderBytes = 256;     // alpha bits + 3 counters, padded
static constexpr int64_t kNoAllocMaxMasterVerts =
    (int64_t)((kNoAllocScratchBytes - kNoAllocHeaderBytes) / (3 * sizeof(double)));
static __device__ __align__(256) unsigned char g_accd_scratch[kNoAllocScratchBytes];

namespace gmcp {
namespace {

__global__ void k_noalloc_reset(unsigned long long* hdr) {
    pass_dep_wait();
    hdr[0] = 0x3FF0000000000000ULL;   // alpha = 1.0
    hdr[1] = 0; hdr[2] = 0; hdr[3] = 0;
}

__global__ void k_noalloc_sub(const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ o, int64_t n) {
    pass_dep_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = a[i] - b[i];
}

// one thread per slave triangle, blockIdx.y selects a chunk of master tris
__global__ void __launch_bounds__(128)
k_accd_brute(SceneView S, Params P, const double* __restrict__ x, const double* __restrict__ dx,
             const double* __restrict__ xm0, const double* __restrict__ dxm, int m_chunk,
             unsigned long long* alpha_bits, long long* counters) {
    pass_dep_wait();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.ns) return;
    const int64_t m_begin = (int64_t)blockIdx.y * m_chunk;
    const int64_t m_end = min((int64_t)S.nmt, m_begin + m_chunk);
    const int32_t* T = S.stri + 3 * t;
    double tlo[3], thi[3];
    swept_vert(x, dx, T[0], tlo, thi);
    for (int a = 1; a < 3; ++a) {
        double l[3], h[3];
        swept_vert(x, dx, T[a], l, h);
        grow_box(tlo, thi, l, h);
    }
    const int e = S.stri_env[t];
    double best = 1.0;
    long long n_pt = 0, n_ee = 0;
    int cap_hit = 0;
    for (int64_t m = m_begin; m < m_end; ++m) {
        if (S.mtri_env[m] != e) continue;
        const int32_t* M = S.mtri + 3 * m;
        double B[6];
        swept_vert(xm0, dxm, M[0], B, B + 3);
        for (int a = 1; a < 3; ++a) {
            double l[3], h[3];
            swept_vert(xm0, dxm, M[a], l, h);
            grow_box(B, B + 3, l, h);
        }
        // every primitive box lies inside its triangle's box
        if (!overlap(tlo, thi, B, B + 3)) continue;
        double X12[12], P12[12];
        int it;
        for (int j = 0; j < 3; ++j) {
            const int32_t v = S.stri_own_vert[3 * t + j];
            if (v < 0) continue;
            double vlo[3], vhi[3];
            swept_vert(x, dx, v, vlo, vhi);
            if (!overlap(vlo, vhi, B, B + 3)) continue;
            for (int c = 0; c < 3; ++c) {
                X12[c] = x[3 * (int64_t)v + c]; P12[c] = dx[3 * (int64_t)v + c];
                for (int a = 0; a < 3; ++a) {
                    X12[3 + 3 * a + c] = xm0[3 * (int64_t)M[a] + c];
                    P12[3 + 3 * a + c] = dxm ? dxm[3 * (int64_t)M[a] + c] : 0.0;
                }
            }
            const double r = accd(0, X12, P12, P.ccd_slack, 1.0, P.ccd_max_iter, &it);
            ++n_pt; cap_hit |= it >= P.ccd_max_iter;
            best = dmin_(best, r);
        }
        for (int j = 0; j < 3; ++j) {
            const int32_t u = S.mtri_own_vert[3 * m + j];
            if (u < 0) continue;
            double ulo[3], uhi[3];
            swept_vert(xm0, dxm, u, ulo, uhi);
            if (!overlap(ulo, uhi, tlo, thi)) continue;
            for (int c = 0; c < 3; ++c) {
                X12[c] = xm0[3 * (int64_t)u + c]; P12[c] = dxm ? dxm[3 * (int64_t)u + c] : 0.0;
                for (int a = 0; a < 3; ++a) {
                    X12[3 + 3 * a + c] = x[3 * (int64_t)T[a] + c];
                    P12[3 + 3 * a + c] = dx[3 * (int64_t)T[a] + c];
                }
            }
            const double r = accd(0, X12, P12, P.ccd_slack, 1.0, P.ccd_max_iter, &it);
            ++n_pt; cap_hit |= it >= P.ccd_max_iter;
            best = dmin_(best, r);
        }
        for (int j = 0; j < 3; ++j) {
            const int32_t es = S.stri_own_edge[3 * t + j];
            if (es < 0) continue;
            const int32_t sa = S.sedge[2 * (int64_t)es], sb = S.sedge[2 * (int64_t)es + 1];
            double alo[3], ahi[3], l2[3], h2[3];
            swept_vert(x, dx, sa, alo, ahi);
            swept_vert(x, dx, sb, l2, h2);
            grow_box(alo, ahi, l2, h2);
            for (int q = 0; q < 3; ++q) {
                const int32_t em = S.mtri_own_edge[3 * m + q];
                if (em < 0) continue;
                const int32_t m0 = S.medge[2 * (int64_t)em], m1 = S.medge[2 * (int64_t)em + 1];
                double blo[3], bhi[3];
                swept_vert(xm0, dxm, m0, blo, bhi);
                swept_vert(xm0, dxm, m1, l2, h2);
                grow_box(blo, bhi, l2, h2);
                if (!overlap(alo, ahi, blo, bhi)) continue;
                for (int c = 0; c < 3; ++c) {
                    X12[c] = x[3 * (int64_t)sa + c]; P12[c] = dx[3 * (int64_t)sa + c];
                    X12[3 + c] = x[3 * (int64_t)sb + c]; P12[3 + c] = dx[3 * (int64_t)sb + c];
                    X12[6 + c] = xm0[3 * (int64_t)m0 + c]; P12[6 + c] = dxm ? dxm[3 * (int64_t)m0 + c] : 0.0;
                    X12[9 + c] = xm0[3 * (int64_t)m1 + c]; P12[9 + c] = dxm ? dxm[3 * (int64_t)m1 + c] : 0.0;
                }
                const double r = accd(1, X12, P12, P.ccd_slack, 1.0, P.ccd_max_iter, &it);
                ++n_ee; cap_hit |= it >= P.ccd_max_iter;
                best = dmin_(best, r);
            }
        }
    }
    if (best < 1.0) atomic_min_pos(alpha_bits, best);
    if (n_pt) atomic_add_ll(&counters[0], n_pt);
    if (n_ee) atomic_add_ll(&counters[1], n_ee);
    if (cap_hit) atomicMax(&counters[2], 1LL);
}

// Device address of g_accd_scratch on the current device.  The array's name
// is only a host-side stand-in, so the address is looked up with the device
// current, on every call: it is not cached, because a context torn down and
// made again on the device (cudaDeviceReset) may place the module elsewhere.
// Once the module is loaded the lookup allocates nothing.
cudaError_t noalloc_scratch(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_accd_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace gmcp

extern "C" ipc_status ipc_accd_min_noalloc(ipc_ctx* h, const double* x_dev, const double* dx_dev,
                                           const double* xm0_dev, const double* xm1_dev,
                                           double* alpha_accd_host, int64_t* n_pairs_host,
                                           int32_t* iter_cap_hit_host) {
    using namespace gmcp;
    if (!h) return IPC_ERR_ARG;
    Ctx& c = ctx_of(h);
    if (!x_dev || !dx_dev || (!xm0_dev && c.nmv > 0) || !alpha_accd_host) {
        c.err = "ipc_accd_min_noalloc: NULL argument";
        return IPC_ERR_ARG;
    }
    if (xm1_dev && c.nmv > kNoAllocMaxMasterVerts) {
        c.err = "ipc_accd_min_noalloc: a moving master needs 24 bytes per master vertex of the "
                "4 MiB built-in scratch, so at most " + std::to_string(kNoAllocMaxMasterVerts) +
                " master vertices; this scene has " + std::to_string(c.nmv);
        return IPC_ERR_CAPACITY;
    }
    auto fail = [&](cudaError_t e, const char* where) {
        cudaGetLastError();
        c.err = std::string("ipc_accd_min_noalloc: ") + where + ": " + cudaGetErrorString(e);
        return IPC_ERR_CUDA;
    };
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
    void* base = nullptr;
    e = noalloc_scratch(&base);
    if (e != cudaSuccess) return fail(e, "cudaGetSymbolAddress");
    unsigned long long* hdr = reinterpret_cast<unsigned long long*>(base);
    long long* counters = reinterpret_cast<long long*>(hdr + 1);
    double* dxm = nullptr;
    k_noalloc_reset<<<1, 1, 0, c.stream>>>(hdr);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "reset");
    if (xm1_dev && c.nmv > 0) {
        dxm = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(base) + kNoAllocHeaderBytes);
        const int64_t n = 3 * c.nmv;
        k_noalloc_sub<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(xm1_dev, xm0_dev, dxm, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "master displacement");
    }
    if (c.ns > 0 && c.nmt > 0) {
        const int m_chunk = 2048;
        dim3 grid((unsigned)((c.ns + 127) / 128), (unsigned)((c.nmt + m_chunk - 1) / m_chunk));
        k_accd_brute<<<grid, 128, 0, c.stream>>>(c.view(), c.P, x_dev, dx_dev, xm0_dev, dxm, m_chunk,
                                                 hdr, counters);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "k_accd_brute");
    }
    // the context's pinned host words (allocated when the context was made)
    e = cudaMemcpyAsync(c.h_counts + 8, hdr, 4 * sizeof(long long), cudaMemcpyDeviceToHost, c.stream);
    if (e != cudaSuccess) return fail(e, "copy back");
    e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return fail(e, "synchronise");
    double a;
    memcpy(&a, c.h_counts + 8, sizeof(double));
    *alpha_accd_host = a;
    if (n_pairs_host) { n_pairs_host[0] = c.h_counts[9]; n_pairs_host[1] = c.h_counts[10]; }
    if (iter_cap_hit_host) *iter_cap_hit_host = c.h_counts[11] != 0;
    return IPC_OK;
}

// dualmap.cu -- the dual-mesh mapper of Sec. 3.2 (Eqs. bary_proj, decomp,
// gram, bary_interp): visual vertices embedded on the simulation surface
// once, then carried along by the deformed simulation triangles every frame.
//
// Precomputation (ipc_dual_map_build): the nearest simulation triangle of
// every visual vertex, found through a uniform grid of the triangles' boxes
// searched in growing shells of cells around the point's cell, with exact
// FP64 point-triangle distances (ties go to the lowest triangle index, so the
// result does not depend on the grid); then (u, v, w) of the projection onto
// the triangle's plane from the 2x2 Gram system and the signed offset delta.
// Per frame (ipc_dual_map_apply): p' = u v0' + v v1' + w v2' + delta n'.
#include <algorithm>
#include <cmath>
#include <string>

#include "gmcp_internal.cuh"

namespace gmcp {
}

namespace {

using gmcp::DBuf;

constexpr int kThreads = 256;
constexpr int64_t kMaxCells = (int64_t)1 << 22;
unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 ld3(const double* P, int64_t i) { return {P[3 * i], P[3 * i + 1], P[3 * i + 2]}; }
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 axpy(D3 a, double s, D3 b) { return {a.x + s * b.x, a.y + s * b.y, a.z + s * b.z}; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm2(D3 a) { return dot(a, a); }

// squared distance from p to segment [a, b]
__device__ double seg_d2(D3 p, D3 a, D3 b) {
    const D3 ab = sub(b, a);
    const double l2 = norm2(ab);
    double t = l2 > 0.0 ? dot(sub(p, a), ab) / l2 : 0.0;
    t = fmin(1.0, fmax(0.0, t));
    return norm2(sub(p, axpy(a, t, ab)));
}

// Squared distance from p to triangle (a, b, c): the closest point lies in
// one of seven Voronoi regions (three vertices, three edges, the face); the
// region follows from the signs of the dot products of p - a, p - b, p - c
// with the edges ab, ac (Ericson, Real-Time Collision Detection, Sec. 5.1.5).
// A degenerate triangle falls back to its three edges.
__device__ double pt_tri_d2(D3 p, D3 a, D3 b, D3 c) {
    const D3 ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
    const double d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) return norm2(ap);
    const D3 bp = sub(p, b);
    const double d3 = dot(ab, bp), d4 = dot(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) return norm2(bp);
    const double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) return norm2(sub(p, axpy(a, d1 / (d1 - d3), ab)));
    const D3 cp = sub(p, c);
    const double d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) return norm2(cp);
    const double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) return norm2(sub(p, axpy(a, d2 / (d2 - d6), ac)));
    const double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0)
        return norm2(sub(p, axpy(b, (d4 - d3) / ((d4 - d3) + (d5 - d6)), sub(c, b))));
    const double den = va + vb + vc;
    if (!(den > 0.0))
        return fmin(seg_d2(p, a, b), fmin(seg_d2(p, a, c), seg_d2(p, b, c)));
    const double v = vb / den, w = vc / den;
    return norm2(sub(p, axpy(axpy(a, v, ab), w, ac)));
}

// flag[0] = 1 if some triangle index is outside [0, nv)
__global__ void k_dm_check(const int32_t* __restrict__ T, int64_t n3, int64_t nv, int32_t* __restrict__ flag) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n3 && (T[k] < 0 || T[k] >= nv)) flag[0] = 1;
}

// per-block min / max of the triangles' boxes and the sum of their largest
// extents (partials [blocks][7], reduced by one block afterwards)
__global__ void k_dm_box_partial(const double* __restrict__ V, const int32_t* __restrict__ T, int64_t nt,
                                 double* __restrict__ part) {
    __shared__ double sh[7][kThreads];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, ext = 0.0;
    if (t < nt) {
        for (int k = 0; k < 3; ++k) {
            const D3 v = ld3(V, T[3 * t + k]);
            lo[0] = fmin(lo[0], v.x); lo[1] = fmin(lo[1], v.y); lo[2] = fmin(lo[2], v.z);
            hi[0] = fmax(hi[0], v.x); hi[1] = fmax(hi[1], v.y); hi[2] = fmax(hi[2], v.z);
        }
        ext = fmax(hi[0] - lo[0], fmax(hi[1] - lo[1], hi[2] - lo[2]));
    }
    for (int c = 0; c < 3; ++c) { sh[c][threadIdx.x] = lo[c]; sh[3 + c][threadIdx.x] = hi[c]; }
    sh[6][threadIdx.x] = ext;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            for (int c = 0; c < 3; ++c) {
                sh[c][threadIdx.x] = fmin(sh[c][threadIdx.x], sh[c][threadIdx.x + s]);
                sh[3 + c][threadIdx.x] = fmax(sh[3 + c][threadIdx.x], sh[3 + c][threadIdx.x + s]);
            }
            sh[6][threadIdx.x] += sh[6][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) part[7 * (int64_t)blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_dm_box_final(const double* __restrict__ part, int64_t nparts, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double r[7] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
    for (int64_t b = 0; b < nparts; ++b) {
        for (int c = 0; c < 3; ++c) {
            r[c] = fmin(r[c], part[7 * b + c]);
            r[3 + c] = fmax(r[3 + c], part[7 * b + 3 + c]);
        }
        r[6] += part[7 * b + 6];
    }
    for (int c = 0; c < 7; ++c) out[c] = r[c];
}

struct Grid {
    double org[3];
    double h, inv;
    int dim[3];
};

__device__ __forceinline__ int cell_of(double x, double org, double inv, int dim) {
    const double u = (x - org) * inv;
    if (!(u >= 0.0)) return 0;
    if (u >= (double)(dim - 1)) return dim - 1;
    return (int)u;
}
__device__ __forceinline__ int64_t cell_id(const Grid& G, int ix, int iy, int iz) {
    return ((int64_t)iz * G.dim[1] + iy) * G.dim[0] + ix;
}

// cell range of triangle t's box
__device__ __forceinline__ void tri_cells(const Grid& G, const double* V, const int32_t* T, int64_t t, int* a,
                                          int* b) {
    const D3 v0 = ld3(V, T[3 * t]), v1 = ld3(V, T[3 * t + 1]), v2 = ld3(V, T[3 * t + 2]);
    const double lo[3] = {fmin(v0.x, fmin(v1.x, v2.x)), fmin(v0.y, fmin(v1.y, v2.y)), fmin(v0.z, fmin(v1.z, v2.z))};
    const double hi[3] = {fmax(v0.x, fmax(v1.x, v2.x)), fmax(v0.y, fmax(v1.y, v2.y)), fmax(v0.z, fmax(v1.z, v2.z))};
    for (int c = 0; c < 3; ++c) {
        a[c] = cell_of(lo[c], G.org[c], G.inv, G.dim[c]);
        b[c] = cell_of(hi[c], G.org[c], G.inv, G.dim[c]);
    }
}

__global__ void k_dm_count(Grid G, const double* __restrict__ V, const int32_t* __restrict__ T, int64_t nt,
                           int32_t* __restrict__ cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int a[3], b[3];
    tri_cells(G, V, T, t, a, b);
    for (int iz = a[2]; iz <= b[2]; ++iz)
        for (int iy = a[1]; iy <= b[1]; ++iy)
            for (int ix = a[0]; ix <= b[0]; ++ix) atomicAdd(&cnt[cell_id(G, ix, iy, iz)], 1);
}

__global__ void k_dm_fill(Grid G, const double* __restrict__ V, const int32_t* __restrict__ T, int64_t nt,
                          int32_t* __restrict__ cur, int32_t* __restrict__ ent) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int a[3], b[3];
    tri_cells(G, V, T, t, a, b);
    for (int iz = a[2]; iz <= b[2]; ++iz)
        for (int iy = a[1]; iy <= b[1]; ++iy)
            for (int ix = a[0]; ix <= b[0]; ++ix) ent[atomicAdd(&cur[cell_id(G, ix, iy, iz)], 1)] = (int32_t)t;
}

// (u, v, w, delta) of p on triangle (v0, v1, v2), Eqs. (decomp) and (gram)
__device__ void coords(D3 p, D3 v0, D3 v1, D3 v2, double* out) {
    const D3 e1 = sub(v1, v0), e2 = sub(v2, v0), d = sub(p, v0);
    D3 n = cross(e1, e2);
    const double len = sqrt(norm2(n));
    n = {n.x / len, n.y / len, n.z / len};
    const double g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
    const double r1 = dot(d, e1), r2 = dot(d, e2);
    const double det = g11 * g22 - g12 * g12;
    const double v = (r1 * g22 - g12 * r2) / det;
    const double w = (g11 * r2 - g12 * r1) / det;
    out[0] = 1.0 - v - w;
    out[1] = v;
    out[2] = w;
    out[3] = dot(d, n);
}

// Nearest triangle of every visual vertex: shells of cells at Chebyshev
// radius r = 0, 1, ... around the point's (clamped) cell.  A triangle not
// met so far lies in no searched cell, so its box, and the triangle, lies
// outside the searched block of cells: the search stops once the best
// distance is below the distance from p to the open faces of that block
// (faces on the grid boundary are closed: no box reaches past them), less a
// margin for the rounding of cell indices, or once the block is the grid.
__global__ void k_dm_nearest(Grid G, const double* __restrict__ V, const int32_t* __restrict__ T,
                             const int32_t* __restrict__ start, const int32_t* __restrict__ ent,
                             const double* __restrict__ P, int64_t np, int32_t* __restrict__ tri_out,
                             double* __restrict__ uvwd_out, double* __restrict__ d2_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const D3 p = ld3(P, i);
    const double pc[3] = {p.x, p.y, p.z};
    int c0[3];
    for (int c = 0; c < 3; ++c) c0[c] = cell_of(pc[c], G.org[c], G.inv, G.dim[c]);
    double best = INFINITY;
    int32_t bt = -1;
    const int rmax = max(G.dim[0], max(G.dim[1], G.dim[2]));
    for (int r = 0; r <= rmax; ++r) {
        int lo[3], hi[3];
        for (int c = 0; c < 3; ++c) { lo[c] = max(0, c0[c] - r); hi[c] = min(G.dim[c] - 1, c0[c] + r); }
        for (int iz = lo[2]; iz <= hi[2]; ++iz)
            for (int iy = lo[1]; iy <= hi[1]; ++iy)
                for (int ix = lo[0]; ix <= hi[0]; ++ix) {
                    const int ch = max(abs(ix - c0[0]), max(abs(iy - c0[1]), abs(iz - c0[2])));
                    if (ch != r) continue;   // inner cells were searched before
                    const int64_t cell = cell_id(G, ix, iy, iz);
                    for (int e = start[cell]; e < start[cell + 1]; ++e) {
                        const int32_t t = ent[e];
                        const double d2 = pt_tri_d2(p, ld3(V, T[3 * t]), ld3(V, T[3 * t + 1]), ld3(V, T[3 * t + 2]));
                        if (d2 < best || (d2 == best && t < bt)) { best = d2; bt = t; }
                    }
                }
        double lb = INFINITY;
        bool open = false;
        for (int c = 0; c < 3; ++c) {
            if (lo[c] > 0) { open = true; lb = fmin(lb, pc[c] - (G.org[c] + lo[c] * G.h)); }
            if (hi[c] < G.dim[c] - 1) { open = true; lb = fmin(lb, (G.org[c] + (hi[c] + 1) * G.h) - pc[c]); }
        }
        if (!open) break;
        lb -= 1e-6 * G.h;
        if (bt >= 0 && lb > 0.0 && best <= lb * lb) break;
    }
    tri_out[i] = bt;
    if (d2_out) d2_out[i] = best;
    double c4[4] = {NAN, NAN, NAN, NAN};
    if (bt >= 0) coords(p, ld3(V, T[3 * bt]), ld3(V, T[3 * bt + 1]), ld3(V, T[3 * bt + 2]), c4);
    for (int c = 0; c < 4; ++c) uvwd_out[4 * i + c] = c4[c];
}

// p' = u v0' + v v1' + w v2' + delta n', Eq. (bary_interp)
// (a triangle index outside [0, nt) gives NaN; vertex indices were checked
// by the build)
__global__ void k_dm_apply(const double* __restrict__ V, const int32_t* __restrict__ T, int64_t nt,
                           const int32_t* __restrict__ tri, const double* __restrict__ uvwd, int64_t np,
                           double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int64_t t = __ldg(tri + i);
    if (t < 0 || t >= nt) {
        out[3 * i] = out[3 * i + 1] = out[3 * i + 2] = NAN;
        return;
    }
    const double2 uv = __ldg(reinterpret_cast<const double2*>(uvwd) + 2 * i);   // (u, v); u is implied
    const double2 wd = __ldg(reinterpret_cast<const double2*>(uvwd) + 2 * i + 1);
    const D3 v0 = ld3(V, __ldg(T + 3 * t)), v1 = ld3(V, __ldg(T + 3 * t + 1)), v2 = ld3(V, __ldg(T + 3 * t + 2));
    // the same point written as v0 + v e1 + w e2 + delta n (u = 1 - v - w),
    // reusing the edges of the normal: fewer FP64 operations, the kernel's
    // bound on this part
    const D3 e1 = sub(v1, v0), e2 = sub(v2, v0);
    const D3 n = cross(e1, e2);
    const double s = wd.y * rsqrt(norm2(n));
    out[3 * i] = v0.x + uv.y * e1.x + wd.x * e2.x + s * n.x;
    out[3 * i + 1] = v0.y + uv.y * e1.y + wd.x * e2.y + s * n.y;
    out[3 * i + 2] = v0.z + uv.y * e1.z + wd.x * e2.z + s * n.z;
}

ipc_status dm_fail(ipc_status st, const std::string& msg) {
    gmcp::set_global_error(msg);
    return st;
}
ipc_status dm_cuda(cudaError_t e, const char* where) {
    return dm_fail(e == cudaErrorMemoryAllocation ? IPC_ERR_OOM : IPC_ERR_CUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

#define DM_TRY(expr, where)                          \
    do {                                             \
        cudaError_t _e = (expr);                     \
        if (_e != cudaSuccess) return dm_cuda(_e, where); \
    } while (0)

}  // namespace

extern "C" {

ipc_status ipc_dual_map_build(const double* V_dev, int64_t nv, const int32_t* T_dev, int64_t nt,
                              const double* P_dev, int64_t np, int32_t* tri_dev, double* uvwd_dev,
                              double* dist2_dev, void* stream) {
    if (!V_dev || !T_dev || nv <= 0 || nt <= 0 || np < 0 || (np > 0 && (!P_dev || !tri_dev || !uvwd_dev)))
        return dm_fail(IPC_ERR_ARG, "ipc_dual_map_build: NULL pointer or empty mesh");
    if (nt >= ((int64_t)1 << 31) || np >= ((int64_t)1 << 40))
        return dm_fail(IPC_ERR_ARG, "ipc_dual_map_build: too many triangles");
    if (np == 0) return IPC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DM_TRY(cudaGetLastError(), "ipc_dual_map_build");
    {
        DBuf<int32_t> flag;
        DM_TRY(flag.alloc(1), "ipc_dual_map_build");
        DM_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int32_t), s), "ipc_dual_map_build");
        k_dm_check<<<nb(3 * nt, kThreads), kThreads, 0, s>>>(T_dev, 3 * nt, nv, flag.p);
        int32_t bad = 0;
        DM_TRY(cudaMemcpyAsync(&bad, flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "ipc_dual_map_build");
        DM_TRY(cudaStreamSynchronize(s), "ipc_dual_map_build");
        if (bad) return dm_fail(IPC_ERR_ARG, "ipc_dual_map_build: triangle index outside [0, nv)");
    }
    // bounding box and mean extent of the triangles
    const unsigned nbt = nb(nt, kThreads);
    DBuf<double> part, box;
    DM_TRY(part.alloc(7 * (size_t)nbt), "ipc_dual_map_build");
    DM_TRY(box.alloc(7), "ipc_dual_map_build");
    k_dm_box_partial<<<nbt, kThreads, 0, s>>>(V_dev, T_dev, nt, part.p);
    k_dm_box_final<<<1, 32, 0, s>>>(part.p, nbt, box.p);
    DM_TRY(cudaGetLastError(), "ipc_dual_map_build");
    double hb[7];
    DM_TRY(cudaMemcpyAsync(hb, box.p, sizeof(hb), cudaMemcpyDeviceToHost, s), "ipc_dual_map_build");
    DM_TRY(cudaStreamSynchronize(s), "ipc_dual_map_build");
    for (int c = 0; c < 6; ++c)
        if (!std::isfinite(hb[c])) return dm_fail(IPC_ERR_ARG, "ipc_dual_map_build: non-finite vertex");
    // cells about the mean triangle extent, at most kMaxCells in all
    Grid G;
    double L[3], Lmax = 0.0;
    for (int c = 0; c < 3; ++c) { L[c] = hb[3 + c] - hb[c]; Lmax = std::max(Lmax, L[c]); }
    double h = hb[6] / (double)nt;
    if (!(h > 0.0)) h = Lmax > 0.0 ? Lmax : 1.0;
    for (;;) {
        int64_t cells = 1;
        for (int c = 0; c < 3; ++c) cells *= (int64_t)std::floor(L[c] / h) + 1;
        if (cells <= kMaxCells) break;
        h *= 1.25;
    }
    for (int c = 0; c < 3; ++c) {
        G.org[c] = hb[c];
        G.dim[c] = (int)std::floor(L[c] / h) + 1;
    }
    G.h = h;
    G.inv = 1.0 / h;
    const int64_t ncell = (int64_t)G.dim[0] * G.dim[1] * G.dim[2];
    DBuf<int32_t> cnt, start, cur, tmp, ent;
    DM_TRY(cnt.alloc((size_t)ncell + 1), "ipc_dual_map_build");
    DM_TRY(start.alloc((size_t)ncell + 2), "ipc_dual_map_build");
    DM_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (ncell + 1), s), "ipc_dual_map_build");
    const size_t ntmp = 2 * gmcp::scan_tmp_size(ncell);
    DM_TRY(tmp.alloc(ntmp), "ipc_dual_map_build");
    k_dm_count<<<nbt, kThreads, 0, s>>>(G, V_dev, T_dev, nt, cnt.p);
    DM_TRY(cudaGetLastError(), "ipc_dual_map_build");
    DM_TRY(gmcp::exclusive_scan_i32(cnt.p, start.p, ncell, tmp.p, ntmp, s), "ipc_dual_map_build");
    int32_t total = 0;
    DM_TRY(cudaMemcpyAsync(&total, start.p + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
           "ipc_dual_map_build");
    DM_TRY(cudaStreamSynchronize(s), "ipc_dual_map_build");
    if (total < 0) return dm_fail(IPC_ERR_CAPACITY, "ipc_dual_map_build: too many cell entries");
    DM_TRY(ent.alloc((size_t)total + 1), "ipc_dual_map_build");
    DM_TRY(cur.alloc((size_t)ncell + 1), "ipc_dual_map_build");
    DM_TRY(cudaMemcpyAsync(cur.p, start.p, sizeof(int32_t) * ncell, cudaMemcpyDeviceToDevice, s),
           "ipc_dual_map_build");
    k_dm_fill<<<nbt, kThreads, 0, s>>>(G, V_dev, T_dev, nt, cur.p, ent.p);
    k_dm_nearest<<<nb(np, kThreads), kThreads, 0, s>>>(G, V_dev, T_dev, start.p, ent.p, P_dev, np, tri_dev,
                                                       uvwd_dev, dist2_dev);
    DM_TRY(cudaGetLastError(), "ipc_dual_map_build");
    DM_TRY(cudaStreamSynchronize(s), "ipc_dual_map_build");   // the scratch buffers are freed on return
    return IPC_OK;
}

ipc_status ipc_dual_map_apply(const double* V_dev, const int32_t* T_dev, int64_t nt, const int32_t* tri_dev,
                              const double* uvwd_dev, int64_t np, double* out_dev, void* stream) {
    if (np < 0 || (np > 0 && (!V_dev || !T_dev || !tri_dev || !uvwd_dev || !out_dev)))
        return dm_fail(IPC_ERR_ARG, "ipc_dual_map_apply: NULL pointer");
    if (np == 0) return IPC_OK;
    if ((reinterpret_cast<uintptr_t>(uvwd_dev) & 15) != 0)
        return dm_fail(IPC_ERR_ARG, "ipc_dual_map_apply: uvwd_dev must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    k_dm_apply<<<nb(np, kThreads), kThreads, 0, s>>>(V_dev, T_dev, nt, tri_dev, uvwd_dev, np, out_dev);
    DM_TRY(cudaGetLastError(), "ipc_dual_map_apply");
    return IPC_OK;
}

}  // extern "C"

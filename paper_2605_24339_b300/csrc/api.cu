// api.cu -- the C ABI of libgmcp (declared in include/gmcp.h): context
// creation (derived topology built on the host and uploaded once), and the
// entry points that queue the contact-pass kernels on the caller's stream.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "gmcp_internal.cuh"

namespace gmcp {

SceneView Ctx::view() const {
    SceneView S;
    S.nv = (int32_t)nv; S.ns = (int32_t)ns; S.nmv = (int32_t)nmv; S.nmt = (int32_t)nmt;
    S.nme = (int32_t)nme; S.nse = (int32_t)nse; S.n_env = n_env;
    S.stri = stri.p; S.mtri = mtri.p; S.medge = medge.p;
    S.me_tri_off = me_tri_off.p; S.me_tri = me_tri.p; S.mv_tri_off = mv_tri_off.p; S.mv_tri = mv_tri.p;
    S.mtri_own_edge = mtri_own_edge.p; S.mtri_own_vert = mtri_own_vert.p;
    S.stri_own_vert = stri_own_vert.p; S.stri_own_edge = stri_own_edge.p; S.sedge = sedge.p;
    S.stri_env = stri_env.p; S.mtri_env = mtri_env.p; S.mvert_env = mvert_env.p;
    S.X = X.p; S.Y0 = Y0.p; S.srest_box = srest_box.p; S.mrest_box = mrest_box.p;
    S.srest_box_f = srest_box_f.p; S.mrest_box_f = mrest_box_f.p; S.mvrest_box_f = mvrest_box_f.p;
    S.grid_org = grid_org.p; S.grid_inv = grid_inv.p; S.grid_dim = grid_dim.p; S.grid_off = grid_off.p;
    S.grid_org_f = grid_org_f.p; S.grid_inv_f = grid_inv_f.p;
    S.margin = margin;
    return S;
}

namespace {

thread_local std::string g_create_error;

struct Fail {
    ipc_status st;
    std::string msg;
};

#define CK(expr)                                                                              \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess)                                                                \
            throw Fail{_e == cudaErrorMemoryAllocation ? IPC_ERR_OOM : IPC_ERR_CUDA,          \
                       std::string(#expr) + ": " + cudaGetErrorString(_e)};                   \
    } while (0)

int32_t env_of(const std::vector<int64_t>& off, int64_t i) {
    auto it = std::upper_bound(off.begin(), off.end(), i);
    return (int32_t)(it - off.begin()) - 1;
}

// unique undirected edges of a triangle list, sorted lexicographically by
// (min, max) vertex; off/adj: CSR of the triangles adjacent to each edge,
// in increasing triangle id
void tri_edges(const int32_t* tris, int64_t n, std::vector<int32_t>& edges,
               std::vector<int32_t>& off, std::vector<int32_t>& adj) {
    // every (min vertex, max vertex, tri) triple, in lexicographic order:
    // bucketed by the min vertex (counting sort), each bucket sorted by (max
    // vertex, tri); buckets are short (the vertex's incident edges)
    int32_t nvert = 0;
    for (int64_t i = 0; i < 3 * n; ++i) nvert = std::max(nvert, tris[i] + 1);
    std::vector<int64_t> boff((size_t)nvert + 1, 0);
    for (int64_t t = 0; t < n; ++t)
        for (int k = 0; k < 3; ++k) boff[(size_t)std::min(tris[3 * t + k], tris[3 * t + (k + 1) % 3]) + 1]++;
    for (int32_t v = 0; v < nvert; ++v) boff[v + 1] += boff[v];
    std::vector<std::pair<int32_t, int32_t>> tr((size_t)n * 3);   // (max vertex, tri)
    {
        std::vector<int64_t> cur(boff.begin(), boff.end() - 1);
        for (int64_t t = 0; t < n; ++t)
            for (int k = 0; k < 3; ++k) {
                const int32_t a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
                tr[(size_t)cur[std::min(a, b)]++] = {std::max(a, b), (int32_t)t};
            }
    }
    edges.clear(); off.clear(); adj.clear();
    adj.reserve(tr.size());
    for (int32_t v = 0; v < nvert; ++v) {
        std::sort(tr.begin() + boff[v], tr.begin() + boff[v + 1]);
        for (int64_t i = boff[v]; i < boff[v + 1]; ++i) {
            if (i == boff[v] || tr[i].first != tr[i - 1].first) {
                edges.push_back(v); edges.push_back(tr[i].first);
                off.push_back((int32_t)adj.size());
            }
            adj.push_back(tr[i].second);
        }
    }
    off.push_back((int32_t)adj.size());
}

__global__ void k_count_sum(const int32_t* __restrict__ cnt, int64_t ns, long long* out) {
    pass_dep_wait();
    // out[0..2] = totals per kind, out[3..5] = maxima
    long long s0 = 0, s1 = 0, s2 = 0;
    int m0 = 0, m1 = 0, m2 = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ns;
         t += (int64_t)gridDim.x * blockDim.x) {
        s0 += cnt[4 * t]; s1 += cnt[4 * t + 1]; s2 += cnt[4 * t + 2];
        m0 = max(m0, cnt[4 * t]); m1 = max(m1, cnt[4 * t + 1]); m2 = max(m2, cnt[4 * t + 2]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o); s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, o)); m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = max(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_add_ll(&out[0], s0); atomic_add_ll(&out[1], s1); atomic_add_ll(&out[2], s2);
        atomicMax(&out[3], (long long)m0); atomicMax(&out[4], (long long)m1); atomicMax(&out[5], (long long)m2);
    }
}

// x[svert[k]] = xs[k] for the slave vertices (ipc_scatter_slave)
__global__ void k_scatter_slave(const int32_t* __restrict__ svert, int64_t n, const double* __restrict__ xs,
                                double* __restrict__ x) {
    pass_dep_wait();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t v = svert[k];
    x[3 * v] = xs[3 * k];
    x[3 * v + 1] = xs[3 * k + 1];
    x[3 * v + 2] = xs[3 * k + 2];
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ o, int64_t n) {
    pass_dep_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = a[i] - b[i];
}

}  // namespace

cudaError_t grow_candidates(Ctx& c, int32_t need_f, int32_t need_e, int32_t need_p);

// Broad phase with automatic regrowth of the per-triangle capacities.
cudaError_t run_candidates(Ctx& c, const double* x, const double* xm, bool lazy) {
    if (lazy) {
        GMCP_CUDA_TRY(cudaMemsetAsync(c.misc_i32.p + 12, 0, 4 * sizeof(int32_t), c.stream));
        GMCP_CUDA_TRY(bp_build_grid(c, xm, nullptr, false, true));
        return bp_query_contact(c, x, xm, true);
    }
    for (int attempt = 0; attempt < 6; ++attempt) {
        GMCP_CUDA_TRY(bp_build_grid(c, xm, nullptr, false));
        GMCP_CUDA_TRY(bp_query_contact(c, x, xm));
        int32_t ov[4];
        GMCP_CUDA_TRY(cudaMemcpyAsync(ov, c.misc_i32.p, sizeof(ov), cudaMemcpyDeviceToHost, c.stream));
        GMCP_CUDA_TRY(cudaStreamSynchronize(c.stream));
        if (ov[1] == 0 && ov[2] == 0 && ov[3] == 0) return cudaSuccess;
        GMCP_CUDA_TRY(grow_candidates(c, ov[1], ov[2], ov[3]));
    }
    return cudaErrorInvalidValue;
}

cudaError_t grow_candidates(Ctx& c, int32_t need_f, int32_t need_e, int32_t need_p) {
    auto grow = [](int32_t cap, int32_t need) {
        int32_t v = cap;
        while (v < need) v *= 2;
        return v;
    };
    c.cap_f = grow(c.cap_f, need_f);
    c.cap_e = grow(c.cap_e, need_e);
    c.cap_p = grow(c.cap_p, need_p);
    GMCP_CUDA_TRY(c.cand_face.ensure((size_t)c.ns * c.cap_f + 1));
    GMCP_CUDA_TRY(c.cand_edge.ensure((size_t)c.ns * c.cap_e + 1));
    GMCP_CUDA_TRY(c.cand_point.ensure((size_t)c.ns * c.cap_p + 1));
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// the fused contact pass: one enqueue of all its work, captured as a CUDA
// graph for repeated calls with the same arguments
// ---------------------------------------------------------------------------
struct ContactPassArgs {
    const double *x, *xm0, *xm1, *dx;
    double* edev;
    void* grad;
    bool hess, counts, host_energy, want_alpha, lazy;
    // host inputs (ipc_contact_pass_host): the slave vertices' positions and
    // displacements in page-locked host memory, scattered into x and dx
    const double* xs_host = nullptr;
    const double* dxs_host = nullptr;
};

// Everything one pass queues (no synchronisation): the master displacement,
// the step bounds' initial values, the broad phase, samples and gathers, the
// step bounds, and (lazy) the copies of host-visible results and capacity
// flags into the pinned area.
cudaError_t enqueue_contact_pass(Ctx& c, const ContactPassArgs& A) {
    // host inputs: the slave vertices' positions are copied and scattered
    // first; their displacements follow on the copy stream (after the
    // positions on the bus) while the broad phase runs, and the two readers
    // of dx (the swept query and the sample evaluation) wait for them
    bool dx_wait = false;
    if (A.xs_host && c.n_svert > 0) {
        const size_t nb = sizeof(double) * 3 * (size_t)c.n_svert;
        const unsigned g = (unsigned)((c.n_svert + 255) / 256);
        GMCP_CUDA_TRY(cudaMemcpyAsync(c.xs_stage.p, A.xs_host, nb, cudaMemcpyHostToDevice, c.stream));
        if (A.dxs_host && A.dx) {
            GMCP_CUDA_TRY(cudaEventRecord(c.ev_xin, c.stream));
            GMCP_CUDA_TRY(cudaStreamWaitEvent(c.h2d_stream, c.ev_xin, 0));
            GMCP_CUDA_TRY(cudaMemcpyAsync(c.dxs_stage.p, A.dxs_host, nb, cudaMemcpyHostToDevice, c.h2d_stream));
            launch_dep(k_scatter_slave, g, 256, 0, c.h2d_stream, c.svert.p, c.n_svert, c.dxs_stage.p,
                                                         const_cast<double*>(A.dx));
            GMCP_CUDA_TRY(cudaGetLastError());
            GMCP_CUDA_TRY(cudaEventRecord(c.ev_dxin, c.h2d_stream));
            dx_wait = true;
        }
        launch_dep(k_scatter_slave, g, 256, 0, c.stream, c.svert.p, c.n_svert, c.xs_stage.p, const_cast<double*>(A.x));
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    const double* dxm = nullptr;
    if (A.dx && A.xm1) {
        GMCP_CUDA_TRY(c.dxm.ensure(3 * (size_t)c.nmv + 3));
        const int64_t n = 3 * c.nmv;
        if (n > 0) {
            launch_dep(k_sub, (unsigned)((n + 255) / 256), 256, 0, c.stream, A.xm1, A.xm0, c.dxm.p, n);
            GMCP_CUDA_TRY(cudaGetLastError());
        }
        dxm = c.dxm.p;
    }
    if (A.dx) {
        GMCP_CUDA_TRY(cudaMemcpyAsync(c.u64_tmp.p, c.pin->init, 2 * sizeof(unsigned long long),
                                      cudaMemcpyHostToDevice, c.stream));
        GMCP_CUDA_TRY(cudaMemsetAsync(c.i64_tmp.p + 8, 0, 4 * sizeof(long long), c.stream));
    }
    // mixed path: the master's FP32 tables depend on xm0 alone, so they are
    // built on the side stream beside the broad phase
    struct PreFlag { bool& f; ~PreFlag() { f = false; } } pre_flag{c.master_pre};
    if (c.P.precision == IPC_PREC_MIXED && c.nmv > 0 && !c.prof.on && !c.P.face_clip) {
        if (!c.aux_stream) GMCP_CUDA_TRY(cudaStreamCreateWithFlags(&c.aux_stream, cudaStreamNonBlocking));
        if (!c.ev_mfork) GMCP_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_mfork, cudaEventDisableTiming));
        if (!c.ev_master) GMCP_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_master, cudaEventDisableTiming));
        GMCP_CUDA_TRY(cudaEventRecord(c.ev_mfork, c.stream));
        GMCP_CUDA_TRY(cudaStreamWaitEvent(c.aux_stream, c.ev_mfork, 0));
        GMCP_CUDA_TRY(master_tables(c, A.xm0, c.aux_stream));
        GMCP_CUDA_TRY(cudaEventRecord(c.ev_master, c.aux_stream));
        c.master_pre = true;
    }
    GMCP_CUDA_TRY(run_candidates(c, A.x, A.xm0, A.lazy));
    // With a static master the swept query reads the same grid and nothing
    // else of the contact evaluation: it runs on a second stream, forked
    // after the grid build and joined before the results are read (the
    // profiler keeps one stream so that its sections stay separate).
    const bool fork = A.dx && !dxm && A.lazy && !c.prof.on;
    if (fork) {
        if (!c.ccd_stream) GMCP_CUDA_TRY(cudaStreamCreateWithFlags(&c.ccd_stream, cudaStreamNonBlocking));
        if (!c.ev_fork) GMCP_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
        if (!c.ev_join) GMCP_CUDA_TRY(cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
        GMCP_CUDA_TRY(cudaEventRecord(c.ev_fork, c.stream));
        GMCP_CUDA_TRY(cudaStreamWaitEvent(c.ccd_stream, c.ev_fork, 0));
        if (dx_wait) GMCP_CUDA_TRY(cudaStreamWaitEvent(c.ccd_stream, c.ev_dxin, 0));
        cudaStream_t main = c.stream;
        c.stream = c.ccd_stream;
        const cudaError_t e = bp_ccd_accd(c, A.x, A.dx, A.xm0, dxm, c.u64_tmp.p + 1, c.i64_tmp.p + 8, true, true);
        c.stream = main;
        GMCP_CUDA_TRY(e);
        GMCP_CUDA_TRY(cudaEventRecord(c.ev_join, c.ccd_stream));
    }
    long long* ctr = nullptr;
    if (A.counts) {
        GMCP_CUDA_TRY(cudaMemsetAsync(c.i64_tmp.p, 0, 8 * sizeof(long long), c.stream));
        ctr = c.i64_tmp.p;
    }
    if (dx_wait) GMCP_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.ev_dxin, 0));
    GMCP_CUDA_TRY(contact_eval(c, A.x, A.xm0, A.edev, A.grad, A.hess, ctr, A.dx, dxm,
                               A.dx ? c.u64_tmp.p : nullptr));
    if (fork)
        GMCP_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.ev_join, 0));
    else if (A.dx)
        GMCP_CUDA_TRY(bp_ccd_accd(c, A.x, A.dx, A.xm0, dxm, c.u64_tmp.p + 1, c.i64_tmp.p + 8, true, A.lazy));
    if (!A.lazy) return cudaSuccess;
    if (A.host_energy)
        GMCP_CUDA_TRY(cudaMemcpyAsync(&c.pin->energy, A.edev, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (A.counts)
        GMCP_CUDA_TRY(cudaMemcpyAsync(c.pin->counts, c.i64_tmp.p, 4 * sizeof(long long), cudaMemcpyDeviceToHost, c.stream));
    if (A.want_alpha) {
        GMCP_CUDA_TRY(cudaMemcpyAsync(c.pin->bits, c.u64_tmp.p, 2 * sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, c.stream));
        GMCP_CUDA_TRY(cudaMemcpyAsync(c.pin->ctr_ccd, c.i64_tmp.p + 8, 4 * sizeof(long long),
                                      cudaMemcpyDeviceToHost, c.stream));
    }
    return cudaMemcpyAsync(c.pin->flags, c.misc_i32.p, 32 * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream);
}

// capacity flags of the last lazy pass (valid after a synchronisation)
bool pass_overflowed(const Ctx& c) {
    const int32_t* f = c.pin->flags;
    return f[1] || f[2] || f[3] || f[12] || f[13] || f[14] || f[15];
}

// The sample items of the last lazy pass did not fit their buffer (the
// pass then took the warp-per-triangle kernel, with the same results):
// make room for the next passes.
cudaError_t grow_items(Ctx& c) {
    const int64_t need = c.pin->flags[16];
    if (need <= c.cap_items) return cudaSuccess;
    c.cap_items = need + need / 2;
    GMCP_CUDA_TRY(c.item_owner.ensure((size_t)c.cap_items));
    GMCP_CUDA_TRY(c.item_rd.ensure(2 * (size_t)c.cap_items));
    GMCP_CUDA_TRY(c.item_rt.ensure(5 * sizeof(double) * (size_t)c.cap_items));
    GMCP_CUDA_TRY(c.item_list.ensure((size_t)c.cap_items));
    GMCP_CUDA_TRY(c.item_mask.ensure((size_t)c.cap_items / 32 + 2));
    GMCP_CUDA_TRY(c.item_mid.ensure((size_t)c.cap_items));
    c.cp_graph.reset();
    return cudaSuccess;
}

cudaError_t grow_after_overflow(Ctx& c) {
    const int32_t* f = c.pin->flags;
    if (f[1] || f[2] || f[3]) GMCP_CUDA_TRY(grow_candidates(c, f[1], f[2], f[3]));
    if (f[12]) GMCP_CUDA_TRY(c.cell_ent.ensure(2 * c.cell_ent.n));
    if (f[13]) {
        c.cap_ccd = std::max(c.cap_ccd, f[13]);
        GMCP_CUDA_TRY(c.ccd_pairs.ensure((size_t)c.cap_ccd));
    }
    if (f[14]) {
        c.cap_coarse_swept = std::max(c.cap_coarse_swept, f[14]);
        GMCP_CUDA_TRY(c.coarse_swept.ensure((size_t)c.cap_coarse_swept));
    }
    if (f[15]) {
        c.cap_coarse = std::max(c.cap_coarse, f[15]);
        GMCP_CUDA_TRY(c.coarse_pairs.ensure((size_t)c.cap_coarse));
    }
    return cudaSuccess;
}

// the arguments and capacities a captured pass depends on
std::vector<uintptr_t> contact_pass_key(const Ctx& c, const ContactPassArgs& A) {
    return {(uintptr_t)A.x, (uintptr_t)A.xm0, (uintptr_t)A.xm1, (uintptr_t)A.dx, (uintptr_t)A.xs_host,
            (uintptr_t)A.dxs_host, (uintptr_t)c.xs_stage.p, (uintptr_t)c.dxs_stage.p, (uintptr_t)A.edev,
            (uintptr_t)A.grad, (uintptr_t)A.hess, (uintptr_t)A.counts, (uintptr_t)A.host_energy,
            (uintptr_t)A.want_alpha, (uintptr_t)c.cap_f, (uintptr_t)c.cap_e, (uintptr_t)c.cap_p,
            (uintptr_t)c.cell_ent.n, (uintptr_t)c.stream, (uintptr_t)c.tune_samples_bpsm,
            (uintptr_t)c.tune_query_bpsm,
            // every context buffer the pass touches: a reallocation between
            // capture and replay must not leave a stale address in the graph
            (uintptr_t)c.red_tmp.p, (uintptr_t)c.red_tmp.n, (uintptr_t)c.cell_ent.p, (uintptr_t)c.cand_face.p,
            (uintptr_t)c.cand_edge.p, (uintptr_t)c.cand_point.p, (uintptr_t)c.cand_count.p, (uintptr_t)c.active.p,
            (uintptr_t)c.qcontact.tri.p, (uintptr_t)c.qcontact.box.p, (uintptr_t)c.qcontact.boxf.p,
            (uintptr_t)c.qcontact.vboxf.p, (uintptr_t)c.qcontact.cell.p, (uintptr_t)c.qswept.tri.p,
            (uintptr_t)c.qswept.boxf.p, (uintptr_t)c.qswept.vboxf.p, (uintptr_t)c.qswept.cell.p,
            (uintptr_t)c.mboxf.p, (uintptr_t)c.ccd_pairs.p, (uintptr_t)c.cap_ccd, (uintptr_t)c.coarse_pairs.p,
            (uintptr_t)c.cap_coarse, (uintptr_t)c.coarse_swept.p, (uintptr_t)c.cap_coarse_swept,
            (uintptr_t)c.ccd_stream, (uintptr_t)c.aux_stream,
            (uintptr_t)c.mcell.p, (uintptr_t)c.cell_cnt.p, (uintptr_t)c.cell_start.p, (uintptr_t)c.scan_tmp.p,
            (uintptr_t)c.tri_E.p, (uintptr_t)c.tri_frame.p, (uintptr_t)c.tri_items.p, (uintptr_t)c.item_owner.p,
            (uintptr_t)c.item_rd.p, (uintptr_t)c.item_rt.p, (uintptr_t)c.cap_items, (uintptr_t)c.item_list.p, (uintptr_t)c.tri_G32.p, (uintptr_t)c.tri_S32.p, (uintptr_t)c.tri_n32.p,
            (uintptr_t)c.tri_G64.p, (uintptr_t)c.tri_S64.p, (uintptr_t)c.tri_n64.p, (uintptr_t)c.cb_val32.p,
            (uintptr_t)c.cb_val64.p, (uintptr_t)c.u64_tmp.p, (uintptr_t)c.i64_tmp.p, (uintptr_t)c.misc_i32.p,
            (uintptr_t)c.dxm.p, (uintptr_t)c.scal.p, (uintptr_t)c.mboxf_in.p, (uintptr_t)c.tri_f32.p,
            (uintptr_t)c.ym32.p, (uintptr_t)c.item_mask.p, (uintptr_t)c.item_mid.p, (uintptr_t)c.tri_mid64.p,
            (uintptr_t)c.tri_mid32.p, (uintptr_t)c.mtri_e32.p, (uintptr_t)c.mtri_pre.p,
            (uintptr_t)c.use_mtri_pre, (uintptr_t)c.use_mtri_e32};
}

// Capture one pass on the context's private capture stream (nothing runs);
// on any failure no graph is kept and calls take the plain path.
void capture_contact_pass(Ctx& c, const ContactPassArgs& A) {
    c.cp_graph.reset();
    if (!c.cap_stream && cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c.cap_stream = nullptr;
        return;
    }
    const std::vector<uintptr_t> key = contact_pass_key(c, A);
    cudaStream_t user = c.stream;
    c.stream = c.cap_stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t e1 = enqueue_contact_pass(c, A);
        const cudaError_t e2 = cudaStreamEndCapture(c.stream, &g);
        e = e1 != cudaSuccess ? e1 : e2;
    }
    c.stream = user;
    int64_t kernels = 0;
    if (e == cudaSuccess && g) {
        size_t n = 0;
        e = cudaGraphGetNodes(g, nullptr, &n);
        std::vector<cudaGraphNode_t> nodes(n);
        if (e == cudaSuccess && n) e = cudaGraphGetNodes(g, nodes.data(), &n);
        for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[i], &t);
            kernels += t == cudaGraphNodeTypeKernel;
        }
    }
    if (e == cudaSuccess && g) e = cudaGraphInstantiate(&c.cp_graph.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c.cp_graph.reset();
        return;
    }
    c.cp_graph.key = key;
    c.cp_graph.kernels = kernels;
}

}  // namespace gmcp

// ===========================================================================
// implicit-Euler time step (paper Sec. 2.1 problem statement; contact
// potential of Sec. 4.2 with the frozen linearisation of each iterate; step
// bound of Sec. 4.5)
// ===========================================================================
namespace gmcp {
namespace {

// Every environment is a problem of its own: the iteration below runs them
// side by side, each with its own energies, residual, step bounds, line
// search and stopping, and every quantity of environment e is computed
// exactly as for a scene holding that environment alone (per-environment
// fixed-order sums, per-environment minima).

// per environment: alpha_e = min(1, alpha_lin, alpha_accd) for x -> x +
// alpha dx with the master moving by dxm (NULL = static), into
// N.h_ealpha.  candidates_current: the broad phase of (x, xm0) is the last
// one run on the context (then it is not repeated and, for a static master,
// the additive CCD reuses its grid).
cudaError_t ccd_bound(Ctx& c, const double* x, const double* dx, const double* xm0, const double* dxm,
                      bool candidates_current) {
    NewtonState& N = *c.newton;
    const int ne = N.n_env;
    unsigned long long* hb = N.h_ebits;
    for (int e = 0; e < ne; ++e) {
        hb[2 * e] = 0x7FF0000000000000ULL;       // +inf
        hb[2 * e + 1] = 0x3FF0000000000000ULL;   // 1.0
    }
    GMCP_CUDA_TRY(cudaMemcpyAsync(N.ebits.p, hb, sizeof(unsigned long long) * 2 * ne, cudaMemcpyHostToDevice,
                                  c.stream));
    GMCP_CUDA_TRY(cudaMemsetAsync(c.i64_tmp.p + 8, 0, 4 * sizeof(long long), c.stream));
    if (!candidates_current) GMCP_CUDA_TRY(run_candidates(c, x, xm0));
    GMCP_CUDA_TRY(contact_alpha_lin(c, x, xm0, dx, dxm, N.ebits.p, 2));
    GMCP_CUDA_TRY(bp_ccd_accd(c, x, dx, xm0, dxm, N.ebits.p + 1, c.i64_tmp.p + 8, dxm == nullptr, false, 2));
    GMCP_CUDA_TRY(cudaMemcpyAsync(hb, N.ebits.p, sizeof(unsigned long long) * 2 * ne, cudaMemcpyDeviceToHost,
                                  c.stream));
    GMCP_CUDA_TRY(cudaStreamSynchronize(c.stream));
    for (int e = 0; e < ne; ++e) {
        double al, aa;
        memcpy(&al, &hb[2 * e], 8);
        memcpy(&aa, &hb[2 * e + 1], 8);
        if (al < INFINITY) al *= (1.0 - 1e-10);
        N.h_ealpha[e] = std::min(1.0, std::min(al, aa));
    }
    return cudaSuccess;
}

// copy es[slot .. slot + k) of every environment to the host (N.h_es, same
// layout) and wait
cudaError_t read_es(Ctx& c, int slot, int k) {
    NewtonState& N = *c.newton;
    GMCP_CUDA_TRY(cudaMemcpy2DAsync(N.h_es + slot, kES * sizeof(double), N.es.p + slot, kES * sizeof(double),
                                    sizeof(double) * k, N.n_env, cudaMemcpyDeviceToHost, c.stream));
    return cudaStreamSynchronize(c.stream);
}

// upload a host mask [n_env] (nonzero = selected) to N.emask + k n_env; the
// stream is drained first, so no earlier copy still reads the pinned slot
const int32_t* put_mask(Ctx& c, int k, const std::vector<uint8_t>& m, bool invert = false) {
    NewtonState& N = *c.newton;
    cudaStreamSynchronize(c.stream);
    int32_t* h = N.h_emask + (size_t)k * N.n_env;
    for (int e = 0; e < N.n_env; ++e) h[e] = (m[e] != 0) != invert ? 1 : 0;
    cudaMemcpyAsync(N.emask.p + (size_t)k * N.n_env, h, sizeof(int32_t) * N.n_env, cudaMemcpyHostToDevice,
                    c.stream);
    return N.emask.p + (size_t)k * N.n_env;
}

// per environment with need[e]: the first j in [0, max_halv] where every
// tet keeps J > 0 (a finite elastic energy) at xi + (a_e 2^-j) dP (j = 0
// first, then batches of 8);
// j_out[e] = -1 if none
cudaError_t first_feasible(Ctx& c, const double* xi, const double* dP, const std::vector<double>& a,
                           int max_halv, const std::vector<uint8_t>& need, std::vector<int>& j_out,
                           std::vector<double>& a_out) {
    NewtonState& N = *c.newton;
    const int ne = N.n_env;
    std::vector<uint8_t> pending(need);
    j_out.assign(ne, -1);
    a_out.assign(ne, 0.0);
    // the first batch tries the step size itself (it is usually feasible),
    // later batches eight halvings at once
    for (int base = 0, na = 1; base <= max_halv; base += na) {
        bool any = false;
        for (int e = 0; e < ne; ++e) any = any || pending[e];
        if (!any) break;
        na = base == 0 ? 1 : std::min(8, max_halv - base + 1);
        for (int e = 0; e < ne; ++e)
            for (int j = 0; j < na; ++j) N.h_eal[8 * e + j] = std::ldexp(a[e], -(base + j));
        GMCP_CUDA_TRY(cudaMemcpyAsync(N.eal.p, N.h_eal, sizeof(double) * 8 * ne, cudaMemcpyHostToDevice, c.stream));
        GMCP_CUDA_TRY(nh_feasible_multi(c, xi, dP, N.eal.p, na, kEsFe));
        GMCP_CUDA_TRY(read_es(c, kEsFe, na));
        for (int e = 0; e < ne; ++e) {
            if (!pending[e]) continue;
            for (int j = 0; j < na; ++j)
                if (std::isfinite(N.h_es[kES * e + kEsFe + j])) {
                    j_out[e] = base + j;
                    a_out[e] = N.h_eal[8 * e + j];
                    pending[e] = 0;
                    break;
                }
        }
    }
    return cudaSuccess;
}

// start point of each environment with need[e]: Dirichlet vertices at xhat
// (their motion must be admissible), free vertices moved toward P by the
// CCD-limited fraction, halved until every tet keeps J > 0.  ok[e] = 0: none
// (x0 = x there, as for environments not asked).  x0 may alias neither x nor P.
cudaError_t start_point(Ctx& c, const double* x, const double* P, double* x0, const std::vector<uint8_t>& need,
                        std::vector<double>& alpha0, std::vector<uint8_t>& ok) {
    NewtonState& N = *c.newton;
    const int ne = N.n_env;
    const int64_t n = 3 * N.nsys;
    std::vector<uint8_t> alive(need);
    std::vector<int> j;
    std::vector<double> aj;
    GMCP_CUDA_TRY(cudaMemcpyAsync(N.xi.p, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.stream));
    bool any_dir = false;
    for (int e = 0; e < ne; ++e) any_dir = any_dir || (alive[e] && N.h_has_dir[e]);
    if (any_dir) {
        GMCP_CUDA_TRY(vec_dir_delta(c, x, N.xhat.p, N.dP.p));
        // the Dirichlet motion moves contact primitives only where Dirichlet
        // vertices lie on a contact surface; elsewhere its bound is exactly 1
        // (no sample's gap and no primitive pair moves)
        bool any_surf = false;
        for (int e = 0; e < ne; ++e) any_surf = any_surf || (alive[e] && N.h_has_dir[e] && N.h_dir_surf[e]);
        if (any_surf) GMCP_CUDA_TRY(ccd_bound(c, x, N.dP.p, master_of(c, x), master_dir_of(c, N.dP.p), false));
        else
            for (int e = 0; e < ne; ++e) N.h_ealpha[e] = 1.0;
        std::vector<uint8_t> chk(ne, 0);
        for (int e = 0; e < ne; ++e) {
            if (!alive[e] || !N.h_has_dir[e]) continue;
            if (N.h_ealpha[e] < 1.0) alive[e] = 0;
            else chk[e] = 1;
        }
        GMCP_CUDA_TRY(vec_set_dir(c, N.xhat.p, N.xi.p));
        GMCP_CUDA_TRY(cudaMemsetAsync(N.dP.p, 0, sizeof(double) * n, c.stream));
        GMCP_CUDA_TRY(first_feasible(c, N.xi.p, N.dP.p, std::vector<double>(ne, 0.0), 0, chk, j, aj));
        for (int e = 0; e < ne; ++e)
            if (chk[e] && j[e] < 0) alive[e] = 0;
    }
    GMCP_CUDA_TRY(vec_free_delta(c, P, N.xi.p, N.dP.p));
    GMCP_CUDA_TRY(ccd_bound(c, N.xi.p, N.dP.p, master_of(c, N.xi.p), master_dir_of(c, N.dP.p), false));
    const std::vector<double> a(N.h_ealpha, N.h_ealpha + ne);
    GMCP_CUDA_TRY(first_feasible(c, N.xi.p, N.dP.p, a, c.prm.max_halvings, alive, j, aj));
    alpha0.assign(ne, 0.0);
    for (int e = 0; e < ne; ++e) {
        if (alive[e] && j[e] < 0) alive[e] = 0;
        N.h_ealpha[e] = alive[e] ? aj[e] : 0.0;
        if (alive[e]) alpha0[e] = aj[e];
    }
    GMCP_CUDA_TRY(cudaMemcpyAsync(N.ealpha.p, N.h_ealpha, sizeof(double) * ne, cudaMemcpyHostToDevice, c.stream));
    const int32_t* m_ok = put_mask(c, 3, alive);
    GMCP_CUDA_TRY(vec_axpy_env(c, N.xi.p, N.dP.p, N.ealpha.p, m_ok, x0));
    const int32_t* m_bad = put_mask(c, 2, alive, true);
    GMCP_CUDA_TRY(vec_copy_env(c, x, m_bad, x0));
    ok = alive;
    return cudaSuccess;
}

}  // namespace

// One implicit-Euler step of every environment.  status_out[e]: 0
// converged, 3 infeasible, 5 not converged, 6 line search.  Joint step
// (deformable master): x, v hold the pad and then the master vertices, and
// f_ext the external nodal forces (or NULL).
cudaError_t newton_run(Ctx& c, double* x, double* v, const double* xm_next, const double* dx_pred,
                       ipc_step_stats* st, int* status_out, const double* f_ext) {
    NewtonState& N = *c.newton;
    const int ne = N.n_env;
    const int64_t n = 3 * N.nsys;
    N.fext = f_ext;
    N.joint_miss = false;
    struct ResetF { NewtonState& N; ~ResetF() { N.fext = nullptr; } } reset_f{N};
    cudaStream_t s = c.stream;
    const double h = c.prm.h, h2 = h * h;
    std::vector<int> status(ne, 0);
    std::vector<uint8_t> run(ne, 1);
    for (int e = 0; e < ne; ++e) st[e] = ipc_step_stats{};
    auto any = [&](const std::vector<uint8_t>& m) {
        for (uint8_t b : m) if (b) return true;
        return false;
    };
    GMCP_CUDA_TRY(cudaMemcpyAsync(N.xt.p, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    GMCP_CUDA_TRY(vec_xhat(c, x, v, N.xhat.p));
    // master motion with the pad held at x^t; an environment whose master
    // cannot move there keeps its master and stops
    if (xm_next && c.nmv > 0 && !N.joint) {
        const int64_t m = 3 * c.nmv;
        GMCP_CUDA_TRY(cudaMemsetAsync(N.tmp.p, 0, sizeof(double) * n, s));
        GMCP_CUDA_TRY(cudaMemcpyAsync(N.dxm.p, xm_next, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
        GMCP_CUDA_TRY(vec_axpy(c, m, -1.0, N.dxm.p, N.xm.p, N.dxm.p));
        GMCP_CUDA_TRY(ccd_bound(c, x, N.tmp.p, N.xm.p, N.dxm.p, false));
        for (int e = 0; e < ne; ++e)
            if (N.h_ealpha[e] < 1.0) { status[e] = 3; run[e] = 0; }
        GMCP_CUDA_TRY(vec_copy_master_env(c, xm_next, put_mask(c, 0, run), N.xm.p));
    }
    // residual scale from the CCD-filtered plain predictor (reading R8)
    std::vector<double> a0, gscale(ne, 0.0);
    std::vector<uint8_t> ok;
    {
        ProfScope ps(c.prof, s, "start_point");
        GMCP_CUDA_TRY(start_point(c, x, N.xhat.p, N.tmp.p, run, a0, ok));
    }
    for (int e = 0; e < ne; ++e)
        if (run[e] && !ok[e]) { status[e] = 3; run[e] = 0; }
    // without a prediction the iteration starts at this point: its system,
    // with the matrix, serves the first iteration too
    const bool reuse = dx_pred == nullptr;
    GMCP_CUDA_TRY(assemble_system(c, N.tmp.p, reuse ? kHessAll : kHessNone));
    GMCP_CUDA_TRY(read_es(c, kEsG2, 1));
    for (int e = 0; e < ne; ++e) gscale[e] = std::sqrt(N.h_es[kES * e + kEsG2]);
    // a predicted start goes through the same CCD-filtered start point and is
    // kept only if its residual is not worse than the plain predictor's
    std::vector<uint8_t> use_pred(ne, 0);
    if (dx_pred && any(run)) {
        std::vector<double> al;
        std::vector<uint8_t> okp;
        GMCP_CUDA_TRY(vec_axpy(c, n, 1.0, x, dx_pred, N.P.p));
        GMCP_CUDA_TRY(start_point(c, x, N.P.p, N.xl.p, run, al, okp));
        if (any(okp)) {
            GMCP_CUDA_TRY(assemble_system(c, N.xl.p, kHessNone));
            GMCP_CUDA_TRY(cudaMemcpyAsync(N.h_ebad, N.ebad.p, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, s));
            GMCP_CUDA_TRY(read_es(c, kEsG2, 1));
            for (int e = 0; e < ne; ++e)
                if (okp[e] && !N.h_ebad[e] && std::sqrt(N.h_es[kES * e + kEsG2]) <= gscale[e]) {
                    use_pred[e] = 1;
                    a0[e] = al[e];
                }
        }
    }
    GMCP_CUDA_TRY(cudaMemcpyAsync(x, N.tmp.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (any(use_pred)) GMCP_CUDA_TRY(vec_copy_env(c, N.xl.p, put_mask(c, 0, use_pred), x));
    for (int e = 0; e < ne; ++e) {
        st[e].pred_used = use_pred[e];
        st[e].alpha0 = a0[e];
        st[e].res0 = gscale[e];
        // floor: force of a 1e-3 strain on one element, h^2 E lbar^2 1e-3
        gscale[e] = std::max(gscale[e], 1e-3 * h2 * c.prm.youngs * N.h_lbar[e] * N.h_lbar[e]);
    }
    std::vector<int> env_pit(ne, 0);
    std::vector<double> al_acc(ne, 0.0);
    const double c0 = 1e-4;
    for (int it = 0; any(run); ++it) {
        // energies, gradient and the contact blocks; the elastic blocks and
        // the matrix only once some environment goes on (the last
        // evaluation of a step, at its converged point, needs neither)
        const bool have_matrix = it == 0 && reuse;
        if (!have_matrix) GMCP_CUDA_TRY(assemble_system(c, x, kHessContact));
        GMCP_CUDA_TRY(cudaMemcpyAsync(N.h_ebad, N.ebad.p, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, s));
        GMCP_CUDA_TRY(read_es(c, kEsEc, 4));
        for (int e = 0; e < ne; ++e) {
            if (!run[e]) continue;
            const double* he = N.h_es + kES * e;
            if (N.h_ebad[e] || !std::isfinite(he[kEsE])) { status[e] = 3; run[e] = 0; continue; }
            st[e].energy = he[kEsE];
            st[e].residual = std::sqrt(he[kEsG2]) / gscale[e];
            if (st[e].residual <= c.prm.newton_tol) { run[e] = 0; continue; }
            if (it >= c.prm.max_newton) { status[e] = 5; run[e] = 0; continue; }
            st[e].newton_iters = it + 1;
        }
        if (!any(run)) break;
        if (!have_matrix) GMCP_CUDA_TRY(finish_hessian(c, x));
        // the environments still iterating solve; the others get b = 0 (their
        // solve stops at once) and a zero direction
        const int32_t* m_run = put_mask(c, 0, run);
        GMCP_CUDA_TRY(vec_neg(c, n, N.G.p, N.tmp.p));
        GMCP_CUDA_TRY(vec_zero_env(c, m_run, N.tmp.p));
        {
            ProfScope ps(c.prof, s, "pcg");
            int pit = 0;
            GMCP_CUDA_TRY(pcg_solve(c, N.tmp.p, N.dirn.p, c.prm.pcg_rel_tol, c.prm.max_pcg, &pit, env_pit.data()));
        }
        for (int e = 0; e < ne; ++e)
            if (run[e]) st[e].pcg_iters_total += env_pit[e];
        GMCP_CUDA_TRY(vec_zero_dir(c, N.dirn.p));
        GMCP_CUDA_TRY(vec_zero_env(c, m_run, N.dirn.p));
        GMCP_CUDA_TRY(dot_env(c, N.G.p, N.dirn.p, kEsGp));
        {
            ProfScope ps(c.prof, s, "step_bound");
            GMCP_CUDA_TRY(ccd_bound(c, x, N.dirn.p, master_of(c, x), master_dir_of(c, N.dirn.p), true));
        }
        const std::vector<double> al(N.h_ealpha, N.h_ealpha + ne);
        GMCP_CUDA_TRY(read_es(c, kEsGp, 1));
        std::vector<double> gp(ne);
        for (int e = 0; e < ne; ++e) gp[e] = N.h_es[kES * e + kEsGp];
        // backtracking on the frozen-linear energy: the batch gives each
        // step size's energy change from x (reading R22; slot 0 is alpha = 0,
        // change 0), tested against 1e-4 alpha G.p; the first batch tries the
        // full step only (it is usually taken), later batches seven halvings
        // at once
        std::vector<uint8_t> searching(run), accepted(ne, 0);
        for (int hv0 = 0, nk = 1; hv0 <= c.prm.max_halvings && any(searching); hv0 += nk) {
            nk = hv0 == 0 ? 1 : std::min(7, c.prm.max_halvings - hv0 + 1);
            for (int e = 0; e < ne; ++e) {
                N.h_eal[8 * e] = 0.0;
                for (int j = 0; j < nk; ++j) N.h_eal[8 * e + 1 + j] = std::ldexp(al[e], -(hv0 + j));
            }
            GMCP_CUDA_TRY(cudaMemcpyAsync(N.eal.p, N.h_eal, sizeof(double) * 8 * ne, cudaMemcpyHostToDevice, s));
            {
                ProfScope ps(c.prof, s, "line_search");
                GMCP_CUDA_TRY(energy_batch(c, x, N.dirn.p, N.eal.p, nk + 1, true, true));
            }
            GMCP_CUDA_TRY(read_es(c, kEsE8, nk + 1));
            for (int e = 0; e < ne; ++e) {
                if (!searching[e]) continue;
                const double* E = N.h_es + kES * e + kEsE8;
                for (int j = 0; j < nk; ++j) {
                    const double a = N.h_eal[8 * e + 1 + j];
                    if (E[1 + j] <= c0 * a * gp[e]) {
                        searching[e] = 0;
                        accepted[e] = 1;
                        al_acc[e] = a;
                        st[e].last_alpha = a;
                        st[e].line_search_halvings += hv0 + j;
                        break;
                    }
                }
            }
        }
        for (int e = 0; e < ne; ++e) {
            if (run[e] && !accepted[e]) { status[e] = 6; run[e] = 0; }
            N.h_ealpha[e] = accepted[e] ? al_acc[e] : 0.0;
        }
        if (any(accepted)) {
            GMCP_CUDA_TRY(cudaMemcpyAsync(N.ealpha.p, N.h_ealpha, sizeof(double) * ne, cudaMemcpyHostToDevice, s));
            GMCP_CUDA_TRY(vec_axpy_env(c, x, N.dirn.p, N.ealpha.p, put_mask(c, 1, accepted), x));
        }
    }
    // converged or out of iterations: the velocity; otherwise x back to x^t
    std::vector<uint8_t> keep(ne);
    for (int e = 0; e < ne; ++e) keep[e] = status[e] == 0 || status[e] == 5;
    GMCP_CUDA_TRY(vec_velocity_env(c, x, N.xt.p, put_mask(c, 0, keep), v));
    GMCP_CUDA_TRY(vec_copy_env(c, N.xt.p, put_mask(c, 1, keep, true), x));
    GMCP_CUDA_TRY(cudaStreamSynchronize(s));
    for (int e = 0; e < ne; ++e) status_out[e] = status[e];
    return cudaSuccess;
}

}  // namespace gmcp

using namespace gmcp;

struct ipc_ctx {
    Ctx c;
};

namespace gmcp {
Ctx& ctx_of(ipc_ctx* h) { return h->c; }
}

static ipc_status fail_ctx(ipc_ctx* ctx, ipc_status st, const std::string& msg) {
    if (ctx) ctx->c.err = msg;
    return st;
}

static ipc_status cuda_fail(ipc_ctx* ctx, cudaError_t e, const char* where) {
    cudaGetLastError();
    return fail_ctx(ctx, e == cudaErrorMemoryAllocation ? IPC_ERR_OOM : IPC_ERR_CUDA,
                    std::string(where) + ": " + cudaGetErrorString(e));
}

#define API_CK(ctx, expr)                                                    \
    do {                                                                     \
        cudaError_t _e = (expr);                                             \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr);             \
    } while (0)

static void build_topology(Ctx& c, const ipc_scene* sc) {
    cudaStream_t s = c.stream;
    const int64_t ns = c.ns, nmt = c.nmt, nmv = c.nmv, nv = c.nv;
    // --- master edges, adjacency and ownership (owner = lowest adjacent tri)
    std::vector<int32_t> medge, me_off, me_adj;
    tri_edges(sc->m_tris, nmt, medge, me_off, me_adj);
    c.nme = (int64_t)medge.size() / 2;
    std::vector<int32_t> mv_off(nmv + 1, 0), mv_adj(3 * nmt);
    for (int64_t t = 0; t < nmt; ++t)
        for (int k = 0; k < 3; ++k) mv_off[sc->m_tris[3 * t + k] + 1]++;
    for (int64_t v = 0; v < nmv; ++v) mv_off[v + 1] += mv_off[v];
    {
        std::vector<int32_t> cur(mv_off.begin(), mv_off.end() - 1);
        for (int64_t t = 0; t < nmt; ++t)
            for (int k = 0; k < 3; ++k) mv_adj[cur[sc->m_tris[3 * t + k]]++] = (int32_t)t;
    }
    std::vector<int32_t> own_e(3 * nmt, -1), own_v(3 * nmt, -1);
    {
        std::vector<int> slot(nmt, 0);
        for (int64_t e = 0; e < c.nme; ++e) {
            const int32_t owner = me_adj[me_off[e]];
            own_e[3 * owner + slot[owner]++] = (int32_t)e;
        }
        std::fill(slot.begin(), slot.end(), 0);
        for (int64_t v = 0; v < nmv; ++v) {
            if (mv_off[v + 1] == mv_off[v]) continue;
            const int32_t owner = mv_adj[mv_off[v]];   // filled in increasing tri order
            own_v[3 * owner + slot[owner]++] = (int32_t)v;
        }
    }
    // --- slave edges and ownership (for CCD)
    std::vector<int32_t> sedge, se_off, se_adj;
    tri_edges(sc->s_tris, ns, sedge, se_off, se_adj);
    c.nse = (int64_t)sedge.size() / 2;
    std::vector<int32_t> sown_e(3 * ns, -1), sown_v(3 * ns, -1), svert;   // svert: vertices of slave tris
    {
        std::vector<int> slot(ns, 0);
        for (int64_t e = 0; e < c.nse; ++e) {
            const int32_t owner = se_adj[se_off[e]];
            sown_e[3 * owner + slot[owner]++] = (int32_t)e;
        }
        std::vector<int32_t> vowner(nv, -1);
        for (int64_t t = 0; t < ns; ++t)
            for (int k = 0; k < 3; ++k) {
                const int32_t v = sc->s_tris[3 * t + k];
                if (vowner[v] < 0) vowner[v] = (int32_t)t;
            }
        std::fill(slot.begin(), slot.end(), 0);
        for (int64_t v = 0; v < nv; ++v)
            if (vowner[v] >= 0) {
                sown_v[3 * vowner[v] + slot[vowner[v]]++] = (int32_t)v;
                svert.push_back((int32_t)v);
            }
    }
    // --- env of each tri
    std::vector<int32_t> s_env(ns), m_env(nmt);
    for (int64_t t = 0; t < ns; ++t) s_env[t] = env_of(c.env_stri_off, t);
    for (int64_t t = 0; t < nmt; ++t) m_env[t] = env_of(c.env_mtri_off, t);
    // --- rest boxes
    std::vector<double> sbox(6 * ns), mbox(6 * nmt);
    auto box = [](const double* P, const int32_t* T, double* out) {
        for (int q = 0; q < 3; ++q) {
            const double a = P[3 * T[0] + q], b = P[3 * T[1] + q], d = P[3 * T[2] + q];
            out[q] = std::min(a, std::min(b, d));
            out[3 + q] = std::max(a, std::max(b, d));
        }
    };
    for (int64_t t = 0; t < ns; ++t) box(sc->pad_rest, sc->s_tris + 3 * t, &sbox[6 * t]);
    for (int64_t t = 0; t < nmt; ++t) box(sc->m_rest, sc->m_tris + 3 * t, &mbox[6 * t]);
    // --- grid per env: master rest box grown by 2 dhat + 5 % of its extent;
    // cell size = max(mean master tri extent, mean slave tri extent + 2 dhat).
    // (The largest master extent made cells up to ~1.5x coarser on meshes of
    // uneven triangles, and a query visits entries ~ cell size^2.)
    const double dhat = c.P.dhat;
    std::vector<double> org(3 * c.n_env), inv(c.n_env);
    std::vector<int32_t> dim(3 * c.n_env);
    std::vector<int64_t> goff(c.n_env + 1, 0);
    double cmax = 1e-3;
    for (int64_t i = 0; i < 3 * nv; ++i) cmax = std::max(cmax, std::fabs(sc->pad_rest[i]));
    for (int64_t i = 0; i < 3 * nmv; ++i) cmax = std::max(cmax, std::fabs(sc->m_rest[i]));
    for (int e = 0; e < c.n_env; ++e) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        double mext = 0.0, sext = 0.0;
        for (int64_t t = c.env_mtri_off[e]; t < c.env_mtri_off[e + 1]; ++t)
            for (int q = 0; q < 3; ++q) {
                lo[q] = std::min(lo[q], mbox[6 * t + q]);
                hi[q] = std::max(hi[q], mbox[6 * t + 3 + q]);
            }
        const int64_t nme_ = c.env_mtri_off[e + 1] - c.env_mtri_off[e];
        for (int64_t t = c.env_mtri_off[e]; t < c.env_mtri_off[e + 1]; ++t) {
            double m = 0.0;
            for (int q = 0; q < 3; ++q) m = std::max(m, mbox[6 * t + 3 + q] - mbox[6 * t + q]);
            mext += m;
        }
        if (nme_ > 0) mext /= (double)nme_;
        const int64_t nse_ = c.env_stri_off[e + 1] - c.env_stri_off[e];
        for (int64_t t = c.env_stri_off[e]; t < c.env_stri_off[e + 1]; ++t) {
            double m = 0.0;
            for (int q = 0; q < 3; ++q) m = std::max(m, sbox[6 * t + 3 + q] - sbox[6 * t + q]);
            sext += m;
        }
        if (nse_ > 0) sext /= (double)nse_;
        if (!(lo[0] <= hi[0]))
            for (int q = 0; q < 3; ++q) { lo[q] = 0.0; hi[q] = 0.0; }
        double h = std::max(mext, sext + 2.0 * dhat);
        if (!(h > 0.0)) h = std::max(dhat, 1e-6);
        const double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
        const double grow = 2.0 * dhat + 0.05 * ext;
        for (int it = 0; it < 64; ++it) {
            int64_t ncell = 1;
            for (int q = 0; q < 3; ++q)
                ncell *= std::max<int64_t>((int64_t)std::ceil((hi[q] - lo[q] + 2 * grow) / h) + 1, 1);
            if (ncell <= ((int64_t)1 << 22)) break;
            h *= 1.26;
        }
        inv[e] = 1.0 / h;
        for (int q = 0; q < 3; ++q) {
            org[3 * e + q] = lo[q] - grow;
            dim[3 * e + q] = (int32_t)std::max<int64_t>((int64_t)std::ceil((hi[q] - lo[q] + 2 * grow) / h) + 1, 1);
        }
        goff[e + 1] = goff[e] + (int64_t)dim[3 * e] * dim[3 * e + 1] * dim[3 * e + 2];
    }
    c.n_cells = goff[c.n_env];
    // slack of the coarse box test: covers the rounding of boxes grown by dhat
    // for coordinates up to 1000x the largest rest coordinate
    c.margin = 4e-13 * cmax + 1e-9 * dhat;
    // --- vertex -> (tri, corner) for the gradient gather
    std::vector<int32_t> vt_off(nv + 1, 0), vt_ent(3 * ns);
    for (int64_t t = 0; t < ns; ++t)
        for (int k = 0; k < 3; ++k) vt_off[sc->s_tris[3 * t + k] + 1]++;
    for (int64_t v = 0; v < nv; ++v) vt_off[v + 1] += vt_off[v];
    {
        std::vector<int32_t> cur(vt_off.begin(), vt_off.end() - 1);
        for (int64_t t = 0; t < ns; ++t)
            for (int k = 0; k < 3; ++k) vt_ent[cur[sc->s_tris[3 * t + k]]++] = (int32_t)(t * 4 + k);
    }
    // --- contact BSR pattern: blocks (T[a], T[b]) of every slave tri, with
    // the contributing (tri, a, b) in increasing order.  The 9 entries of
    // every tri are bucketed by row T[a] (counting sort) and each row sorted
    // by (column, source), which is the lexicographic order of (row, column,
    // source); rows are short (the vertex's incident tris).
    std::vector<int64_t> boff(nv + 1, 0);
    for (int64_t t = 0; t < ns; ++t)
        for (int a = 0; a < 3; ++a) boff[sc->s_tris[3 * t + a] + 1] += 3;
    for (int64_t v = 0; v < nv; ++v) boff[v + 1] += boff[v];
    std::vector<std::pair<int32_t, int32_t>> be((size_t)ns * 9);   // (column, source)
    {
        std::vector<int64_t> cur(boff.begin(), boff.end() - 1);
        for (int64_t t = 0; t < ns; ++t)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    be[(size_t)cur[sc->s_tris[3 * t + a]]++] = {sc->s_tris[3 * t + b], (int32_t)(t * 16 + a * 4 + b)};
    }
    std::vector<int32_t> row(nv + 1, 0), col, src_off, src;
    src.reserve(be.size());
    for (int64_t v = 0; v < nv; ++v) {
        std::sort(be.begin() + boff[v], be.begin() + boff[v + 1]);
        for (int64_t i = boff[v]; i < boff[v + 1]; ++i) {
            if (i == boff[v] || be[i].first != be[i - 1].first) {
                col.push_back(be[i].first);
                src_off.push_back((int32_t)src.size());
                row[v + 1]++;
            }
            src.push_back(be[i].second);
        }
    }
    src_off.push_back((int32_t)src.size());
    std::vector<std::pair<int32_t, int32_t>>().swap(be);
    for (int64_t v = 0; v < nv; ++v) row[v + 1] += row[v];
    c.cb_nnzb = (int64_t)col.size();
    c.h_cb_row = row;
    c.h_cb_col = col;

    CK(c.stri.upload(sc->s_tris, 3 * ns, s));
    CK(c.mtri.upload(sc->m_tris, 3 * nmt, s));
    CK(c.medge.upload(medge.data(), medge.size(), s));
    CK(c.me_tri_off.upload(me_off.data(), me_off.size(), s));
    CK(c.me_tri.upload(me_adj.data(), me_adj.size(), s));
    CK(c.mv_tri_off.upload(mv_off.data(), mv_off.size(), s));
    CK(c.mv_tri.upload(mv_adj.data(), mv_adj.size(), s));
    CK(c.mtri_own_edge.upload(own_e.data(), own_e.size(), s));
    CK(c.mtri_own_vert.upload(own_v.data(), own_v.size(), s));
    CK(c.stri_own_vert.upload(sown_v.data(), sown_v.size(), s));
    c.n_svert = (int64_t)svert.size();
    CK(c.svert.upload(svert.data(), svert.size(), s));
    CK(c.vbound_c.ensure(8 * (size_t)nv + 8));
    CK(c.vbound_s.ensure(12 * (size_t)nv + 12));
    CK(c.stri_own_edge.upload(sown_e.data(), sown_e.size(), s));
    CK(c.sedge.upload(sedge.data(), sedge.size(), s));
    CK(c.stri_env.upload(s_env.data(), s_env.size(), s));
    CK(c.mtri_env.upload(m_env.data(), m_env.size(), s));
    {
        std::vector<int32_t> mv_env((size_t)nmv + 1, 0);
        for (int e = 0; e < c.n_env; ++e)
            for (int64_t u = c.env_mvert_off[e]; u < c.env_mvert_off[e + 1]; ++u) mv_env[u] = e;
        CK(c.mvert_env.upload(mv_env.data(), mv_env.size(), s));
    }
    CK(c.X.upload(sc->pad_rest, 3 * nv, s));
    CK(c.Y0.upload(sc->m_rest, 3 * nmv, s));
    CK(c.srest_box.upload(sbox.data(), sbox.size(), s));
    CK(c.mrest_box.upload(mbox.data(), mbox.size(), s));
    {
        // FP32 copies rounded outward (lo down, hi up)
        auto down = [](double v) { float f = (float)v; return (double)f > v ? std::nextafter(f, -INFINITY) : f; };
        auto up = [](double v) { float f = (float)v; return (double)f < v ? std::nextafter(f, INFINITY) : f; };
        auto outward = [&](const std::vector<double>& b) {
            std::vector<float> o(b.size());
            for (size_t k = 0; k < b.size(); k += 6)
                for (int q = 0; q < 3; ++q) { o[k + q] = down(b[k + q]); o[k + 3 + q] = up(b[k + 3 + q]); }
            return o;
        };
        const std::vector<float> sf = outward(sbox), mf = outward(mbox);
        std::vector<float> vf(6 * (size_t)nmv + 6);
        for (int64_t u = 0; u < nmv; ++u)
            for (int q = 0; q < 3; ++q) {
                vf[6 * u + q] = down(sc->m_rest[3 * u + q]);
                vf[6 * u + 3 + q] = up(sc->m_rest[3 * u + q]);
            }
        CK(c.srest_box_f.upload(sf.data(), sf.size(), s));
        CK(c.mrest_box_f.upload(mf.data(), mf.size(), s));
        CK(c.mvrest_box_f.upload(vf.data(), vf.size(), s));
        CK(cudaStreamSynchronize(s));   // the host vectors end here
    }
    CK(c.grid_org.upload(org.data(), org.size(), s));
    CK(c.grid_inv.upload(inv.data(), inv.size(), s));
    std::vector<float> org_f(org.begin(), org.end()), inv_f(inv.begin(), inv.end());
    CK(c.grid_org_f.upload(org_f.data(), org_f.size(), s));
    CK(c.grid_inv_f.upload(inv_f.data(), inv_f.size(), s));
    CK(c.grid_dim.upload(dim.data(), dim.size(), s));
    CK(c.grid_off.upload(goff.data(), goff.size(), s));
    CK(c.vt_off.upload(vt_off.data(), vt_off.size(), s));
    CK(c.vt_ent.upload(vt_ent.data(), vt_ent.size(), s));
    CK(c.cb_row.upload(row.data(), row.size(), s));
    CK(c.cb_col.upload(col.data(), col.size(), s));
    CK(c.cb_src_off.upload(src_off.data(), src_off.size(), s));
    CK(c.cb_src.upload(src.data(), src.size(), s));
    // the host vectors above must outlive the asynchronous copies
    CK(cudaStreamSynchronize(s));
}

// Face rule of level L = 1, 2 (4^L samples): centroids of the uniform
// midpoint subdivision, upright cells (3i+1, 3j+1, 3k+1)/(3n) with
// i+j+k = n-1 first, then inverted cells (3i+2, 3j+2, 3k+2)/(3n) with
// i+j+k = n-2; n = 2^L.  Unused slots are zero.
static void face_rule_table(double* tab /*[2][16][3]*/) {
    for (int L = 1; L <= 2; ++L) {
        double* r = tab + 48 * (L - 1);
        for (int q = 0; q < 48; ++q) r[q] = 0.0;
        const int n = 1 << L;
        int c = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; i + j < n; ++j, ++c) {
                const int k = n - 1 - i - j;
                r[3 * c] = (double)(3 * i + 1) / (double)(3 * n);
                r[3 * c + 1] = (double)(3 * j + 1) / (double)(3 * n);
                r[3 * c + 2] = (double)(3 * k + 1) / (double)(3 * n);
            }
        for (int i = 0; i < n - 1; ++i)
            for (int j = 0; i + j < n - 1; ++j, ++c) {
                const int k = n - 2 - i - j;
                r[3 * c] = (double)(3 * i + 2) / (double)(3 * n);
                r[3 * c + 1] = (double)(3 * j + 2) / (double)(3 * n);
                r[3 * c + 2] = (double)(3 * k + 2) / (double)(3 * n);
            }
    }
}

static void alloc_call_buffers(Ctx& c) {
    const int64_t ns = c.ns;
    cudaStream_t s = c.stream;
    CK(c.cand_face.ensure((size_t)ns * c.cap_f + 1));
    CK(c.cand_edge.ensure((size_t)ns * c.cap_e + 1));
    CK(c.cand_point.ensure((size_t)ns * c.cap_p + 1));
    CK(c.cand_count.ensure((size_t)ns * 4 + 4));
    CK(c.active.ensure((size_t)ns + 1));
    CK(c.misc_i32.ensure(32));
    CK(cudaMemsetAsync(c.misc_i32.p, 0, sizeof(int32_t) * 32, s));
    CK(c.tri_E.ensure((size_t)ns + 1));
    CK(cudaMemsetAsync(c.tri_E.p, 0, sizeof(double) * (ns + 1), s));
    if (c.P.precision == IPC_PREC_MIXED) {
        CK(c.tri_G32.ensure(3 * (size_t)ns + 3)); CK(c.tri_S32.ensure(6 * (size_t)ns + 6));
        CK(c.tri_n32.ensure(3 * (size_t)ns + 3)); CK(c.cb_val32.ensure(9 * (size_t)c.cb_nnzb + 9));
        CK(cudaMemsetAsync(c.tri_G32.p, 0, sizeof(float) * (3 * ns + 3), s));
        CK(cudaMemsetAsync(c.tri_S32.p, 0, sizeof(float) * (6 * ns + 6), s));
        CK(cudaMemsetAsync(c.tri_n32.p, 0, sizeof(float) * (3 * ns + 3), s));
    } else {
        CK(c.tri_G64.ensure(3 * (size_t)ns + 3)); CK(c.tri_S64.ensure(6 * (size_t)ns + 6));
        CK(c.tri_n64.ensure(3 * (size_t)ns + 3)); CK(c.cb_val64.ensure(9 * (size_t)c.cb_nnzb + 9));
        CK(cudaMemsetAsync(c.tri_G64.p, 0, sizeof(double) * (3 * ns + 3), s));
        CK(cudaMemsetAsync(c.tri_S64.p, 0, sizeof(double) * (6 * ns + 6), s));
        CK(cudaMemsetAsync(c.tri_n64.p, 0, sizeof(double) * (3 * ns + 3), s));
    }
    // touched-output lists: stamps start below the first pass number, the
    // Hessian blocks start at zero
    CK(c.tri_stamp.ensure((size_t)ns + 1));
    CK(c.v_stamp.ensure((size_t)c.nv + 1));
    CK(c.b_stamp.ensure((size_t)c.cb_nnzb + 1));
    CK(c.v_list.ensure((size_t)c.nv + 1));
    CK(c.b_list0.ensure((size_t)c.cb_nnzb + 1));
    CK(c.b_list1.ensure((size_t)c.cb_nnzb + 1));
    CK(cudaMemsetAsync(c.tri_stamp.p, 0, sizeof(int32_t) * (ns + 1), s));
    CK(cudaMemsetAsync(c.v_stamp.p, 0, sizeof(int32_t) * (c.nv + 1), s));
    CK(cudaMemsetAsync(c.b_stamp.p, 0, sizeof(int32_t) * (c.cb_nnzb + 1), s));
    {
        int32_t* lists[2] = {c.b_list0.p, c.b_list1.p};
        CK(c.b_lists.upload(lists, 2, s));
        CK(cudaStreamSynchronize(s));
    }
    if (c.P.precision == IPC_PREC_MIXED)
        CK(cudaMemsetAsync(c.cb_val32.p, 0, sizeof(float) * 9 * (c.cb_nnzb + 1), s));
    else
        CK(cudaMemsetAsync(c.cb_val64.p, 0, sizeof(double) * 9 * (c.cb_nnzb + 1), s));
    CK(c.u64_tmp.ensure(8));
    CK(c.i64_tmp.ensure(16));
    CK(c.scal.ensure(16));
    CK(cudaMallocHost(reinterpret_cast<void**>(&c.h_scalars), 16 * sizeof(double)));
    CK(cudaMallocHost(reinterpret_cast<void**>(&c.h_counts), 16 * sizeof(long long)));
    CK(cudaMallocHost(reinterpret_cast<void**>(&c.pin), sizeof(PinnedIO)));
    memset(c.pin, 0, sizeof(PinnedIO));
    c.pin->init[0] = 0x7FF0000000000000ULL;   // alpha_lin starts at +inf
    c.pin->init[1] = 0x3FF0000000000000ULL;   // alpha_accd starts at 1
}

extern "C" {

ipc_status ipc_create(const ipc_params* params, const ipc_scene* scene, ipc_ctx** out) {
    g_create_error.clear();
    if (!out) { g_create_error = "ipc_create: out is NULL"; return IPC_ERR_ARG; }
    *out = nullptr;
    if (!params || !scene) { g_create_error = "ipc_create: NULL params or scene"; return IPC_ERR_ARG; }
    if (scene->n_env < 1 || !scene->env_vert_off || !scene->env_stri_off || !scene->env_mvert_off ||
        !scene->env_mtri_off || !scene->env_tet_off) {
        g_create_error = "ipc_create: scene needs n_env >= 1 and all env offset arrays";
        return IPC_ERR_ARG;
    }
    if (scene->n_vert <= 0 || scene->n_stri < 0 || scene->n_mvert < 0 || scene->n_mtri < 0 ||
        !scene->pad_rest || (scene->n_stri && !scene->s_tris) || (scene->n_mtri && !scene->m_tris) ||
        (scene->n_mvert && !scene->m_rest)) {
        g_create_error = "ipc_create: missing scene arrays";
        return IPC_ERR_ARG;
    }
    if (scene->n_vert >= ((int64_t)1 << 31) || scene->n_stri >= ((int64_t)1 << 27) ||
        scene->n_mtri >= ((int64_t)1 << 31) || scene->n_tet >= ((int64_t)1 << 31)) {
        g_create_error = "ipc_create: sizes exceed the 32-bit index range";
        return IPC_ERR_ARG;
    }
    if (params->face_rule_level != 1 && params->face_rule_level != 2) {
        g_create_error = "ipc_create: face_rule_level must be 1 or 2";
        return IPC_ERR_ARG;
    }
    if (!(params->dhat > 0.0) || !(params->ccd_slack > 0.0 && params->ccd_slack < 1.0) ||
        params->ccd_max_iter < 1 || (params->face_sampler != 0 && params->face_sampler != 1) ||
        (params->precision != IPC_PREC_FP64 && params->precision != IPC_PREC_MIXED)) {
        g_create_error = "ipc_create: invalid dhat, ccd_slack, ccd_max_iter, face_sampler or precision";
        return IPC_ERR_ARG;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || params->device < 0 || ndev <= params->device) {
        g_create_error = std::string("ipc_create: no usable CUDA device: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return IPC_ERR_CUDA;
    }
    ipc_ctx* ctx = new ipc_ctx();
    Ctx& c = ctx->c;
    try {
        c.prm = *params;
        c.device = params->device;
        CK(cudaSetDevice(c.device));
        c.stream = (cudaStream_t)params->stream;
        c.P.precision = params->precision;
        c.P.dhat = params->dhat; c.P.kappa = params->kappa; c.P.kappa_edge = params->kappa_edge;
        c.P.kappa_point = params->kappa_point; c.P.delta_T = params->delta_T; c.P.delta_e = params->delta_e;
        c.P.L = params->face_rule_level; c.P.nk = 1 << (2 * c.P.L);
        c.P.dhat_guard = params->dhat_guard; c.P.kappa_guard = params->kappa_guard;
        c.P.ccd_slack = params->ccd_slack; c.P.ccd_max_iter = params->ccd_max_iter;
        c.P.face_clip = params->face_sampler;
        c.P.inv_dhat = 1.0 / params->dhat;
        c.P.kappa_f = (float)c.P.kappa; c.P.kappa_edge_f = (float)c.P.kappa_edge;
        c.P.kappa_point_f = (float)c.P.kappa_point;
        c.P.delta_T_f = (float)c.P.delta_T; c.P.delta_e_f = (float)c.P.delta_e;
        c.P.dhat_hi = (float)params->dhat;
        c.P.dhat_lo = (float)(params->dhat - (double)c.P.dhat_hi);
        c.P.inv_dhat_f = (float)c.P.inv_dhat;
        {
            const double r = params->dhat * (1.2 / 0.9);
            float f = (float)(r * r);
            if ((double)f < r * r) f = std::nextafter(f, INFINITY);
            c.P.far_r2_f = f * (1.0f + 1e-6f);
        }
        c.graphs = params->use_graphs != 0;
        c.n_env = scene->n_env;
        auto cp = [&](const int64_t* p) { return std::vector<int64_t>(p, p + scene->n_env + 1); };
        c.env_vert_off = cp(scene->env_vert_off); c.env_tet_off = cp(scene->env_tet_off);
        c.env_stri_off = cp(scene->env_stri_off); c.env_mvert_off = cp(scene->env_mvert_off);
        c.env_mtri_off = cp(scene->env_mtri_off);
        c.nv = scene->n_vert; c.nt = scene->n_tet; c.ns = scene->n_stri;
        c.nmv = scene->n_mvert; c.nmt = scene->n_mtri;
        for (int64_t i = 0; i < 3 * c.ns; ++i)
            if (scene->s_tris[i] < 0 || scene->s_tris[i] >= c.nv) throw Fail{IPC_ERR_ARG, "s_tris index out of range"};
        for (int64_t i = 0; i < 3 * c.nmt; ++i)
            if (scene->m_tris[i] < 0 || scene->m_tris[i] >= c.nmv) throw Fail{IPC_ERR_ARG, "m_tris index out of range"};
        {
            double tab[96];
            face_rule_table(tab);
            CK(bp_init_constants(tab));
            CK(contact_init_constants(tab));
        }
        if (c.nt > 0 && !scene->tets) throw Fail{IPC_ERR_ARG, "n_tet > 0 but tets is NULL"};
        for (int64_t i = 0; i < 4 * c.nt; ++i)
            if (scene->tets[i] < 0 || scene->tets[i] >= c.nv) throw Fail{IPC_ERR_ARG, "tets index out of range"};
        if (c.nt >= ((int64_t)1 << 27)) throw Fail{IPC_ERR_ARG, "n_tet must be below 2^27"};
        // kept for the time stepper, whose state is built on its first call
        c.h_X.assign(scene->pad_rest, scene->pad_rest + 3 * c.nv);
        c.h_Y0.assign(scene->m_rest, scene->m_rest + 3 * c.nmv);
        c.h_stri.assign(scene->s_tris, scene->s_tris + 3 * c.ns);
        c.h_mtri.assign(scene->m_tris, scene->m_tris + 3 * c.nmt);
        if (c.nt > 0) c.h_tets.assign(scene->tets, scene->tets + 4 * c.nt);
        if (scene->dirichlet) c.h_dir.assign(scene->dirichlet, scene->dirichlet + c.nv);
        else c.h_dir.assign(c.nv, 0);
        build_topology(c, scene);
        alloc_call_buffers(c);
        CK(cudaStreamSynchronize(c.stream));
    } catch (const Fail& f) {
        g_create_error = "ipc_create: " + f.msg;
        cudaGetLastError();
        ipc_destroy(ctx);
        return f.st;
    } catch (const std::exception& ex) {
        g_create_error = std::string("ipc_create: ") + ex.what();
        ipc_destroy(ctx);
        return IPC_ERR_OOM;
    }
    *out = ctx;
    return IPC_OK;
}

void ipc_destroy(ipc_ctx* ctx) {
    if (!ctx) return;
    Ctx& c = ctx->c;
    cudaSetDevice(c.device);
    cudaStreamSynchronize(c.stream);
    if (c.h_scalars) cudaFreeHost(c.h_scalars);
    if (c.h_counts) cudaFreeHost(c.h_counts);
    c.cp_graph.reset();
    c.pcg_graph.reset();
    if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
    if (c.ccd_stream) cudaStreamDestroy(c.ccd_stream);
    if (c.h2d_stream) cudaStreamDestroy(c.h2d_stream);
    if (c.ev_xin) cudaEventDestroy(c.ev_xin);
    if (c.ev_dxin) cudaEventDestroy(c.ev_dxin);
    if (c.aux_stream) cudaStreamDestroy(c.aux_stream);
    if (c.ev_touch0) cudaEventDestroy(c.ev_touch0);
    if (c.ev_touch1) cudaEventDestroy(c.ev_touch1);
    if (c.ev_master) cudaEventDestroy(c.ev_master);
    if (c.ev_mfork) cudaEventDestroy(c.ev_mfork);
    if (c.ev_samples) cudaEventDestroy(c.ev_samples);
    if (c.ev_fork) cudaEventDestroy(c.ev_fork);
    if (c.ev_join) cudaEventDestroy(c.ev_join);
    if (c.pin) cudaFreeHost(c.pin);
    delete ctx;   // every DBuf member frees its device memory
}

const char* ipc_last_error(const ipc_ctx* ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->c.err.c_str();
}

ipc_status ipc_candidates(ipc_ctx* ctx, const double* x_dev, const double* xm_dev,
                          ipc_candidate_counts* counts) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!x_dev || (!xm_dev && c.nmv > 0)) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_candidates: NULL positions");
    API_CK(ctx, cudaSetDevice(c.device));
    API_CK(ctx, run_candidates(c, x_dev, xm_dev));
    if (counts) {
        API_CK(ctx, cudaMemsetAsync(c.i64_tmp.p, 0, 8 * sizeof(long long), c.stream));
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(1024, (c.ns + 255) / 256));
        launch_dep(k_count_sum, (unsigned)blocks, 256, 0, c.stream, c.cand_count.p, c.ns, c.i64_tmp.p);
        API_CK(ctx, cudaGetLastError());
        API_CK(ctx, cudaMemcpyAsync(c.h_counts, c.i64_tmp.p, 6 * sizeof(long long), cudaMemcpyDeviceToHost, c.stream));
        API_CK(ctx, cudaStreamSynchronize(c.stream));
        counts->face = c.h_counts[0]; counts->edge = c.h_counts[1]; counts->point = c.h_counts[2];
        counts->max_per_tri[0] = (int32_t)c.h_counts[3];
        counts->max_per_tri[1] = (int32_t)c.h_counts[4];
        counts->max_per_tri[2] = (int32_t)c.h_counts[5];
    }
    return IPC_OK;
}

ipc_status ipc_candidates_copy(ipc_ctx* ctx, int32_t kind, int32_t* pairs_host, int64_t capacity,
                               int64_t* n_out) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (kind < 0 || kind > 2 || !n_out) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_candidates_copy: bad kind or n_out");
    API_CK(ctx, cudaSetDevice(c.device));
    const int32_t cap = kind == 0 ? c.cap_f : (kind == 1 ? c.cap_e : c.cap_p);
    const int32_t* lists = kind == 0 ? c.cand_face.p : (kind == 1 ? c.cand_edge.p : c.cand_point.p);
    std::vector<int32_t> cnt(4 * c.ns + 4), L((size_t)c.ns * cap + 1);
    API_CK(ctx, cudaMemcpyAsync(cnt.data(), c.cand_count.p, sizeof(int32_t) * 4 * c.ns, cudaMemcpyDeviceToHost, c.stream));
    API_CK(ctx, cudaMemcpyAsync(L.data(), lists, sizeof(int32_t) * c.ns * cap, cudaMemcpyDeviceToHost, c.stream));
    API_CK(ctx, cudaStreamSynchronize(c.stream));
    int64_t n = 0;
    for (int64_t t = 0; t < c.ns; ++t) n += std::min(cnt[4 * t + kind], cap);
    *n_out = n;
    if (!pairs_host) return IPC_OK;
    if (capacity < n) return fail_ctx(ctx, IPC_ERR_CAPACITY, "ipc_candidates_copy: capacity too small");
    int64_t k = 0;
    for (int64_t t = 0; t < c.ns; ++t) {
        const int m = std::min(cnt[4 * t + kind], cap);
        for (int j = 0; j < m; ++j) {
            pairs_host[2 * k] = (int32_t)t;
            pairs_host[2 * k + 1] = L[(size_t)t * cap + j];
            ++k;
        }
    }
    return IPC_OK;
}

ipc_status ipc_barrier_eval(ipc_ctx* ctx, const double* x_dev, const double* xm_dev,
                            double* energy_dev, double* energy_host, void* grad_dev,
                            ipc_bsr_view* hess, ipc_sample_counts* counts) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!x_dev || (!xm_dev && c.nmv > 0)) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_barrier_eval: NULL positions");
    API_CK(ctx, cudaSetDevice(c.device));
    API_CK(ctx, run_candidates(c, x_dev, xm_dev));
    long long* ctr = nullptr;
    if (counts) {
        API_CK(ctx, cudaMemsetAsync(c.i64_tmp.p, 0, 8 * sizeof(long long), c.stream));
        ctr = c.i64_tmp.p;
    }
    double* edev = energy_dev;
    if (energy_host && !energy_dev) edev = c.scal.p;
    API_CK(ctx, contact_eval(c, x_dev, xm_dev, edev, grad_dev, hess != nullptr, ctr));
    if (energy_host)
        API_CK(ctx, cudaMemcpyAsync(c.h_scalars, edev, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (counts)
        API_CK(ctx, cudaMemcpyAsync(c.h_counts, c.i64_tmp.p, 4 * sizeof(long long), cudaMemcpyDeviceToHost, c.stream));
    int32_t n_query = 0;
    if (counts)
        API_CK(ctx, cudaMemcpyAsync(&n_query, c.misc_i32.p + 8, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    if (energy_host || counts) API_CK(ctx, cudaStreamSynchronize(c.stream));
    if (energy_host) *energy_host = c.h_scalars[0];
    if (counts) {
        counts->face = c.h_counts[0]; counts->edge = c.h_counts[1]; counts->point = c.h_counts[2];
        counts->guard = 0; counts->face_evaluated = c.h_counts[3]; counts->query_tris = n_query;
    }
    if (hess) {
        const bool f32 = c.P.precision == IPC_PREC_MIXED;
        hess->n_rows = c.nv;
        hess->nnzb = c.cb_nnzb;
        hess->row_ptr_dev = c.cb_row.p;
        hess->col_idx_dev = c.cb_col.p;
        hess->vals_dev = f32 ? (const void*)c.cb_val32.p : (const void*)c.cb_val64.p;
        hess->dtype = f32 ? 1 : 0;
    }
    return IPC_OK;
}

ipc_status ipc_master_grad(ipc_ctx* ctx, const double* x_dev, const double* xm_dev, double* grad_m_dev) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!x_dev || (c.nmv > 0 && (!xm_dev || !grad_m_dev)))
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_master_grad: NULL pointer");
    if (c.nmv == 0) return IPC_OK;
    API_CK(ctx, cudaSetDevice(c.device));
    API_CK(ctx, run_candidates(c, x_dev, xm_dev));
    // the rows summed in a fixed order (entries sorted by master vertex, then
    // by value), so repeated calls agree bitwise
    API_CK(ctx, cudaMemsetAsync(grad_m_dev, 0, sizeof(double) * 3 * (size_t)c.nmv, c.stream));
    API_CK(ctx, sorted_master_terms(c, x_dev, xm_dev, c.nv + c.nmv, c.nv, grad_m_dev, false, nullptr, nullptr,
                                    nullptr, nullptr, nullptr));
    return IPC_OK;
}

ipc_status ipc_master_hess(ipc_ctx* ctx, const double* x_dev, const double* xm_dev, int64_t capacity,
                           int32_t* ij_dev, double* blk_dev, int64_t* n_host) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!x_dev || !n_host || capacity < 0 || (capacity > 0 && (!ij_dev || !blk_dev)) || (c.nmv > 0 && !xm_dev))
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_master_hess: NULL pointer or negative capacity");
    *n_host = 0;
    if (c.nmv == 0) return IPC_OK;
    API_CK(ctx, cudaSetDevice(c.device));
    API_CK(ctx, run_candidates(c, x_dev, xm_dev));
    API_CK(ctx, contact_master_hess(c, x_dev, xm_dev, ij_dev, blk_dev, capacity, c.u64_tmp.p + 2));
    unsigned long long n = 0;
    API_CK(ctx, cudaMemcpyAsync(&n, c.u64_tmp.p + 2, sizeof(n), cudaMemcpyDeviceToHost, c.stream));
    API_CK(ctx, cudaStreamSynchronize(c.stream));
    *n_host = (int64_t)n;
    if ((int64_t)n > capacity)
        return fail_ctx(ctx, IPC_ERR_CAPACITY, "ipc_master_hess: more blocks than capacity (*n_host holds the count)");
    return IPC_OK;
}

ipc_status ipc_ccd_max_step(ipc_ctx* ctx, const double* x_dev, const double* dx_dev,
                            const double* xm0_dev, const double* xm1_dev, double* alpha_host,
                            ipc_ccd_info* info) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!x_dev || !dx_dev || (!xm0_dev && c.nmv > 0) || !alpha_host)
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_ccd_max_step: NULL argument");
    API_CK(ctx, cudaSetDevice(c.device));
    const double* dxm = nullptr;
    if (xm1_dev) {
        API_CK(ctx, c.dxm.ensure(3 * (size_t)c.nmv + 3));
        const int64_t n = 3 * c.nmv;
        if (n > 0) {
            launch_dep(k_sub, (unsigned)((n + 255) / 256), 256, 0, c.stream, xm1_dev, xm0_dev, c.dxm.p, n);
            API_CK(ctx, cudaGetLastError());
        }
        dxm = c.dxm.p;
    }
    // alpha bits: [0] = alpha_lin (init +inf), [1] = alpha_accd (init 1.0)
    const unsigned long long init[2] = {0x7FF0000000000000ULL, 0x3FF0000000000000ULL};
    API_CK(ctx, cudaMemcpyAsync(c.u64_tmp.p, init, sizeof(init), cudaMemcpyHostToDevice, c.stream));
    API_CK(ctx, cudaMemsetAsync(c.i64_tmp.p + 8, 0, 4 * sizeof(long long), c.stream));
    API_CK(ctx, run_candidates(c, x_dev, xm0_dev));
    API_CK(ctx, contact_alpha_lin(c, x_dev, xm0_dev, dx_dev, dxm, c.u64_tmp.p));
    API_CK(ctx, bp_ccd_accd(c, x_dev, dx_dev, xm0_dev, dxm, c.u64_tmp.p + 1, c.i64_tmp.p + 8));
    unsigned long long bits[2];
    long long ctr[4];
    int32_t n_swept = 0;
    API_CK(ctx, cudaMemcpyAsync(bits, c.u64_tmp.p, sizeof(bits), cudaMemcpyDeviceToHost, c.stream));
    API_CK(ctx, cudaMemcpyAsync(ctr, c.i64_tmp.p + 8, sizeof(ctr), cudaMemcpyDeviceToHost, c.stream));
    API_CK(ctx, cudaMemcpyAsync(&n_swept, c.misc_i32.p + 9, sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
    API_CK(ctx, cudaStreamSynchronize(c.stream));
    double al, aa;
    memcpy(&al, &bits[0], 8);
    memcpy(&aa, &bits[1], 8);
    // rounding-order differences in the linearised gap may only shrink the step
    if (al < INFINITY) al *= (1.0 - 1e-10);
    const double a = std::min(1.0, std::min(al, aa));
    *alpha_host = a;
    if (info) {
        info->alpha = a; info->alpha_lin = al; info->alpha_accd = aa;
        info->n_pairs_pt = ctr[0]; info->n_pairs_ee = ctr[1]; info->iter_cap_hit = (int32_t)(ctr[2] != 0);
        info->swept_tris = n_swept;
    }
    return IPC_OK;
}

static ipc_status contact_pass_impl(ipc_ctx* ctx, const double* x_dev, const double* xm0_dev,
                                    const double* xm1_dev, const double* dx_dev, double* energy_dev,
                                    double* energy_host, void* grad_dev, ipc_bsr_view* hess,
                                    double* alpha_host, ipc_ccd_info* info, ipc_sample_counts* counts,
                                    const double* xs_host, const double* dxs_host) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!x_dev || (!xm0_dev && c.nmv > 0)) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_contact_pass: NULL positions");
    API_CK(ctx, cudaSetDevice(c.device));
    const bool want_alpha = dx_dev && (alpha_host || info);
    // a call that returns host values synchronises once at the end; it then
    // also checks the capacity flags and redoes the pass after growing
    const bool lazy = energy_host || counts || want_alpha;
    double* edev = energy_dev;
    if (energy_host && !energy_dev) edev = c.scal.p;
    ContactPassArgs A{x_dev, xm0_dev, xm1_dev, dx_dev, edev, grad_dev, hess != nullptr, counts != nullptr,
                      energy_host != nullptr, want_alpha, lazy, xs_host, dxs_host};
    if (!lazy) {
        API_CK(ctx, enqueue_contact_pass(c, A));
    } else {
        bool done = false;
        const bool use_graph = c.graphs && !c.prof.on;
        if (use_graph && c.cp_graph.exec && c.cp_graph.key == contact_pass_key(c, A)) {
            API_CK(ctx, cudaGraphLaunch(c.cp_graph.exec, c.stream));
            API_CK(ctx, cudaStreamSynchronize(c.stream));
            if (!pass_overflowed(c)) done = true;
            else c.cp_graph.reset();
        }
        if (!done) {
            for (int attempt = 0;; ++attempt) {
                if (attempt >= 6) return fail_ctx(ctx, IPC_ERR_CAPACITY, "ipc_contact_pass: capacities did not settle");
                API_CK(ctx, enqueue_contact_pass(c, A));
                API_CK(ctx, cudaStreamSynchronize(c.stream));
                if (!pass_overflowed(c)) break;
                API_CK(ctx, grow_after_overflow(c));
            }
            API_CK(ctx, grow_items(c));
            if (use_graph) capture_contact_pass(c, A);
        } else if (c.pin->flags[16] > c.cap_items) {
            API_CK(ctx, grow_items(c));
        }
        // the next passes' choice of the face pre-filter's master table
        c.use_mtri_pre = c.P.precision == IPC_PREC_MIXED && (int64_t)c.pin->flags[16] >= 8 * c.nmt;
        c.use_mtri_e32 = c.P.precision == IPC_PREC_MIXED && (int64_t)c.pin->flags[16] >= c.nmt;
    }
    if (energy_host) *energy_host = c.pin->energy;
    if (counts) {
        counts->face = c.pin->counts[0]; counts->edge = c.pin->counts[1]; counts->point = c.pin->counts[2];
        counts->guard = 0; counts->face_evaluated = c.pin->counts[3];
        counts->query_tris = c.pin->flags[8];
    }
    if (hess) {
        const bool f32 = c.P.precision == IPC_PREC_MIXED;
        hess->n_rows = c.nv; hess->nnzb = c.cb_nnzb;
        hess->row_ptr_dev = c.cb_row.p; hess->col_idx_dev = c.cb_col.p;
        hess->vals_dev = f32 ? (const void*)c.cb_val32.p : (const void*)c.cb_val64.p;
        hess->dtype = f32 ? 1 : 0;
    }
    if (want_alpha) {
        double al, aa;
        memcpy(&al, &c.pin->bits[0], 8);
        memcpy(&aa, &c.pin->bits[1], 8);
        if (al < INFINITY) al *= (1.0 - 1e-10);
        const double a = std::min(1.0, std::min(al, aa));
        if (alpha_host) *alpha_host = a;
        if (info) {
            info->alpha = a; info->alpha_lin = al; info->alpha_accd = aa;
            info->n_pairs_pt = c.pin->ctr_ccd[0]; info->n_pairs_ee = c.pin->ctr_ccd[1];
            info->iter_cap_hit = (int32_t)(c.pin->ctr_ccd[2] != 0);
            info->swept_tris = c.pin->flags[9];
        }
    }
    return IPC_OK;
}

ipc_status ipc_contact_pass(ipc_ctx* ctx, const double* x_dev, const double* xm0_dev,
                            const double* xm1_dev, const double* dx_dev, double* energy_dev,
                            double* energy_host, void* grad_dev, ipc_bsr_view* hess,
                            double* alpha_host, ipc_ccd_info* info, ipc_sample_counts* counts) {
    return contact_pass_impl(ctx, x_dev, xm0_dev, xm1_dev, dx_dev, energy_dev, energy_host, grad_dev, hess,
                             alpha_host, info, counts, nullptr, nullptr);
}

// a pointer into page-locked host memory (the copies are captured into
// the pass's graph, which pageable memory cannot be)
static bool page_locked(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

ipc_status ipc_contact_pass_host(ipc_ctx* ctx, const double* xs_host, const double* dxs_host, double* x_dev,
                                 double* dx_dev, const double* xm0_dev, const double* xm1_dev,
                                 double* energy_dev, double* energy_host, void* grad_dev, ipc_bsr_view* hess,
                                 double* alpha_host, ipc_ccd_info* info, ipc_sample_counts* counts) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!xs_host || !x_dev || (dxs_host && !dx_dev) || (dx_dev && !dxs_host))
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_contact_pass_host: NULL pointer (dxs_host and dx_dev go together)");
    if (c.n_svert > 0 && (!page_locked(xs_host) || (dxs_host && !page_locked(dxs_host))))
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_contact_pass_host: host inputs must be page-locked");
    API_CK(ctx, cudaSetDevice(c.device));
    if (!c.h2d_stream) API_CK(ctx, cudaStreamCreateWithFlags(&c.h2d_stream, cudaStreamNonBlocking));
    if (!c.ev_xin) API_CK(ctx, cudaEventCreateWithFlags(&c.ev_xin, cudaEventDisableTiming));
    if (!c.ev_dxin) API_CK(ctx, cudaEventCreateWithFlags(&c.ev_dxin, cudaEventDisableTiming));
    API_CK(ctx, c.xs_stage.ensure(3 * (size_t)c.n_svert + 3));
    if (dxs_host) API_CK(ctx, c.dxs_stage.ensure(3 * (size_t)c.n_svert + 3));
    return contact_pass_impl(ctx, x_dev, xm0_dev, xm1_dev, dx_dev, energy_dev, energy_host, grad_dev, hess,
                             alpha_host, info, counts, xs_host, dxs_host);
}

ipc_status ipc_autotune(ipc_ctx* ctx, const double* x_dev, const double* xm0_dev, const double* dx_dev,
                        int32_t reps, int32_t* samples_bpsm_out, int32_t* query_bpsm_out, double* ms_out) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!x_dev || (!xm0_dev && c.nmv > 0)) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_autotune: NULL positions");
    if (reps < 1) reps = 3;
    API_CK(ctx, cudaSetDevice(c.device));
    const bool graphs = c.graphs, prof = c.prof.on;
    c.graphs = false;
    c.prof.on = false;
    cudaEvent_t e0, e1;
    API_CK(ctx, cudaEventCreate(&e0));
    API_CK(ctx, cudaEventCreate(&e1));
    double energy = 0.0, alpha = 0.0;
    ipc_status st = IPC_OK;
    // median time of `reps` full passes (after one untimed pass)
    auto time_pass = [&](double* ms) -> ipc_status {
        std::vector<float> t;
        for (int r = 0; r <= reps; ++r) {
            cudaEventRecord(e0, c.stream);
            ipc_status q = ipc_contact_pass(ctx, x_dev, xm0_dev, nullptr, dx_dev, nullptr, &energy, nullptr,
                                            nullptr, dx_dev ? &alpha : nullptr, nullptr, nullptr);
            if (q != IPC_OK) return q;
            cudaEventRecord(e1, c.stream);
            cudaEventSynchronize(e1);
            float m = 0.f;
            cudaEventElapsedTime(&m, e0, e1);
            if (r > 0) t.push_back(m);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return IPC_OK;
    };
    const int cand_q[] = {2, 4, 8, 16, 32};
    const int cand_s[] = {1, 2, 4, 8, 16};
    double best = 1e300;
    int bq = c.tune_query_bpsm, bs = c.tune_samples_bpsm;
    for (int q : cand_q) {
        c.tune_query_bpsm = q;
        double ms;
        if ((st = time_pass(&ms)) != IPC_OK) break;
        if (ms < best) { best = ms; bq = q; }
    }
    c.tune_query_bpsm = bq;
    if (st == IPC_OK) {
        best = 1e300;
        for (int b : cand_s) {
            c.tune_samples_bpsm = b;
            double ms;
            if ((st = time_pass(&ms)) != IPC_OK) break;
            if (ms < best) { best = ms; bs = b; }
        }
        c.tune_samples_bpsm = bs;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.graphs = graphs;
    c.prof.on = prof;
    c.cp_graph.reset();
    if (st != IPC_OK) return st;
    if (samples_bpsm_out) *samples_bpsm_out = bs;
    if (query_bpsm_out) *query_bpsm_out = bq;
    if (ms_out) *ms_out = best;
    return IPC_OK;
}

ipc_status ipc_slave_vertices(ipc_ctx* ctx, int32_t* ids_host, int64_t* n_host) {
    if (!ctx || !n_host) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    *n_host = c.n_svert;
    if (ids_host && c.n_svert > 0) {
        API_CK(ctx, cudaMemcpy(ids_host, c.svert.p, sizeof(int32_t) * c.n_svert, cudaMemcpyDeviceToHost));
    }
    return IPC_OK;
}

ipc_status ipc_scatter_slave(ipc_ctx* ctx, const double* xs_dev, double* x_dev) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (c.n_svert == 0) return IPC_OK;
    if (!xs_dev || !x_dev) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_scatter_slave: NULL pointer");
    launch_dep(k_scatter_slave, (unsigned)((c.n_svert + 255) / 256), 256, 0, c.stream, c.svert.p, c.n_svert, xs_dev, x_dev);
    API_CK(ctx, cudaGetLastError());
    return IPC_OK;
}

ipc_status ipc_set_launch_shape(ipc_ctx* ctx, int32_t samples_bpsm, int32_t query_bpsm) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (samples_bpsm < 1 || samples_bpsm > 64 || query_bpsm < 1 || query_bpsm > 64)
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_set_launch_shape: blocks per SM must be in [1, 64]");
    c.tune_samples_bpsm = samples_bpsm;
    c.tune_query_bpsm = query_bpsm;
    c.cp_graph.reset();
    return IPC_OK;
}

ipc_status ipc_set_item_capacity(ipc_ctx* ctx, int64_t capacity) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (capacity < 1 || capacity > ((int64_t)1 << 31) - 1)
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_set_item_capacity: capacity must be in [1, 2^31 - 1]");
    c.cap_items = capacity;
    c.cp_graph.reset();
    return IPC_OK;
}

ipc_status ipc_profile(ipc_ctx* ctx, int32_t mode, int32_t max_sections, char* names_host,
                       double* ms_host, int64_t* calls_host, int32_t* n_sections) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    API_CK(ctx, cudaSetDevice(c.device));
    if (mode == 0) { c.prof.collect(); c.prof.on = false; return IPC_OK; }
    if (mode == 1) { c.prof.reset(); c.prof.on = true; return IPC_OK; }
    if (mode != 2) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_profile: mode must be 0, 1 or 2");
    c.prof.collect();
    int n = 0;
    for (int i = 0; i < Profiler::kMax && c.prof.names[i]; ++i) {
        if (n < max_sections) {
            if (names_host) {
                strncpy(names_host + 32 * n, c.prof.names[i], 31);
                names_host[32 * n + 31] = 0;
            }
            if (ms_host) ms_host[n] = c.prof.ms[i];
            if (calls_host) calls_host[n] = c.prof.calls[i];
        }
        ++n;
    }
    if (n_sections) *n_sections = n;
    return IPC_OK;
}

ipc_status ipc_contact_pass_kernels(ipc_ctx* ctx, int64_t* kernels_host) {
    if (!ctx || !kernels_host) return IPC_ERR_ARG;
    *kernels_host = ctx->c.cp_graph.exec ? ctx->c.cp_graph.kernels : -1;
    return IPC_OK;
}

static ipc_status newton_status(ipc_ctx* ctx, int status) {
    switch (status) {
        case 0: return IPC_OK;
        case 3: return fail_ctx(ctx, IPC_ERR_INFEASIBLE, "ipc_newton_step: infeasible (master motion blocked, "
                                                         "inverted tet or no admissible start)");
        case 5: return fail_ctx(ctx, IPC_ERR_NOT_CONVERGED, "ipc_newton_step: max_newton reached");
        default: return fail_ctx(ctx, IPC_ERR_LINESEARCH, "ipc_newton_step: line search exhausted max_halvings");
    }
}

static ipc_status step_checks(ipc_ctx* ctx) {
    Ctx& c = ctx->c;
    if (c.nt == 0 && c.h_mtets.empty()) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_newton_step: the scene has no tets");
    if (!(c.prm.h > 0.0) || !(c.prm.density > 0.0) || !(c.prm.youngs > 0.0) ||
        !(c.prm.poisson > -1.0 && c.prm.poisson < 0.5) || c.prm.max_newton < 0 || c.prm.max_pcg < 1 ||
        c.prm.max_halvings < 0)
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_newton_step: invalid h, material or iteration limits");
    return IPC_OK;
}

ipc_status ipc_set_master_body(ipc_ctx* ctx, const ipc_master_body* body) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!body || (body->n_mtet > 0 && !body->m_tets) || body->n_mtet < 0)
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_set_master_body: NULL body or tets");
    if (c.n_env != 1) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_set_master_body: one environment only");
    if (c.newton) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_set_master_body: the time stepper already exists");
    for (int64_t i = 0; i < 4 * body->n_mtet; ++i)
        if (body->m_tets[i] < 0 || body->m_tets[i] >= c.nmv)
            return fail_ctx(ctx, IPC_ERR_ARG, "ipc_set_master_body: m_tets index out of range");
    if (c.nv + c.nmv >= ((int64_t)1 << 30) || c.nt + body->n_mtet >= ((int64_t)1 << 27))
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_set_master_body: system too large");
    c.h_mtets.assign(body->m_tets, body->m_tets + 4 * body->n_mtet);
    if (body->m_dirichlet) c.h_mdir.assign(body->m_dirichlet, body->m_dirichlet + c.nmv);
    else c.h_mdir.assign(c.nmv, 0);
    c.joint_radius = body->pattern_radius;
    c.joint = true;
    return IPC_OK;
}

ipc_status ipc_newton_step_joint(ipc_ctx* ctx, double* x_dev, double* v_dev, const double* f_ext_dev,
                                 ipc_step_stats* stats) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.joint) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_newton_step_joint: no master body (ipc_set_master_body)");
    if (!x_dev || !v_dev) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_newton_step_joint: NULL x or v");
    const ipc_status chk = step_checks(ctx);
    if (chk != IPC_OK) return chk;
    API_CK(ctx, cudaSetDevice(c.device));
    const auto t_start = std::chrono::steady_clock::now();
    API_CK(ctx, newton_setup(c));
    int status = 0;
    ipc_step_stats st{};
    const cudaError_t e = newton_run(c, x_dev, v_dev, nullptr, nullptr, &st, &status, f_ext_dev);
    if (e != cudaSuccess && c.newton && c.newton->joint_miss) {
        cudaGetLastError();
        return fail_ctx(ctx, IPC_ERR_CAPACITY, "ipc_newton_step_joint: a contact block fell outside the "
                                               "slave-master block pattern (raise pattern_radius)");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ipc_newton_step_joint");
    st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = st;
    if (status == 0) ++c.step_count;
    return newton_status(ctx, status);
}

ipc_status ipc_newton_step_envs(ipc_ctx* ctx, double* x_dev, double* v_dev, const double* xm_next_dev,
                                const double* dx_pred_dev, ipc_step_stats* stats_host, int32_t* status_host) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    if (c.joint) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_newton_step: the context has a master body "
                                                   "(ipc_newton_step_joint)");
    if (!x_dev || !v_dev) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_newton_step: NULL x or v");
    if (c.nt == 0) return fail_ctx(ctx, IPC_ERR_ARG, "ipc_newton_step: the scene has no tets");
    if (!(c.prm.h > 0.0) || !(c.prm.density > 0.0) || !(c.prm.youngs > 0.0) ||
        !(c.prm.poisson > -1.0 && c.prm.poisson < 0.5) || c.prm.max_newton < 0 || c.prm.max_pcg < 1 ||
        c.prm.max_halvings < 0)
        return fail_ctx(ctx, IPC_ERR_ARG, "ipc_newton_step: invalid h, material or iteration limits");
    API_CK(ctx, cudaSetDevice(c.device));
    const auto t_start = std::chrono::steady_clock::now();
    API_CK(ctx, newton_setup(c));
    const int ne = c.n_env;
    std::vector<int> status(ne, 0);
    std::vector<ipc_step_stats> st(ne);
    const cudaError_t e = newton_run(c, x_dev, v_dev, xm_next_dev, dx_pred_dev, st.data(), status.data(), nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ipc_newton_step");
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    int first_bad = 0;
    for (int k = 0; k < ne; ++k) {
        st[k].ms_total = ms;
        if (stats_host) stats_host[k] = st[k];
        if (status_host) status_host[k] = status[k] == 0 ? IPC_OK : status[k] == 3 ? IPC_ERR_INFEASIBLE
                                                         : status[k] == 5 ? IPC_ERR_NOT_CONVERGED
                                                                          : IPC_ERR_LINESEARCH;
        if (!first_bad && status[k]) first_bad = status[k];
    }
    if (!first_bad) ++c.step_count;
    return newton_status(ctx, first_bad);
}

ipc_status ipc_newton_step(ipc_ctx* ctx, double* x_dev, double* v_dev, const double* xm_next_dev,
                           const double* dx_pred_dev, ipc_step_stats* stats) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx->c;
    const int ne = std::max(c.n_env, 1);
    std::vector<ipc_step_stats> st(ne);
    const ipc_status r = ipc_newton_step_envs(ctx, x_dev, v_dev, xm_next_dev, dx_pred_dev, st.data(), nullptr);
    if (stats && (r == IPC_OK || r == IPC_ERR_INFEASIBLE || r == IPC_ERR_NOT_CONVERGED || r == IPC_ERR_LINESEARCH)) {
        // several environments: counts summed, newton_iters and residual the
        // largest, alpha0 / last_alpha the smallest, energy summed,
        // pred_used the number of environments that used the prediction
        ipc_step_stats a = st[0];
        for (int k = 1; k < ne; ++k) {
            const ipc_step_stats& b = st[k];
            a.newton_iters = std::max(a.newton_iters, b.newton_iters);
            a.pcg_iters_total += b.pcg_iters_total;
            a.line_search_halvings += b.line_search_halvings;
            a.residual = std::max(a.residual, b.residual);
            a.res0 = std::max(a.res0, b.res0);
            a.alpha0 = std::min(a.alpha0, b.alpha0);
            a.last_alpha = std::min(a.last_alpha, b.last_alpha);
            a.energy += b.energy;
            a.pred_used += b.pred_used;
        }
        *stats = a;
    }
    return r;
}

}  // extern "C"

namespace gmcp {
// errors of the context-free entry points (the dual-mesh mapper), read by
// ipc_last_error(NULL)
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace gmcp

// gmcp_internal.cuh -- internal types shared by the libgmcp translation units.
//
// Layout in HBM (all device arrays owned by the context unless noted):
//   positions            caller-owned FP64 [n][3] (x, y, z per vertex)
//   slave / master tris  int32 [n][3]; master edges int32 [n][2] sorted (a<b)
//   per-slave-tri output energy (FP64), gradient coefficients G[3], Hessian
//                        coefficients S[6] and the frozen normal n[3] (FP64
//                        or FP32 by precision), written by the sample kernel
//                        and read by the deterministic gathers
//   candidate lists      fixed-capacity slots per slave triangle, sorted
//   broad-phase grid     dense uniform grid per environment, counting-sorted
//                        master triangle ids per cell
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "gmcp.h"

namespace gmcp {

// ------------------------------------------------------------------------
// device buffers
// ------------------------------------------------------------------------
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    cudaError_t alloc(size_t count) {
        release();
        if (count == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), count * sizeof(T));
        if (e != cudaSuccess) { p = nullptr; return e; }
        n = count;
        return cudaSuccess;
    }
    cudaError_t ensure(size_t count) { return count <= n ? cudaSuccess : alloc(count); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    cudaError_t upload(const T* host, size_t count, cudaStream_t s) {
        cudaError_t e = ensure(count);
        if (e != cudaSuccess || count == 0) return e;
        return cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, s);
    }
};

// ------------------------------------------------------------------------
// read-only scene view passed to kernels by value
// ------------------------------------------------------------------------
struct SceneView {
    int32_t nv, ns, nmv, nmt, nme, nse, n_env;
    const int32_t* stri;          // [ns][3]
    const int32_t* mtri;          // [nmt][3]
    const int32_t* medge;         // [nme][2]
    const int32_t* me_tri_off;    // [nme+1] master edge -> adjacent tris
    const int32_t* me_tri;
    const int32_t* mv_tri_off;    // [nmv+1] master vertex -> adjacent tris
    const int32_t* mv_tri;
    const int32_t* mtri_own_edge; // [nmt][3] edges owned by the tri (lowest adjacent id), -1
    const int32_t* mtri_own_vert; // [nmt][3]
    const int32_t* stri_own_vert; // [ns][3] slave surface vertices owned by the tri
    const int32_t* stri_own_edge; // [ns][3] slave edges owned by the tri (ids into sedge)
    const int32_t* sedge;         // [nse][2]
    const int32_t* stri_env;      // [ns]
    const int32_t* mtri_env;      // [nmt]
    const int32_t* mvert_env;     // [nmv]
    const double* X;              // pad rest [nv][3]
    const double* Y0;             // master at t = 0 [nmv][3]
    const double* srest_box;      // [ns][6] rest box of slave tris (lo xyz, hi xyz)
    const double* mrest_box;      // [nmt][6] rest box of master tris
    // the same boxes in FP32 rounded outward (lo down, hi up), and each
    // master vertex's rest position as such a box: certain lower bounds of
    // rest distances
    const float* srest_box_f;     // [ns][6]
    const float* mrest_box_f;     // [nmt][6]
    const float* mvrest_box_f;    // [nmv][6]
    // broad-phase grid, one dense box of cells per environment
    const double* grid_org;       // [n_env][3]
    const double* grid_inv;       // [n_env] 1 / cell size
    const int32_t* grid_dim;      // [n_env][3]
    const int64_t* grid_off;      // [n_env+1] first cell of each env
    const float* grid_org_f;      // [n_env][3] the same origin and inverse cell size
    const float* grid_inv_f;      // [n_env]    rounded to FP32 (conservative cell ranges)
    double margin;                // coarse-test slack (covers rounding of grown boxes)
};

struct Params {
    int precision;
    double dhat, kappa, kappa_edge, kappa_point, delta_T, delta_e;
    int L, nk;
    double dhat_guard, kappa_guard;
    double ccd_slack;
    int ccd_max_iter;
    int face_clip;         // 1: the paper's clipped-overlap face samples (ipc_params.face_sampler)
    double inv_dhat;       // 1 / dhat
    float far_r2_f;        // (dhat 1.2/0.9)^2 rounded up to FP32 and raised by 1e-6: rest boxes whose
                           // certain FP32 distance bound reaches it are rest-far in FP64 too
    // FP32 copies for the certified FP32 items of the mixed path: the
    // stiffnesses, the gamma radii, dhat as a pair (hi + lo) and 1 / dhat
    float kappa_f, kappa_edge_f, kappa_point_f, delta_T_f, delta_e_f, dhat_hi, dhat_lo, inv_dhat_f;
};

// Candidate list storage: fixed capacity per slave triangle.
struct CandView {
    int32_t cap_f, cap_e, cap_p;
    int32_t* face;      // [ns][cap_f]
    int32_t* edge;      // [ns][cap_e]
    int32_t* point;     // [ns][cap_p]
    int32_t* count;     // [ns][4]: face, edge, point, pad
    int32_t* active;    // [ns] slave tris with at least one candidate
    int32_t* n_active;  // scalar
    int32_t* overflow;  // [3] max count seen per kind (for regrowth)
    int32_t* work;      // work counter of the sample kernel (reset before each launch)
};

// Dynamic work distribution for persistent warps: lane 0 takes the next item
// index from a global counter and broadcasts it (all lanes must call).
__device__ __forceinline__ int next_item(int32_t* counter, int lane) {
    int i = 0;
    if (lane == 0) i = atomicAdd(counter, 1);
    return __shfl_sync(0xffffffffu, i, 0);
}
// the same, g consecutive items at a time (returns the first)
__device__ __forceinline__ int next_items(int32_t* counter, int lane, int g) {
    int i = 0;
    if (lane == 0) i = atomicAdd(counter, g);
    return __shfl_sync(0xffffffffu, i, 0);
}

// ------------------------------------------------------------------------
// section profiler: CUDA events around named groups of launches on the
// context stream; elapsed times are collected when the caller asks
// ------------------------------------------------------------------------
struct Profiler {
    static constexpr int kMax = 16;
    bool on = false;
    const char* names[kMax] = {nullptr};
    double ms[kMax] = {0};
    long long calls[kMax] = {0};
    struct Pending { int sec; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    int sec(const char* name) {
        for (int i = 0; i < kMax; ++i) {
            if (names[i] == name) return i;
            if (!names[i]) { names[i] = name; return i; }
        }
        return kMax - 1;
    }
    void collect() {
        for (auto& p : pending) {
            float t = 0.f;
            cudaEventSynchronize(p.b);
            cudaEventElapsedTime(&t, p.a, p.b);
            ms[p.sec] += t;
            calls[p.sec] += 1;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
    void reset() {
        collect();
        for (int i = 0; i < kMax; ++i) { ms[i] = 0; calls[i] = 0; }
    }
    ~Profiler() {
        for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

struct ProfScope {
    Profiler& P;
    cudaStream_t s;
    int sec = -1;
    cudaEvent_t a{}, b{};
    ProfScope(Profiler& p, cudaStream_t st, const char* name) : P(p), s(st) {
        if (!P.on) return;
        sec = P.sec(name);
        a = P.get(); b = P.get();
        cudaEventRecord(a, s);
    }
    ~ProfScope() {
        if (sec < 0) return;
        cudaEventRecord(b, s);
        P.pending.push_back({sec, a, b});
    }
};

// ------------------------------------------------------------------------
// time-stepper state (built on the first ipc_newton_step): tet data, the
// global block pattern (vertex adjacency through tets, plus the diagonal and
// the contact pattern) with per-block contribution lists, and the solver's
// vectors
// ------------------------------------------------------------------------
// A segmented sum: blocks of 2048 elements counted from each segment's
// (environment's) first element; per block: segment, first element, end,
// first block of the segment.  With one segment the blocks and the order of
// the sums are those of reduce_sum.
struct SegRed {
    int64_t nblk = 0;
    DBuf<int4> blk;
    DBuf<int32_t> nblk_env;    // [n_env] blocks of each segment
    DBuf<int32_t> first_blk;   // [n_env] first block of each segment
};

// per-environment Newton scalars ([n_env][kES] doubles)
constexpr int kES = 64;
enum : int {
    kEsEc = 0, kEsEe = 1, kEsE = 2, kEsG2 = 3, kEsEin = 4, kEsGp = 5,
    kEsE8 = 8,      // [8] line-search totals
    kEsEin8 = 16,   // [8] inertia terms
    kEsEe8 = 24,    // [8] elastic energies
    kEsEc8 = 32,    // [8] lagged contact energies
    kEsAl = 40,     // [8] the step sizes being tried
    kEsFe = 48      // [8] elastic energies of the start-point halvings
};

struct NewtonState {
    double mu = 0, lam = 0;
    int64_t nnzb = 0;
    // the system's vertices and tets: the pad's, or (joint step with a
    // deformable master) the pad's followed by the master body's
    bool joint = false;
    int64_t nsys = 0, ntsys = 0;
    DBuf<double> Xsys;                   // [nsys][3] rest positions
    const double* fext = nullptr;        // external nodal forces of the current step (joint), or NULL
    // joint step: the summed master blocks at their pattern positions
    DBuf<double> xvals;                  // [nnzb][9] master blocks (FP64, unscaled), zero elsewhere
    bool joint_miss = false;             // a contact block fell outside the pattern
    DBuf<int32_t> tets;                  // [nt][4]
    DBuf<double> Dminv, vol, mass;       // [nt][9], [nt], [nv]
    DBuf<uint8_t> dir;                   // [nv]
    DBuf<int32_t> vte_off, vte;          // vertex -> tet corner (t*4+a)
    DBuf<int32_t> rp, ci;                // block pattern (CSR)
    int64_t nslice = 0, ngroups = 0;     // sliced-ELL storage of the blocks (i, j >= i): 32 rows per slice
    int64_t nlgroups = 0;                // groups of the lower lists (blocks j < i, read transposed)
    int64_t nvp = 0;                     // PCG vector rows: nv padded to a multiple of 4 (padding zero)
    DBuf<int32_t> goff;                  // [nslice + 1] first group (32 stored blocks) of each slice
    DBuf<int32_t> gslice;                // [ngroups] slice of each group
    DBuf<int32_t> sci;                   // [ngroups][32] column of each stored block, -1 for padding
    DBuf<int32_t> llen;                  // [nv] blocks j < i of each row
    DBuf<int32_t> lgoff;                 // [nslice + 1] first lower group of each slice
    DBuf<int32_t> lcol, lmir;            // [nlgroups + 1][32] column j, and group * 32 + lane of block (j, i)
    DBuf<int32_t> bt_off, bt;            // block -> (t*16 + a*4 + b)
    DBuf<int32_t> cmap;                  // block -> contact block or -1
    DBuf<double> tE, tG, tE8;            // per-tet energy [nt], gradient [nt][12], energies [8][nt]
                                         // (mixed path: tG holds the gradient as FP32 pairs hi, lo)
    DBuf<float> Dm2, vol2;               // mixed path: Dm^-1 [nt][9] and volumes [nt] as FP32 pairs
    DBuf<float> uh4, ul4, ph4, pl4;      // mixed path: x - X and a direction p split into pairs [nv][4] each
    DBuf<double> tH64;                   // per-tet Hessian, 10 blocks [nt][10][10] (FP64 path)
    DBuf<float> tH32;                    // the same in FP32, [nt][10][12] (mixed path)
    DBuf<double> A64, Pinv;              // global matrix [ngroups][288] (FP64 path), P^-1 [nvp][9]
    DBuf<float> A32, p32, r32, z32, Ap32, Pinv32;   // FP32 matrix and PCG vectors (mixed path; z [nvp][4], p [2][nvp][4])
    DBuf<float> xh32, xl32;              // mixed-path PCG solution as a float pair hi + lo [3 nvp]
    DBuf<double> part;                   // PCG per-block partial sums [2][blocks]
    DBuf<unsigned> counters;             // PCG last-block counters
    DBuf<double> r, z, p, Ap, w;         // PCG vectors r, z, Ap [3 nvp], p [nvp][4]; w [3 nv]
    DBuf<double> xhat, xt, G, dirn, tmp, P, dP, xi, xl;   // [3 nv]
    DBuf<double> cgrad64;                // contact gradient [3 nv] (FP64 path)
    DBuf<float> cgrad32;                 // contact gradient [3 nv] (mixed path)
    DBuf<double> xm, dxm;                // current master [nmv][3] and its motion
    DBuf<double> ein8;                   // [8][nv] inertia energy terms
    DBuf<double> triE8;                  // [8][ns] lagged contact energies
    DBuf<double> scal;                   // solver scalars
    // environments: the PCG works per environment (own scalars, stopping,
    // reductions), on rows padded per environment to a multiple of four
    int n_env = 1;
    DBuf<int32_t> vprow;                 // [nv] padded PCG row of each vertex
    DBuf<int32_t> prow_v;                // [nvp] vertex of each padded row, -1 for padding
    int64_t nblk_v = 0, nblk_p = 0;      // blocks of the vertex-row and padded-row kernels
    DBuf<int4> blk_v, blk_p;             // per block: env, first row, end row, first block of the env
    std::vector<int32_t> h_env_nblk_v, h_env_nblk_p;   // blocks per env
    DBuf<int32_t> env_nblk_v, env_nblk_p;
    DBuf<double> escal;                  // [n_env][kEnvScal] per-environment PCG scalars
    // environments of at most kSmallRows rows: solved by one block each
    int64_t n_small = 0;
    DBuf<int4> small_envs;               // [n_small] env, first row, end row
    DBuf<int32_t> env_small;             // [n_env] 1 = small
    DBuf<double> sm64;                   // their PCG vectors r, z, p, Ap (FP64 in both paths)
    DBuf<int32_t> vert_env, tet_env;     // [nv], [nt] environment of each vertex / tet
    SegRed seg_v3, seg_v, seg_t, seg_s;  // segmented sums over 3 nv, nv, nt, ns elements
    DBuf<double> seg_part;               // block partials of the segmented sums
    DBuf<double> es;                     // [n_env][kES] per-environment Newton scalars
    DBuf<int32_t> ebad;                  // [n_env] inverted-tet flag per environment
    DBuf<double> ealpha;                 // [n_env] step size per environment
    DBuf<double> eal;                    // [n_env][8] step sizes tried per environment
    DBuf<int32_t> emask;                 // [4][n_env] environment masks
    DBuf<unsigned long long> ebits;      // [n_env][2] step bounds (linearised, additive CCD) as bits
    DBuf<double> ezero;                  // one 0.0
    std::vector<double> h_lbar;          // cube root of each environment's mean tet volume
    std::vector<uint8_t> h_has_dir;      // environment has Dirichlet vertices
    std::vector<uint8_t> h_dir_surf;     // ... among the vertices of its contact surfaces
    // pinned host copies (one allocation, h_pin)
    void* h_pin = nullptr;
    double* h_es = nullptr;              // [n_env][kES]
    double* h_eal = nullptr;             // [n_env][8]
    double* h_ealpha = nullptr;          // [n_env]
    unsigned long long* h_ebits = nullptr;   // [n_env][2]
    int32_t* h_emask = nullptr;          // [4][n_env]
    int32_t* h_ebad = nullptr;           // [n_env]
    DBuf<unsigned> ecount;               // [3][n_env] last-block counters (init/spmv, update, spare)
    double* h_pcg = nullptr;             // pinned [n_env][4]: break, done, iterations (host reads)
    ~NewtonState() {
        if (h_pcg) cudaFreeHost(h_pcg);
        if (h_pin) cudaFreeHost(h_pin);
    }
};

// A captured CUDA graph and the arguments it was captured with.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<uintptr_t> key;
    int64_t kernels = 0;           // kernel nodes of the captured graph
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
        kernels = 0;
    }
    ~GraphCache() { reset(); }
};

// Pinned host storage for every host <-> device transfer a captured graph
// performs (a graph replays copies from and to fixed host addresses).
struct PinnedIO {
    unsigned long long init[2];   // alpha_lin / alpha_accd initial bits
    unsigned long long bits[2];
    long long ctr_ccd[4];
    long long counts[8];
    int32_t flags[32];
    double energy;
    double pcg[4];
};

// slave tris whose query box meets a non-empty cell, with their boxes
struct QueryBufs {
    DBuf<int32_t> tri, cell;
    DBuf<double> box;
    DBuf<float> boxf, vboxf;
};

struct WarmStart;              // learned warm start (warmstart.cu)
void ws_destroy(WarmStart* w);

// misc_i32 slots used by the contact evaluation's touched-output lists
constexpr int kSlotPass = 18;    // contact evaluations so far (stamps of this one)
constexpr int kSlotHPass = 19;   // those that assembled the Hessian
constexpr int kSlotVCount = 20;  // vertices listed in this evaluation
constexpr int kSlotBCount = 21;  // [2] blocks listed, by Hessian-pass parity
constexpr int kSlotItemList = 23; // face items that passed the FP32 pre-tests (listed from the front)
constexpr int kSlotItemList2 = 24; // edge and point items that passed (listed from the back)
constexpr int kSlotItemMid = 25;   // face items past the FP32 pre-filter (listed from the front)
constexpr int kSlotItemMid2 = 26;  // edge and point items past it (listed from the back)

// ------------------------------------------------------------------------
// the context
// ------------------------------------------------------------------------
struct Ctx {
    ipc_params prm;
    Params P;
    cudaStream_t stream = nullptr;
    std::string err;
    int device = 0;

    // sizes
    int64_t nv = 0, nt = 0, ns = 0, nmv = 0, nmt = 0, nme = 0, nse = 0;
    int n_env = 0;
    int64_t n_cells = 0;

    // host copies needed for topology
    std::vector<int64_t> env_vert_off, env_tet_off, env_stri_off, env_mvert_off, env_mtri_off;

    // static device topology
    DBuf<int32_t> stri, mtri, medge, me_tri_off, me_tri, mv_tri_off, mv_tri;
    DBuf<int32_t> mtri_own_edge, mtri_own_vert, stri_own_vert, stri_own_edge, sedge;
    DBuf<int32_t> stri_env, mtri_env, mvert_env;
    DBuf<double> X, Y0, srest_box, mrest_box;
    DBuf<float> srest_box_f, mrest_box_f, mvrest_box_f;
    // mixed path, per pass: the middle sample stage's inputs computed once per
    // triangle or sample instead of once per item (see k_tri_frame, k_mtri_e32)
    DBuf<double> tri_mid64;                     // [n_active][4]: ns . dx_a (3) and the sum of their magnitudes
    DBuf<float> tri_mid32;                      // [n_active][12]: unit normal, x1 - x0, x2 - x0 in FP32
    DBuf<float> mtri_e32;                       // [nmt][8]: y1 - y0, y2 - y0 of each master tri in FP32
    DBuf<float> mtri_pre;                       // [nmt][24]: each master tri's part of the FP32 face pre-filter
    DBuf<double> grid_org, grid_inv;
    DBuf<float> grid_org_f, grid_inv_f;
    DBuf<int32_t> grid_dim;
    DBuf<int64_t> grid_off;
    double margin = 0.0;

    // gather topology: vertex -> (tri, corner), contact BSR pattern and its
    // per-block contribution lists
    DBuf<int32_t> vt_off, vt_ent;              // [nv+1], entries tri*4+corner
    DBuf<int32_t> cb_row, cb_col;              // contact BSR [nv+1], [nnzb]
    DBuf<int32_t> cb_src_off, cb_src;          // [nnzb+1], entries tri*16+a*4+b
    int64_t cb_nnzb = 0;

    // per-call broad-phase buffers
    DBuf<int4> mcell;                           // [nmt] lowest cell (x, y, z) and env
    DBuf<float> mboxf;                          // conservative FP32 master boxes
    DBuf<float> mboxf_in;                       // FP32 boxes inside the exact static master boxes
    DBuf<int2> ccd_pairs;                       // primitive pairs for ACCD
    DBuf<int2> coarse_pairs, coarse_swept;      // (query entry, master) pairs: contact, swept
    int32_t cap_ccd = 0, cap_coarse = 0, cap_coarse_swept = 0;
    QueryBufs qcontact, qswept;                 // filtered slave tris of the two queries
    int64_t n_svert = 0;
    DBuf<int32_t> svert;                        // [n_svert] vertices of slave tris (ascending)
    DBuf<float> vbound_c;                       // [nv][8] per-vertex FP32 bounds for the contact query
    DBuf<float> vbound_s;                       // [nv][12] per-vertex FP32 swept bounds for the swept query
    cudaStream_t ccd_stream = nullptr;          // the swept query's branch of a contact pass
    cudaStream_t h2d_stream = nullptr;          // host-input passes: the displacements' copy
    cudaEvent_t ev_xin = nullptr, ev_dxin = nullptr;   // positions copied / displacements scattered
    DBuf<double> xs_stage, dxs_stage;           // [n_svert][3] host inputs on the device
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t aux_stream = nullptr;          // touched-output lists beside the sample evaluation
    cudaEvent_t ev_touch0 = nullptr, ev_touch1 = nullptr, ev_samples = nullptr;
    cudaEvent_t ev_master = nullptr;   // the master's FP32 tables done on the side stream
    cudaEvent_t ev_mfork = nullptr;    // a contact pass's start, for that side stream
    bool side_master = false;          // set while a contact pass has forked the side stream
    bool master_pre = false;           // the tables of this pass are already enqueued (ev_master)
    // the face pre-filter reads a per-master-triangle table (built each pass
    // over every master triangle) instead of forming each triangle's part
    // per item; set after a contact pass whose sample items outnumbered the
    // master triangles eightfold (results are the same either way)
    bool use_mtri_pre = false;
    // the master triangles' FP32 edges are tabled per pass only when the
    // last pass had at least one face item per master triangle (else the
    // middle stage forms them from xm: the same values)
    bool use_mtri_e32 = false;
    // master entries of the samples (gradient rows and Hessian blocks of the
    // master vertices) and their counting sort by destination row
    int64_t ml_cap = 0;
    DBuf<int32_t> ml_ij;                 // [cap][2] (row, col), col -1 = a gradient row
    DBuf<double> ml_blk;                 // [cap][9]
    DBuf<unsigned long long> ml_count;   // entries needed
    DBuf<int32_t> ml_cnt, ml_off, ml_cur, ml_perm, ml_tmp, ml_err;
    DBuf<int32_t> cell_cnt, cell_start, cell_ent;
    DBuf<int32_t> scan_tmp;
    DBuf<int32_t> cand_face, cand_edge, cand_point, cand_count, active, misc_i32;
    int32_t cap_f = 32, cap_e = 32, cap_p = 16;

    // per-call sample outputs
    DBuf<double> tri_E;
    DBuf<double> tri_frame;                     // [n_active][8] frames of the active slave tris
    DBuf<int32_t> tri_items;                    // [n_active][2] first item slot, item count
    DBuf<int32_t> item_owner;                   // [cap_items] active index of each item slot
    DBuf<double> item_rd;                       // [cap_items][2] energy, step bound
    DBuf<unsigned char> item_rt;                // [cap_items][5] c1, c2, b (FP32 or FP64)
    DBuf<int32_t> item_list;                    // [cap_items] slots that passed the pre-tests
    DBuf<uint32_t> item_mask;                   // [cap_items / 32 + 1] slots that hold a record
    DBuf<int32_t> item_mid;                     // [cap_items] slots past the FP32 pre-filter
    DBuf<float> tri_f32;                        // [n_active][64] FP32 samples, normal, vertices (env frame)
    DBuf<float> ym32;                           // [nmv][4] master vertices in FP32 (env frame)
    int64_t cap_items = 0;
    // outputs touched by the active triangles (pass stamps and lists)
    DBuf<int32_t> tri_stamp, v_stamp, b_stamp;  // [ns], [nv], [cb_nnzb]
    DBuf<int32_t> v_list, b_list0, b_list1;     // [nv], [cb_nnzb] x 2
    DBuf<int32_t*> b_lists;                     // device copy of {b_list0, b_list1}
    DBuf<double> tri_G64, tri_S64, tri_n64;
    DBuf<float> tri_G32, tri_S32, tri_n32;
    DBuf<double> cb_val64;
    DBuf<float> cb_val32;
    DBuf<double> red_tmp;                       // reduction partials
    DBuf<unsigned long long> u64_tmp;           // alpha minima
    DBuf<long long> i64_tmp;                    // counters
    DBuf<double> dxm;                           // master displacement for CCD
    DBuf<double> scal;                          // device scalars (energy, ...)

    // pinned host scratch for scalars
    double* h_scalars = nullptr;
    long long* h_counts = nullptr;

    Profiler prof;

    // launch shapes chosen by the autotuner (ipc_autotune); results do not
    // depend on them
    int tune_samples_bpsm = 8;     // k_samples blocks per SM (256 threads)
    int tune_query_bpsm = 8;       // persistent query / CCD blocks per SM

    // CUDA graphs
    bool graphs = false;
    GraphCache cp_graph;           // ipc_contact_pass
    GraphCache pcg_graph;          // one PCG chunk
    cudaStream_t cap_stream = nullptr;   // private stream graphs are captured on
    PinnedIO* pin = nullptr;

    // host copies kept for the time stepper
    std::vector<int32_t> h_tets;
    std::vector<uint8_t> h_dir;
    std::vector<double> h_X;
    std::vector<double> h_Y0;                  // master rest positions
    std::vector<int32_t> h_stri, h_mtri;       // slave and master triangles
    // deformable master (joint step): the master body's tets and Dirichlet
    // flags, and the radius of the slave-master block pattern
    bool joint = false;
    std::vector<int32_t> h_mtets;
    std::vector<uint8_t> h_mdir;
    double joint_radius = 0.0;
    std::vector<int32_t> h_cb_row, h_cb_col;
    std::unique_ptr<NewtonState> newton;
    std::unique_ptr<WarmStart, void (*)(WarmStart*)> ws{nullptr, ws_destroy};
    int64_t step_count = 0;        // time steps completed by ipc_newton_step (saved in snapshots)

    SceneView view() const;
    CandView cand() {
        CandView c;
        c.cap_f = cap_f; c.cap_e = cap_e; c.cap_p = cap_p;
        c.face = cand_face.p; c.edge = cand_edge.p; c.point = cand_point.p;
        c.count = cand_count.p; c.active = active.p;
        c.n_active = misc_i32.p; c.overflow = misc_i32.p + 1; c.work = misc_i32.p + 4;
        return c;
    }
};

// ------------------------------------------------------------------------
// launchers implemented in the .cu files
// ------------------------------------------------------------------------
// broadphase.cu
cudaError_t bp_init_constants(const double* rule_l1l2);
// lazy: size the entries for the worst rigid pose instead of reading the
// exact total back (no synchronisation); overflow sets misc_i32[12]
cudaError_t bp_build_grid(Ctx& c, const double* xm, const double* dxm, bool swept, bool lazy = false);
cudaError_t bp_query_contact(Ctx& c, const double* x, const double* xm, bool lazy = false);
// ACCD over swept pairs; reuse_grid: the cells already hold the master
// triangles at xm0 (static master, same call), so the swept grid equals them
cudaError_t bp_ccd_accd(Ctx& c, const double* x, const double* dx, const double* xm0,
                        const double* dxm, unsigned long long* alpha_bits, long long* counters,
                        bool reuse_grid = false, bool lazy = false, int alpha_stride = 0);
// the master's FP32 tables of the mixed path from xm on stream s (contact.cu)
cudaError_t master_tables(Ctx& c, const double* xm, cudaStream_t s);
// scan.cu
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                               size_t tmp_n, cudaStream_t s);
size_t scan_tmp_size(int64_t n);
// api.cu
// lazy: no synchronisation; the caller must check misc_i32[1..3] and [12]
cudaError_t run_candidates(Ctx& c, const double* x, const double* xm, bool lazy = false);
// contact.cu
cudaError_t contact_init_constants(const double* rule_l1l2);
// contact_eval also bounds the step (Eq. ccd) along dx / dxm into alpha_bits
// when dx is non-NULL
cudaError_t contact_eval(Ctx& c, const double* x, const double* xm, double* energy_dev,
                         void* grad_dev, bool want_hess, long long* counters,
                         const double* dx = nullptr, const double* dxm = nullptr,
                         unsigned long long* alpha_bits = nullptr);
cudaError_t contact_alpha_lin(Ctx& c, const double* x, const double* xm, const double* dx,
                              const double* dxm, unsigned long long* alpha_bits, int alpha_stride = 0);
cudaError_t reduce_sum(Ctx& c, const double* in, int64_t n, double* out, const int32_t* stamp = nullptr,
                       const int32_t* pass = nullptr);
int sm_count(int device);
// frozen-linear ("lagged") contact energy of the samples active at (x, xm),
// evaluated at x + alphas[j] p for j < na (na <= 8) into energies_dev[j]
// (FP64 in both precisions; energies_dev NULL: the per-triangle terms
// triE8 [na][ns] only); needs the candidate lists of (x, xm).
// alphas_stride > 0: a slave triangle of environment e uses
// alphas_dev[alphas_stride * e + j]; pm: the master's direction (a
// deformable master, NULL = static)
cudaError_t contact_lagged(Ctx& c, const double* x, const double* xm, const double* p,
                           const double* alphas_dev, int na, double* triE8, double* energies_dev,
                           int alphas_stride = 0, const double* pm = nullptr);
// slave-master (slave row) and master-master Hessian blocks of the active
// samples, appended in arbitrary order; *count receives the number needed;
// rows: also the master vertices' gradient rows, as entries (row, -1)
cudaError_t contact_master_hess(Ctx& c, const double* x, const double* xm, int32_t* ij, double* blk,
                                int64_t cap, unsigned long long* count, bool rows = false, bool blocks = true);
// the master entries of the samples at (x, xm) -- gradient rows, and with
// xvals the blocks too -- sorted by destination row (then by value) and
// summed in that order: row r (joint numbering) into rows_out[3 (r -
// row_base)] (FP32 or FP64), blocks (col >= row) into xvals at their place in
// the pattern (rp, llen, ci); *miss set when a block has no place
cudaError_t sorted_master_terms(Ctx& c, const double* x, const double* xm, int64_t nrows, int64_t row_base,
                                void* rows_out, bool rows_f32, const int32_t* rp, const int32_t* llen,
                                const int32_t* ci, double* xvals, bool* miss);
// newton.cu
cudaError_t newton_setup(Ctx& c);
// The Newton iteration runs per environment: each sum below is one
// fixed-order sum per environment, the same as over a scene holding that
// environment alone; the results go to N.es [n_env][kES].
// elastic energy per environment into es[kEsEe]; inverted-tet flags in N.ebad
cudaError_t nh_eval(Ctx& c, const double* x, bool want_hess);
// elastic energies at x + alphas_env[8 e + j] p (j < na <= 8) into es[slot +
// j]; +inf where a tet of the environment has J <= 0; delta: their change
// from x (per tet, against the energies of the last nh_eval at x)
cudaError_t nh_energy_multi(Ctx& c, const double* x, const double* p, const double* alphas_env, int na, int slot,
                            bool delta = false);
// inversion test alone: es[slot + j] = 0 where every tet of the environment
// keeps J > 0 at x + alphas_env[8 e + j] p (j < na <= 8), +inf where not (the
// same decision as nh_energy_multi's)
cudaError_t nh_feasible_multi(Ctx& c, const double* x, const double* p, const double* alphas_env, int na,
                              int slot);
// changes of the total energy from x to x + alphas_env[8 e + j] p into
// es[kEsE8 + j]; ee0: alphas_env[8 e] = 0
cudaError_t energy_batch(Ctx& c, const double* x, const double* p, const double* alphas_env, int na,
                         bool with_contact, bool ee0);
// es[kEsEc], es[kEsEe], es[kEsE], es[kEsG2] at x, the gradient N.G and
// optionally the matrix
// what assemble_system evaluates besides the energies and the gradient:
// nothing, the contact (and master) Hessian blocks, or every Hessian block
// and the global matrix
enum : int { kHessNone = 0, kHessContact = 1, kHessAll = 2 };
cudaError_t assemble_system(Ctx& c, const double* x, int hess);
// the elastic Hessian blocks and the global matrix at the x of the last
// assemble_system(c, x, kHessContact)
cudaError_t finish_hessian(Ctx& c, const double* x);
// a . b per environment (3 nv entries) into es[slot]
cudaError_t dot_env(Ctx& c, const double* a, const double* b, int slot);
// the master positions / direction that go with system positions x /
// direction p (the joint step's master rows, else the kinematic master /
// NULL); the joint step's master rows and blocks
const double* master_of(Ctx& c, const double* x);
const double* master_dir_of(Ctx& c, const double* p);
cudaError_t joint_master_terms(Ctx& c, const double* x, bool want_hess);
cudaError_t pcg_solve(Ctx& c, const double* b, double* xout, double rel_tol, int max_it, int* iters,
                      int* env_iters = nullptr);   // env_iters: [n_env] iterations per environment
// elementwise helpers
cudaError_t vec_axpy(Ctx& c, int64_t n, double a, const double* x, const double* p, double* out);
cudaError_t vec_xhat(Ctx& c, const double* x, const double* v, double* xhat);
cudaError_t vec_dir_delta(Ctx& c, const double* x, const double* xhat, double* dP);
cudaError_t vec_set_dir(Ctx& c, const double* src, double* dst);
cudaError_t vec_free_delta(Ctx& c, const double* P, const double* xi, double* dP);
cudaError_t vec_zero_dir(Ctx& c, double* p);
cudaError_t vec_velocity(Ctx& c, const double* x, const double* xt, double* v);
cudaError_t vec_neg(Ctx& c, int64_t n, const double* a, double* out);
// per environment (mask [n_env], nonzero = selected)
cudaError_t vec_axpy_env(Ctx& c, const double* x, const double* p, const double* alpha_env, const int32_t* mask,
                         double* out);   // out = x + alpha_env[e] p (selected), x (others)
cudaError_t vec_copy_env(Ctx& c, const double* src, const int32_t* mask, double* dst);   // selected only
cudaError_t vec_zero_env(Ctx& c, const int32_t* mask, double* a);                        // unselected only
cudaError_t vec_copy_master_env(Ctx& c, const double* src, const int32_t* mask, double* dst);   // master vertices
cudaError_t vec_velocity_env(Ctx& c, const double* x, const double* xt, const int32_t* mask, double* v);
// api.cu: the context behind an ABI handle
Ctx& ctx_of(ipc_ctx* h);
// errors of the context-free entry points, read by ipc_last_error(NULL) (api.cu)
void set_global_error(const std::string& msg);

// learned warm start: the state a snapshot carries (warmstart.cu)
struct WsState {
    double lr = 0, beta1 = 0, beta2 = 0, eps = 0, pos_scale = 0, disp_scale = 0, force_scale = 0;
    int64_t step = 0;                // Adam steps taken
    std::vector<float> P, M1, M2;    // FP32 parameters and Adam moments
};
// host copies of the network's parameters, moments and settings (c.ws set)
cudaError_t ws_state_get(Ctx& c, WsState* out);
// replace them (c.ws set, same parameter count) and refresh the BF16 copies
cudaError_t ws_state_set(Ctx& c, const WsState& in);
int64_t ws_param_count();

// Programmatic dependent launch for the kernels of the contact pass: each is
// launched with programmatic stream serialisation, so that its blocks are
// scheduled while its predecessor in the stream drains, and each begins with
// griddepcontrol.wait, which holds it until the predecessor has finished and
// its memory is visible.  Every such kernel waits before anything else, so a
// kernel's completion still implies that of every kernel before it in the
// stream.  Launched without the attribute, the wait is a no-op.
__device__ __forceinline__ void pass_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

}  // namespace gmcp

// integer atomic add on a signed 64-bit counter (two's complement wraps the same)
__device__ __forceinline__ void atomic_add_ll(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

#define GMCP_CUDA_TRY(expr)                                                          \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess) return _e;                                            \
    } while (0)

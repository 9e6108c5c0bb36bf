// warmstart.cu -- the learned warm start: a per-vertex MLP 32-256-256-256-3
// (ReLU) that predicts the correction of the plain predictor,
//   x^{t+1} ~ x^t + h v^t + s * y(features),
// trained on states the solver produces.  The two dense contractions per
// layer run on the 5th-generation tensor cores:
//   activations  C[m, n] = A[m, :] . W[n, :]   (M = vertices, N = 256, K = 32 | 256)
//   weight grads dW[o, i] = sum_m dZ[m, o] H[m, i]  (M = 256, N = 256 | 32, K = vertices)
// as tcgen05.mma kind::f16 (BF16 operands in shared memory, FP32 accumulators
// in tensor memory), issued by one thread, completion signalled through an
// mbarrier, accumulators read back with tcgen05.ld.  Operand tiles come in
// by TMA (cp.async.bulk.tensor) in the swizzled K-major layout (rows of 64
// or 32 BF16 values, 16-byte pieces permuted by the row index, 8-row groups
// 1024 or 512 B apart), through rings of shared-memory stages, with loads,
// MMAs and the epilogue in separate warps.  The 256 -> 3 head, bias sums and
// Adam run on the CUDA cores.  Every sum is in a fixed order, so training is
// deterministic.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gmcp_internal.cuh"

namespace gmcp {

struct WarmStart {
    int64_t n = 0, mp = 0;                 // vertices, padded to a multiple of 128
    double lr = 1e-3, beta1 = 0.9, beta2 = 0.999, eps = 1e-8;
    double pos_scale = 1, disp_scale = 1, force_scale = 1;
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    int64_t step = 0;
    // parameters: FP32 master copies, Adam moments, BF16 copies for the
    // tensor cores (W and W^T)
    DBuf<float> P, M1, M2, G;              // flattened [W1 b1 W2 b2 W3 b3 W4 b4]
    DBuf<__nv_bfloat16> W1, W2, W3, W2t, W3t;
    // activations
    DBuf<__nv_bfloat16> f, fT, h1, h2, h3, h1T, h2T, dz3, dz3T, dz2, dz2T, dz1T;
    DBuf<float> y, dy, part;              // FP32 partial sums (split-K weight gradients, head)
    DBuf<double> dpart;                   // FP64 per-block partial sums (mask, loss)
    DBuf<uint8_t> surf;
    DBuf<double> cgrad64;
    DBuf<float> cgrad32;
    DBuf<int> err;
    DBuf<double> scal;
};

namespace {

constexpr int kHid = 256, kIn = 32, kOut = 3;
// offsets into the flattened parameter vector
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
                  kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid,
                  kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kOut * kHid, kNParam = kOffB4 + kOut;

// ------------------------------------------------------------- tcgen05 ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;");
}
// bounded wait on an mbarrier phase; false when the limit is reached
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase) {
    const uint32_t a = smem_u32(mbar);
    for (long long it = 0; it < (1ll << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P1;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(phase));
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ----------------------------------------------------- activation GEMM ---
// C = epilogue(A W^T), A [mp][K] BF16 row-major, W [256][K] BF16 row-major
// (K-major), persistent over 128-row tiles with W resident in shared memory.
// EPI 0: + bias, ReLU.  EPI 1: times (mask > 0), mask [mp][256] BF16 (the
// previous layer's activation).  Writes C [mp][256] (if non-null) and
// C^T [256][mp] (if non-null).  The operand tiles are brought in by the
// tensor-memory accelerator (cp.async.bulk.tensor) in the swizzled K-major
// layout: each tile row holds KC = min(K, 64) BF16 values (128 or 64 bytes)
// with its 16-byte pieces permuted by the row index, the layout both TMA and
// the tcgen05 shared-memory descriptors name SWIZZLE_128B / SWIZZLE_64B.
// Roles: warp 0 loads (W once, then the A chunks of every tile into a ring
// of NST stages), warp 1 issues the MMAs (one thread), warps 2..9 run the
// epilogue out of two tensor-memory accumulators, so that loads, MMAs and
// the epilogue of three consecutive tiles overlap.  The MMAs of a tile run
// in increasing K, one K = 16 step at a time.
__device__ __forceinline__ uint64_t umma_desc_sw(uint32_t saddr, int swz_bytes) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                                   // leading offset: unused when swizzled
    d |= (uint64_t)(((8u * (uint32_t)swz_bytes) >> 4) & 0x3FFFu) << 32;  // 8-row groups apart
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(swz_bytes == 128 ? 2 : 4) << 61;         // SWIZZLE_128B | SWIZZLE_64B
    return d;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// 2D tiled TMA load of box (x, y) into shared memory, completing on mbar
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}

// 16 accumulator columns into r[] without waiting; tmem_ld_wait32 then
// waits for the outstanding loads and ties the 32 registers to that point
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait32(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i += 8)
        asm volatile("" : "+r"(r[i]), "+r"(r[i + 1]), "+r"(r[i + 2]), "+r"(r[i + 3]), "+r"(r[i + 4]),
                     "+r"(r[i + 5]), "+r"(r[i + 6]), "+r"(r[i + 7]));
}

// epilogue of one 128-row tile: this warp's 32 rows (TMEM lane quarter),
// columns [128 half, 128 half + 128), 32 columns per TMEM wait; the bias
// comes from shared memory
template <int K, int EPI>
__device__ __forceinline__ void act_epilogue_rows(uint32_t tacc, int quarter, int half, int64_t m0, int64_t mp,
                                                  const float* __restrict__ sbias,
                                                  const __nv_bfloat16* __restrict__ mask,
                                                  __nv_bfloat16* __restrict__ C, __nv_bfloat16* __restrict__ CT) {
    const int lane = threadIdx.x & 31;
    const int r = quarter * 32 + lane;
    const int64_t gr = m0 + r;
    for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 32) {
        uint4 mk[4];
        if (EPI == 1) {
            const uint4* mp4 = reinterpret_cast<const uint4*>(mask + gr * 256 + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) mk[q] = __ldg(mp4 + q);
        }
        uint32_t u[32];
        const uint32_t ta = tacc + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
        tmem_ld16_nowait(ta, u);
        tmem_ld16_nowait(ta + 16u, u + 16);
        tmem_ld_wait32(u);
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(u[i]);
        if (EPI == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i] + sbias[c0 + i], 0.0f);
        } else {
            const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(mk);
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (!(__bfloat162float(mb[i]) > 0.0f)) v[i] = 0.0f;
        }
        __align__(16) __nv_bfloat16 o[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) o[i] = __float2bfloat16_rn(v[i]);
        if (C) {
            uint4* dst = reinterpret_cast<uint4*>(C + gr * 256 + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
        }
        if (CT) {
#pragma unroll
            for (int i = 0; i < 32; ++i) CT[(int64_t)(c0 + i) * mp + gr] = o[i];
        }
    }
}

template <int K>
struct ActTma {
    static constexpr int KC = K < 64 ? K : 64;          // BF16 values per tile row (one swizzle span)
    static constexpr int SWZ = KC * 2;                  // bytes per tile row: 128 or 64
    static constexpr int NCH = K / KC;                  // K chunks
    static constexpr int NST = K >= 256 ? 5 : 8;        // A ring stages
    static constexpr uint32_t A_BYTES = 128u * SWZ;     // one A chunk (128 rows)
    static constexpr uint32_t W_BYTES = 256u * SWZ;     // one W chunk (256 rows)
    static constexpr size_t SMEM = (size_t)NCH * W_BYTES + (size_t)NST * A_BYTES + 1024 + 1024;  // + alignment, bias
    static constexpr int THREADS = 320;
};

template <int K, int EPI>
__global__ void __launch_bounds__(320, 1)
k_umma_act_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW, int64_t mp,
               const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask,
               __nv_bfloat16* __restrict__ C, __nv_bfloat16* __restrict__ CT, int* __restrict__ err) {
    using T = ActTma<K>;
    extern __shared__ uint8_t smem_raw[];
    // the swizzled tiles want 1024-byte aligned bases
    const uint32_t base_u = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((base_u + 1023u) & ~1023u) - base_u);
    uint8_t* sW = smem;                                  // NCH chunks of 256 rows
    uint8_t* sA = smem + T::NCH * T::W_BYTES;            // NST chunks of 128 rows
    float* sbias = reinterpret_cast<float*>(sA + T::NST * T::A_BYTES);   // [256] (EPI 0)
    __shared__ __align__(8) uint64_t full[T::NST], empty[T::NST], wfull, accf[2], acce[2];
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 1) tmem_alloc(&tslot, 512);
    if (EPI == 0)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) sbias[i] = bias[i];
    if (threadIdx.x == 0) {
        for (int i = 0; i < T::NST; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        mbar_init(&wfull, 1);
        for (int i = 0; i < 2; ++i) { mbar_init(&accf[i], 1); mbar_init(&acce[i], 8); }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int64_t ntiles = mp / 128;
    if (warp == 0) {
        if (lane == 0) {
            // producer
            mbar_expect_tx(&wfull, T::NCH * T::W_BYTES);
            for (int c = 0; c < T::NCH; ++c) tma_load_2d(sW + c * T::W_BYTES, &tmW, c * T::KC, 0, &wfull);
            uint32_t it = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int c = 0; c < T::NCH; ++c, ++it) {
                    const uint32_t st = it % T::NST, ph = (it / T::NST) & 1u;
                    if (!mbar_wait(&empty[st], ph ^ 1u)) { atomicExch(err, 1); ok = false; break; }
                    mbar_expect_tx(&full[st], T::A_BYTES);
                    tma_load_2d(sA + st * T::A_BYTES, &tmA, c * T::KC, (int)(tile * 128), &full[st]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            const uint32_t idesc = idesc_bf16(128, 256);
            bool ok = mbar_wait(&wfull, 0);
            if (!ok) atomicExch(err, 1);
            uint32_t it = 0, t = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++t) {
                const uint32_t b = t & 1u, use = t >> 1;
                if (!mbar_wait(&acce[b], (use & 1u) ^ 1u)) { atomicExch(err, 1); break; }
                tc_fence_after();
                for (int c = 0; c < T::NCH; ++c, ++it) {
                    const uint32_t st = it % T::NST, ph = (it / T::NST) & 1u;
                    if (!mbar_wait(&full[st], ph)) { atomicExch(err, 1); ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + st * T::A_BYTES), w0 = smem_u32(sW + c * T::W_BYTES);
#pragma unroll
                    for (int kk = 0; kk < T::KC / 16; ++kk)
                        umma_bf16(tmem + b * 256u, umma_desc_sw(a0 + 32u * kk, T::SWZ),
                                  umma_desc_sw(w0 + 32u * kk, T::SWZ), idesc, (c > 0 || kk > 0) ? 1u : 0u);
                    umma_commit(&empty[st]);             // the stage is free once these MMAs finish
                }
                if (ok) umma_commit(&accf[b]);
            }
        }
    } else {
        // epilogue: warps 2..9; warp w reads TMEM lanes 32 (w % 4) .. (its quarter of the tile's rows)
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        uint32_t t = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++t) {
            const uint32_t b = t & 1u, use = t >> 1;
            const bool got = mbar_wait(&accf[b], use & 1u);
            if (!__all_sync(0xffffffffu, got)) { atomicExch(err, 1); break; }   // the whole warp leaves
            tc_fence_after();
            act_epilogue_rows<K, EPI>(tmem + b * 256u, quarter, half, tile * 128, mp, sbias, mask, C, CT);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------ weight-gradient GEMM ---
// partial[b][o][n] = sum over this CTA's vertex range of AT[o][m] BT[n][m]
// (AT [256][mp], BT [NP][mp], BF16 row-major), split-K over vertices in
// 64-wide chunks, two M = 128 accumulators (o < 128, o >= 128), and the row
// sums of AT over the same range (the bias gradient): bpart[b][o].  The
// chunks come in by TMA (128-byte swizzled K-major tiles: AT chunk 256 x 64,
// BT chunk NP x 64) through a ring of NST stages.  Warp 0 loads, warp 1
// issues the MMAs, warps 2..9 take the bias row sums from each staged AT
// chunk (one row a thread, un-permuting the swizzle so that each row is
// summed in increasing m) and, at the end, write the accumulators.
template <int NP>
struct WgradTma {
    static constexpr int KC = 64;
    static constexpr uint32_t SA = 256u * 128u, SB = (uint32_t)NP * 128u;
    static constexpr int NST = NP >= 256 ? 3 : 5;
    static constexpr uint32_t NCOL = (2 * NP) < 32 ? 32 : 2 * NP;
    static constexpr size_t SMEM = (size_t)NST * (SA + SB) + 1024;
};

template <int NP>
__global__ void __launch_bounds__(320, 1)
k_umma_wgrad_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t mp,
                 float* __restrict__ partial, float* __restrict__ bpart, int* __restrict__ err) {
    using T = WgradTma<NP>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t base_u = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((base_u + 1023u) & ~1023u) - base_u);
    __shared__ __align__(8) uint64_t full[T::NST], empty[T::NST], accf;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 1) tmem_alloc(&tslot, T::NCOL);
    if (threadIdx.x == 0) {
        // a stage is free when its MMAs finished (one commit) and the eight
        // row-sum warps are done with it
        for (int i = 0; i < T::NST; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 9); }
        mbar_init(&accf, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    const int64_t nch = mp / T::KC;
    const int64_t c0 = nch * blockIdx.x / gridDim.x, c1 = nch * (blockIdx.x + 1) / gridDim.x;
    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t ch = c0; ch < c1; ++ch, ++it) {
                const uint32_t st = it % T::NST, ph = (it / T::NST) & 1u;
                if (!mbar_wait(&empty[st], ph ^ 1u)) { atomicExch(err, 1); break; }
                uint8_t* sA = smem + st * (T::SA + T::SB);
                mbar_expect_tx(&full[st], T::SA + T::SB);
                tma_load_2d(sA, &tmA, (int)(ch * T::KC), 0, &full[st]);
                tma_load_2d(sA + T::SA, &tmB, (int)(ch * T::KC), 0, &full[st]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, NP);
            uint32_t it = 0;
            bool ok = true;
            for (int64_t ch = c0; ch < c1; ++ch, ++it) {
                const uint32_t st = it % T::NST, ph = (it / T::NST) & 1u;
                if (!mbar_wait(&full[st], ph)) { atomicExch(err, 1); ok = false; break; }
                tc_fence_after();
                const uint32_t a0 = smem_u32(smem + st * (T::SA + T::SB)), b0 = a0 + T::SA;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int s = 0; s < T::KC / 16; ++s)
                        umma_bf16(tmem + (uint32_t)(h * NP), umma_desc_sw(a0 + (uint32_t)h * 16384u + 32u * s, 128),
                                  umma_desc_sw(b0 + 32u * s, 128), idesc, (ch > c0 || s > 0) ? 1u : 0u);
                umma_commit(&empty[st]);
            }
            if (ok && c1 > c0) umma_commit(&accf);
        }
    } else {
        const int row = (warp - 2) * 32 + lane;          // AT row summed by this thread
        float rs = 0.0f;
        bool ok = true;
        uint32_t it = 0;
        for (int64_t ch = c0; ch < c1; ++ch, ++it) {
            const uint32_t st = it % T::NST, ph = (it / T::NST) & 1u;
            const bool got = mbar_wait(&full[st], ph);
            if (!__all_sync(0xffffffffu, got)) { atomicExch(err, 1); ok = false; break; }
            const uint8_t* rowp = smem + st * (T::SA + T::SB) + (row >> 3) * 1024 + (row & 7) * 128;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < T::KC / 8; ++j) {
                const uint4 u = *reinterpret_cast<const uint4*>(rowp + ((j ^ (row & 7)) << 4));
                const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
                for (int i = 0; i < 8; ++i) acc += __bfloat162float(b[i]);
            }
            rs += acc;
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
        // warps 2..9: accumulator h = (warp - 2) / 4, TMEM lanes 32 (warp % 4) ..
        const int quarter = warp & 3, h = (warp - 2) >> 2;
        const int o = h * 128 + quarter * 32 + lane;
        bool have = ok && c1 > c0 && mbar_wait(&accf, 0);
        if (ok && c1 > c0 && !have) atomicExch(err, 1);
        have = __all_sync(0xffffffffu, have);          // tcgen05.ld wants the whole warp
        tc_fence_after();
        float* out = partial + (int64_t)blockIdx.x * 256 * NP;
        for (int n0 = 0; n0 < NP; n0 += 16) {
            float v[16];
            if (have) {
                tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(h * NP + n0), v);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) out[(int64_t)o * NP + n0 + i] = v[i];
        }
        bpart[(int64_t)blockIdx.x * 256 + row] = rs;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, T::NCOL);
}

// ------------------------------------------------------- CUDA-core part ---
// BF16 copies of the weights (W1, W2, W3) and of W2^T, W3^T
__global__ void k_params_bf16(const float* __restrict__ P, __nv_bfloat16* __restrict__ W1, __nv_bfloat16* __restrict__ W2,
                              __nv_bfloat16* __restrict__ W3, __nv_bfloat16* __restrict__ W2t,
                              __nv_bfloat16* __restrict__ W3t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHid * kIn) W1[i] = __float2bfloat16_rn(P[kOffW1 + i]);
    if (i < kHid * kHid) {
        const int o = i / kHid, j = i % kHid;
        const __nv_bfloat16 a = __float2bfloat16_rn(P[kOffW2 + i]);
        const __nv_bfloat16 b = __float2bfloat16_rn(P[kOffW3 + i]);
        W2[i] = a; W3[i] = b;
        W2t[j * kHid + o] = a; W3t[j * kHid + o] = b;
    }
}

// y = h3 W4^T + b4 (FP32), one thread per vertex
__global__ void __launch_bounds__(256)
k_head_fwd(const __nv_bfloat16* __restrict__ h3, const float* __restrict__ P, int64_t n, float* __restrict__ y) {
    __shared__ float w4[kOut * kHid];
    for (int i = threadIdx.x; i < kOut * kHid; i += blockDim.x) w4[i] = P[kOffW4 + i];
    __syncthreads();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    float a0 = P[kOffB4], a1 = P[kOffB4 + 1], a2 = P[kOffB4 + 2];
    for (int j0 = 0; j0 < kHid; j0 += 8) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(h3 + m * kHid + j0));
        const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float hv = __bfloat162float(hb[i]);
            a0 += hv * w4[j0 + i]; a1 += hv * w4[kHid + j0 + i]; a2 += hv * w4[2 * kHid + j0 + i];
        }
    }
    y[3 * m] = a0; y[3 * m + 1] = a1; y[3 * m + 2] = a2;
}

constexpr int kRedT = 256;
__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double sh[kRedT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < kRedT / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// per-block partial sums of the mask (fixed order)
__global__ void __launch_bounds__(kRedT) k_mask_sum(const float* __restrict__ mask, int64_t n, double* __restrict__ part) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double r = block_sum_d(m < n ? (double)mask[m] : 0.0);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}
// out = sum of np partials in a fixed order (strided per thread, then a tree)
__global__ void __launch_bounds__(1024) k_sum_parts(const double* __restrict__ part, int64_t np, double* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < np; i += 1024) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = sh[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *out = v;
    }
}

// Head forward and backward, persistent: each block walks a contiguous range
// of 32-vertex tiles (8 warps, 4 rows per warp; lane l owns columns l,
// l + 32, ..., so row accesses are coalesced and W4 reads conflict-free):
// y, the loss term m (y - t)^2 / (3 sum m), dy = 2 m (y - t) / (3 sum m),
// dz3 = (dy W4) * (h3 > 0) written row-major and, through a padded shared
// tile, as dz3^T.  Each lane also accumulates dW4 and db4 over the rows it
// visits; per block, the warps' sums are combined in warp order into
// wpart[block][4][256] (rows 0-2 dW4, row 3 db4 in its first 3 entries).
constexpr int kHeadRows = 32;
constexpr int kHeadLd = kHid + 4;                 // row stride of the transposition tile (BF16 values)
// Per-vertex head and loss: lane l of a warp holds columns 8 l .. 8 l + 7
// of a row (one 16-byte load of h3, one 16-byte store of dz3) and the
// matching 24 weights of W4 in registers; the three dot products are summed
// over the warp by butterfly shuffles.  Each block walks tiles of 32 rows;
// dz3^T leaves through a shared-memory transposition in 16-byte pieces.
__global__ void __launch_bounds__(256, 2)
k_head_bwd(const __nv_bfloat16* __restrict__ h3, const float* __restrict__ P, const float* __restrict__ target,
           const float* __restrict__ mask, int64_t n, int64_t mp, const double* __restrict__ msum,
           float* __restrict__ y, float* __restrict__ dy, __nv_bfloat16* __restrict__ dz3,
           __nv_bfloat16* __restrict__ dz3T, double* __restrict__ loss_part, float* __restrict__ wpart) {
    __shared__ __align__(16) __nv_bfloat16 tileT[kHeadRows][kHeadLd];
    __shared__ double lsh[8];
    __shared__ float wsh[8][4][32];
    __shared__ double inv_den_s;
    // one FP64 reciprocal per block (FP64 runs at a small fraction of FP32 here)
    if (threadIdx.x == 0) inv_den_s = *msum > 0.0 ? 1.0 / (3.0 * (*msum)) : 0.0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = 8 * lane;                       // this lane's first column
    float w[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 8; ++i) w[c][i] = P[kOffW4 + c * kHid + j0 + i];
    const float inv_den = (float)inv_den_s;
    const float b0 = P[kOffB4], b1 = P[kOffB4 + 1], b2 = P[kOffB4 + 2];
    const int64_t ntile = mp / kHeadRows;
    const int64_t t0 = ntile * blockIdx.x / gridDim.x, t1 = ntile * (blockIdx.x + 1) / gridDim.x;
    double lterm = 0.0;
    float gw[3][8], gb[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 8; ++i) gw[c][i] = 0.0f;
    // the warp's 4 rows of a tile travel together, and the next tile's rows
    // (with their masks and targets) are loaded while this one is processed
    constexpr int RW = kHeadRows / 8;
    uint4 raw[RW];
    float mkv[RW], tgv[RW];
    auto load_rows = [&](int64_t tile, uint4* rw, float* mk, float* tg) {
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) {
            const int64_t m = tile * kHeadRows + warp * RW + rr;
            rw[rr] = __ldg(reinterpret_cast<const uint4*>(h3 + m * kHid + j0));
            mk[rr] = m < n ? __ldg(mask + m) : 0.0f;
            tg[rr] = (m < n && lane < 3) ? __ldg(target + 3 * m + lane) : 0.0f;
        }
    };
    if (t0 < t1) load_rows(t0, raw, mkv, tgv);
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t m0 = tile * kHeadRows;
        float hv[RW][8], acc[RW][3], mkc[RW], tgc[RW];
        // the tile's loss terms in FP32 (12 at most), added to the FP64 sum once a
        // tile: FP64 instructions run at a small fraction of the FP32 rate here
        float tile_loss = 0.0f;
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) {
            const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&raw[rr]);
#pragma unroll
            for (int i = 0; i < 8; ++i) hv[rr][i] = __bfloat162float(hb[i]);
            mkc[rr] = mkv[rr];
            tgc[rr] = tgv[rr];
        }
        if (tile + 1 < t1) load_rows(tile + 1, raw, mkv, tgv);
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) {
            acc[rr][0] = acc[rr][1] = acc[rr][2] = 0.0f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[rr][0] += hv[rr][i] * w[0][i];
                acc[rr][1] += hv[rr][i] * w[1][i];
                acc[rr][2] += hv[rr][i] * w[2][i];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int rr = 0; rr < RW; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[rr][c] += __shfl_xor_sync(0xffffffffu, acc[rr][c], o);
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) {
            const int r = warp * RW + rr;
            const int64_t m = m0 + r;
            // every lane holds y; lane c < 3 forms component c of the loss
            // term and of dy in FP32, lane 0 sums the loss terms
            float dc = 0.0f;
            const bool live = m < n && mkc[rr] != 0.0f && inv_den > 0.0f;
            float lt = 0.0f;
            if (live && lane < 3) {
                const float yy = acc[rr][lane] + (lane == 0 ? b0 : (lane == 1 ? b1 : b2));
                const float e = yy - tgc[rr];
                const float mk = mkc[rr];
                lt = mk * e * e * inv_den;
                dc = 2.0f * mk * e * inv_den;
                y[3 * m + lane] = yy;
            }
            const float d0 = __shfl_sync(0xffffffffu, dc, 0), d1 = __shfl_sync(0xffffffffu, dc, 1),
                        d2 = __shfl_sync(0xffffffffu, dc, 2);
            const float l1 = __shfl_sync(0xffffffffu, lt, 1), l2 = __shfl_sync(0xffffffffu, lt, 2);
            tile_loss += (lt + l1) + l2;               // lane 0's copy is the one kept
            if (lane < 3) dy[3 * m + lane] = dc;
            gb[0] += d0; gb[1] += d1; gb[2] += d2;
            __align__(16) __nv_bfloat16 o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                gw[0][i] += d0 * hv[rr][i]; gw[1][i] += d1 * hv[rr][i]; gw[2][i] += d2 * hv[rr][i];
                const float g = d0 * w[0][i] + d1 * w[1][i] + d2 * w[2][i];
                o[i] = __float2bfloat16_rn(hv[rr][i] > 0.0f ? g : 0.0f);
            }
            const uint4 ov = *reinterpret_cast<const uint4*>(o);
            *reinterpret_cast<uint4*>(dz3 + m * kHid + j0) = ov;
            // kHeadLd * 2 bytes is a multiple of 8: two 8-byte pieces
            uint2* tp = reinterpret_cast<uint2*>(&tileT[r][j0]);
            tp[0] = make_uint2(ov.x, ov.y);
            tp[1] = make_uint2(ov.z, ov.w);
        }
        if (lane == 0) lterm += (double)tile_loss;
        __syncthreads();
        // dz3^T[j][m0 .. m0 + 31]: four threads a column, eight rows (16 bytes) each
        for (int idx = threadIdx.x; idx < 4 * kHid; idx += blockDim.x) {
            const int j = idx >> 2, seg = idx & 3;
            __align__(16) __nv_bfloat16 col[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) col[q] = tileT[8 * seg + q][j];
            *reinterpret_cast<uint4*>(dz3T + (int64_t)j * mp + m0 + 8 * seg) = *reinterpret_cast<const uint4*>(col);
        }
        __syncthreads();
    }
    // combine the warps' dW4 / db4 sums in warp order, one column slice at a time
    float* out = wpart + (int64_t)blockIdx.x * 4 * kHid;
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int c = 0; c < 3; ++c) wsh[warp][c][lane] = gw[c][i];
        wsh[warp][3][lane] = (i == 0 && lane < 3) ? gb[lane] : 0.0f;
        __syncthreads();
        if (threadIdx.x < 128) {
            const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
            float t = 0.0f;
            for (int w8 = 0; w8 < 8; ++w8) t += wsh[w8][c][l];
            // slot c < 3: column 8 l + i of dW4 row c; slot 3: db4 (lanes 0..2 of slice 0)
            if (c < 3) out[c * kHid + 8 * l + i] = t;
            else if (i == 0) out[3 * kHid + l] = t;
        }
        __syncthreads();
    }
    if (lane == 0) lsh[warp] = lterm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) t += lsh[w8];
        loss_part[blockIdx.x] = t;
    }
}

// out[l] = sum_p partial[p][l] in order p = 0 .. np-1 (optionally strided)
__global__ void k_reduce_part(const float* __restrict__ partial, int64_t np, int64_t stride, int64_t L,
                              float* __restrict__ out) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    // sixteen loads in flight at a time, added in the same order p = 0, 1, ...
    float s = 0.0f;
    int64_t p = 0;
    for (; p + 16 <= np; p += 16) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = partial[(p + q) * stride + l];
#pragma unroll
        for (int q = 0; q < 16; ++q) s += v[q];
    }
    for (; p < np; ++p) s += partial[p * stride + l];
    out[l] = s;
}

// Adam (bias-corrected) on the flattened FP32 parameters; omb1 = 1 - beta1
// and omb2 = 1 - beta2 come from the host in FP64 (1 - 0.999f in FP32 is
// 1.3e-5 away from 1e-3)
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M1,
                       float* __restrict__ M2, int64_t n, float lr, float b1, float b2, float omb1, float omb2,
                       float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float a = b1 * M1[i] + omb1 * g;
    const float b = b2 * M2[i] + omb2 * g * g;
    M1[i] = a;
    M2[i] = b;
    P[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

struct FeatScales {
    float inv_pos, inv_disp, inv_force, h;
    float lo[3], inv_ext[3];
};

// 32 features per vertex (rows >= n are zero):
//  0-2 (x - X) / pos_scale       3-5 h v / disp_scale      6-8 X mapped to [-1, 1]
//  9 Dirichlet flag              10 slave-surface flag     11-13 contact force / force_scale (clamped +-8)
//  14 contact active             15-26 sin, cos (pi k Xn), k = 1, 2, per axis      27-31 zero
template <class TG>
__global__ void __launch_bounds__(256)
k_features(const double* __restrict__ x, const double* __restrict__ v, const double* __restrict__ X,
           const uint8_t* __restrict__ dir, const uint8_t* __restrict__ surf, const TG* __restrict__ cg,
           int64_t n, int64_t mp, FeatScales S, __nv_bfloat16* __restrict__ f, __nv_bfloat16* __restrict__ fT) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= mp) return;
    float o[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) o[i] = 0.0f;
    if (m < n) {
        float xn[3];
        for (int c = 0; c < 3; ++c) {
            o[c] = (float)(x[3 * m + c] - X[3 * m + c]) * S.inv_pos;
            o[3 + c] = (float)(S.h * v[3 * m + c]) * S.inv_disp;
            xn[c] = 2.0f * ((float)X[3 * m + c] - S.lo[c]) * S.inv_ext[c] - 1.0f;
            o[6 + c] = xn[c];
        }
        o[9] = dir[m] ? 1.0f : 0.0f;
        o[10] = surf[m] ? 1.0f : 0.0f;
        float act = 0.0f;
        for (int c = 0; c < 3; ++c) {
            const float g = cg ? -(float)cg[3 * m + c] : 0.0f;   // contact force = -grad Psi
            o[11 + c] = fminf(fmaxf(g * S.inv_force, -8.0f), 8.0f);
            if (g != 0.0f) act = 1.0f;
        }
        o[14] = act;
        for (int c = 0; c < 3; ++c)
            for (int k = 1; k <= 2; ++k) {
                const float a = 3.14159265358979f * (float)k * xn[c];
                o[15 + 4 * c + 2 * (k - 1)] = sinf(a);
                o[15 + 4 * c + 2 * (k - 1) + 1] = cosf(a);
            }
    }
    __align__(16) __nv_bfloat16 b[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) {
        b[i] = __float2bfloat16_rn(o[i]);
        fT[(int64_t)i * mp + m] = b[i];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        reinterpret_cast<uint4*>(f + m * kIn)[q] = reinterpret_cast<const uint4*>(b)[q];
}

// dx = h v + disp_scale y
__global__ void k_predict(const float* __restrict__ y, const double* __restrict__ v, int64_t n, double h,
                          double disp, double* __restrict__ dx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    dx[i] = h * v[i] + disp * (double)y[i];
}

unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// at least this much dynamic shared memory keeps one CTA per SM, so the
// tensor-memory allocations of co-resident CTAs never exceed 512 columns
constexpr size_t kOneCtaSmem = 120 * 1024;

// cuTensorMapEncodeTiled from the driver (through the runtime, so the library
// needs no link against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// tensor map of a row-major BF16 matrix [rows][cols] (cols contiguous),
// read in boxes of box_rows x box_cols with the swizzle of a box_cols * 2
// byte row (128 or 64 bytes)
cudaError_t bf16_tmap(CUtensorMap* m, const __nv_bfloat16* base, int64_t rows, int cols, int box_rows,
                      int box_cols) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return cudaErrorNotSupported;
    if (((uintptr_t)base & 15u) != 0 || (cols * 2) % 16 != 0 || (box_cols * 2 != 128 && box_cols * 2 != 64))
        return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           box_cols * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int K, int EPI>
cudaError_t launch_act(Ctx& c, WarmStart& W, const __nv_bfloat16* A, const __nv_bfloat16* Wt, const float* bias,
                       const __nv_bfloat16* mask, __nv_bfloat16* C, __nv_bfloat16* CT) {
    using T = ActTma<K>;
    CUtensorMap ta, tw;
    GMCP_CUDA_TRY(bf16_tmap(&ta, A, W.mp, K, 128, T::KC));
    GMCP_CUDA_TRY(bf16_tmap(&tw, Wt, 256, K, 256, T::KC));
    const size_t sm = std::max(T::SMEM, kOneCtaSmem);
    GMCP_CUDA_TRY(cudaFuncSetAttribute(k_umma_act_tma<K, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int grid = (int)std::min<int64_t>(sm_count(c.device), W.mp / 128);
    k_umma_act_tma<K, EPI><<<grid, T::THREADS, sm, c.stream>>>(ta, tw, W.mp, bias, mask, C, CT, W.err.p);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_wgrad(Ctx& c, WarmStart& W, const __nv_bfloat16* AT, const __nv_bfloat16* BT, float* out,
                         float* bias_out) {
    using T = WgradTma<NP>;
    CUtensorMap ta, tb;
    GMCP_CUDA_TRY(bf16_tmap(&ta, AT, 256, W.mp, 256, T::KC));
    GMCP_CUDA_TRY(bf16_tmap(&tb, BT, NP, W.mp, NP, T::KC));
    const size_t sm = std::max(T::SMEM, kOneCtaSmem);
    GMCP_CUDA_TRY(cudaFuncSetAttribute(k_umma_wgrad_tma<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int grid = sm_count(c.device);
    float* bpart = W.part.p + (size_t)grid * 256 * NP;
    k_umma_wgrad_tma<NP><<<grid, 320, sm, c.stream>>>(ta, tb, W.mp, W.part.p, bpart, W.err.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    k_reduce_part<<<nb(256 * NP, 256), 256, 0, c.stream>>>(W.part.p, grid, 256 * NP, 256 * NP, out);
    k_reduce_part<<<1, 256, 0, c.stream>>>(bpart, grid, 256, 256, bias_out);
    return cudaGetLastError();
}

}  // namespace

// forward through the three hidden layers (features already in W.f / W.fT)
static cudaError_t ws_hidden(Ctx& c, WarmStart& W, bool keep_transposes) {
    const float* P = W.P.p;
    GMCP_CUDA_TRY((launch_act<kIn, 0>(c, W, W.f.p, W.W1.p, P + kOffB1, nullptr, W.h1.p, keep_transposes ? W.h1T.p : nullptr)));
    GMCP_CUDA_TRY((launch_act<kHid, 0>(c, W, W.h1.p, W.W2.p, P + kOffB2, nullptr, W.h2.p, keep_transposes ? W.h2T.p : nullptr)));
    return launch_act<kHid, 0>(c, W, W.h2.p, W.W3.p, P + kOffB3, nullptr, W.h3.p, nullptr);
}

static cudaError_t ws_check_err(Ctx& c, WarmStart& W, bool* bad) {
    int e = 0;
    GMCP_CUDA_TRY(cudaMemcpyAsync(&e, W.err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    GMCP_CUDA_TRY(cudaStreamSynchronize(c.stream));
    *bad = e != 0;
    return cudaSuccess;
}

// forward + backward into W.G; loss into *loss (host, synchronises)
static cudaError_t ws_backward(Ctx& c, WarmStart& W, const float* target, const float* mask, double* loss) {
    cudaStream_t s = c.stream;
    const int64_t n = W.n, mp = W.mp;
    GMCP_CUDA_TRY(ws_hidden(c, W, true));
    double* sc = W.scal.p;
    const unsigned gn = nb(n, kRedT);
    k_mask_sum<<<gn, kRedT, 0, s>>>(mask, n, W.dpart.p);
    k_sum_parts<<<1, 1024, 0, s>>>(W.dpart.p, (int64_t)gn, sc);
    const unsigned gh = (unsigned)std::min<int64_t>(4 * sm_count(c.device), mp / kHeadRows);
    float* wp = W.part.p;
    k_head_bwd<<<gh, 256, 0, s>>>(W.h3.p, W.P.p, target, mask, n, mp, sc, W.y.p, W.dy.p, W.dz3.p, W.dz3T.p,
                                  W.dpart.p, wp);
    k_sum_parts<<<1, 1024, 0, s>>>(W.dpart.p, (int64_t)gh, sc + 1);
    GMCP_CUDA_TRY(cudaGetLastError());
    float* G = W.G.p;
    // layer 4 from the head's per-block partials
    k_reduce_part<<<nb(3 * kHid, 256), 256, 0, s>>>(wp, gh, 4 * kHid, 3 * kHid, G + kOffW4);
    k_reduce_part<<<1, 32, 0, s>>>(wp + 3 * kHid, gh, 4 * kHid, 3, G + kOffB4);
    GMCP_CUDA_TRY(cudaGetLastError());
    // layer 3: dW3 = dz3^T h2, db3
    GMCP_CUDA_TRY(launch_wgrad<kHid>(c, W, W.dz3T.p, W.h2T.p, G + kOffW3, G + kOffB3));
    // dz2 = (dz3 W3) * (h2 > 0)
    GMCP_CUDA_TRY((launch_act<kHid, 1>(c, W, W.dz3.p, W.W3t.p, nullptr, W.h2.p, W.dz2.p, W.dz2T.p)));
    GMCP_CUDA_TRY(launch_wgrad<kHid>(c, W, W.dz2T.p, W.h1T.p, G + kOffW2, G + kOffB2));
    // dz1 = (dz2 W2) * (h1 > 0)
    GMCP_CUDA_TRY((launch_act<kHid, 1>(c, W, W.dz2.p, W.W2t.p, nullptr, W.h1.p, nullptr, W.dz1T.p)));
    GMCP_CUDA_TRY(launch_wgrad<kIn>(c, W, W.dz1T.p, W.fT.p, G + kOffW1, G + kOffB1));
    GMCP_CUDA_TRY(cudaGetLastError());
    if (loss) {
        GMCP_CUDA_TRY(cudaMemcpyAsync(loss, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    return cudaSuccess;
}

void ws_destroy(WarmStart* w) { delete w; }

int64_t ws_param_count() { return kNParam; }

cudaError_t ws_state_get(Ctx& c, WsState* o) {
    WarmStart& W = *c.ws;
    o->lr = W.lr; o->beta1 = W.beta1; o->beta2 = W.beta2; o->eps = W.eps;
    o->pos_scale = W.pos_scale; o->disp_scale = W.disp_scale; o->force_scale = W.force_scale;
    o->step = W.step;
    o->P.resize(kNParam); o->M1.resize(kNParam); o->M2.resize(kNParam);
    GMCP_CUDA_TRY(cudaMemcpyAsync(o->P.data(), W.P.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, c.stream));
    GMCP_CUDA_TRY(cudaMemcpyAsync(o->M1.data(), W.M1.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, c.stream));
    GMCP_CUDA_TRY(cudaMemcpyAsync(o->M2.data(), W.M2.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, c.stream));
    return cudaStreamSynchronize(c.stream);
}

cudaError_t ws_state_set(Ctx& c, const WsState& in) {
    WarmStart& W = *c.ws;
    if ((int64_t)in.P.size() != kNParam || (int64_t)in.M1.size() != kNParam || (int64_t)in.M2.size() != kNParam)
        return cudaErrorInvalidValue;
    W.lr = in.lr; W.beta1 = in.beta1; W.beta2 = in.beta2; W.eps = in.eps;
    W.pos_scale = in.pos_scale; W.disp_scale = in.disp_scale; W.force_scale = in.force_scale;
    W.step = in.step;
    cudaStream_t s = c.stream;
    GMCP_CUDA_TRY(cudaMemcpyAsync(W.P.p, in.P.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
    GMCP_CUDA_TRY(cudaMemcpyAsync(W.M1.p, in.M1.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
    GMCP_CUDA_TRY(cudaMemcpyAsync(W.M2.p, in.M2.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
    k_params_bf16<<<nb(kHid * kHid, 256), 256, 0, s>>>(W.P.p, W.W1.p, W.W2.p, W.W3.p, W.W2t.p, W.W3t.p);
    GMCP_CUDA_TRY(cudaGetLastError());
    return cudaStreamSynchronize(s);
}

}  // namespace gmcp

using namespace gmcp;

static ipc_status ws_fail(Ctx& c, ipc_status st, const std::string& m) {
    c.err = m;
    return st;
}
#define WS_CK(c, expr)                                                                      \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return ws_fail(c, _e == cudaErrorMemoryAllocation ? IPC_ERR_OOM : IPC_ERR_CUDA, \
                           std::string(#expr) + ": " + cudaGetErrorString(_e));             \
        }                                                                                   \
    } while (0)

extern "C" {

ipc_status ipc_ws_create(ipc_ctx* ctx, const ipc_ws_params* prm) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!prm || !prm->params_host || !(prm->lr > 0.0) || !(prm->pos_scale > 0.0) || !(prm->disp_scale > 0.0) ||
        !(prm->force_scale > 0.0))
        return ws_fail(c, IPC_ERR_ARG, "ipc_ws_create: NULL parameters or non-positive lr / scales");
    WS_CK(c, cudaSetDevice(c.device));
    std::unique_ptr<WarmStart> W(new WarmStart());
    W->n = c.nv;
    W->mp = (c.nv + 127) / 128 * 128;
    W->lr = prm->lr; W->beta1 = prm->beta1; W->beta2 = prm->beta2; W->eps = prm->eps;
    W->pos_scale = prm->pos_scale; W->disp_scale = prm->disp_scale; W->force_scale = prm->force_scale;
    for (int q = 0; q < 3; ++q) { W->lo[q] = 1e300; W->hi[q] = -1e300; }
    for (int64_t v = 0; v < c.nv; ++v)
        for (int q = 0; q < 3; ++q) {
            W->lo[q] = std::min(W->lo[q], c.h_X[3 * v + q]);
            W->hi[q] = std::max(W->hi[q], c.h_X[3 * v + q]);
        }
    std::vector<uint8_t> surf(c.nv, 0);
    {
        std::vector<int32_t> st((size_t)3 * c.ns);
        WS_CK(c, cudaMemcpy(st.data(), c.stri.p, sizeof(int32_t) * st.size(), cudaMemcpyDeviceToHost));
        for (int32_t v : st) surf[v] = 1;
    }
    const int64_t mp = W->mp;
    cudaStream_t s = c.stream;
    WS_CK(c, W->P.upload(prm->params_host, kNParam, s));
    WS_CK(c, W->M1.ensure(kNParam)); WS_CK(c, W->M2.ensure(kNParam)); WS_CK(c, W->G.ensure(kNParam));
    WS_CK(c, cudaMemsetAsync(W->M1.p, 0, sizeof(float) * kNParam, s));
    WS_CK(c, cudaMemsetAsync(W->M2.p, 0, sizeof(float) * kNParam, s));
    WS_CK(c, W->W1.ensure(kHid * kIn)); WS_CK(c, W->W2.ensure(kHid * kHid)); WS_CK(c, W->W3.ensure(kHid * kHid));
    WS_CK(c, W->W2t.ensure(kHid * kHid)); WS_CK(c, W->W3t.ensure(kHid * kHid));
    WS_CK(c, W->f.ensure(mp * kIn)); WS_CK(c, W->fT.ensure(mp * kIn));
    for (DBuf<__nv_bfloat16>* b : {&W->h1, &W->h2, &W->h3, &W->h1T, &W->h2T, &W->dz3, &W->dz3T, &W->dz2, &W->dz2T, &W->dz1T})
        WS_CK(c, b->ensure((size_t)mp * kHid));
    WS_CK(c, W->y.ensure(3 * mp)); WS_CK(c, W->dy.ensure(3 * mp));
    // partial sums: split-K weight gradients [SMs][256][256] plus scratch
    WS_CK(c, W->part.ensure(std::max((size_t)std::max(sm_count(c.device), 1) * (kHid * kHid + kHid),
                                     (size_t)4 * kHid * ((mp + 2047) / 2048)) + 1024));
    WS_CK(c, W->dpart.ensure((size_t)(mp + 31) / 32 + 16));
    WS_CK(c, W->surf.upload(surf.data(), surf.size(), s));
    if (c.P.precision == IPC_PREC_MIXED) WS_CK(c, W->cgrad32.ensure(3 * (size_t)c.nv));
    else WS_CK(c, W->cgrad64.ensure(3 * (size_t)c.nv));
    WS_CK(c, W->err.ensure(1)); WS_CK(c, cudaMemsetAsync(W->err.p, 0, sizeof(int), s));
    WS_CK(c, W->scal.ensure(8));
    WS_CK(c, cudaMemsetAsync(W->f.p, 0, sizeof(__nv_bfloat16) * mp * kIn, s));
    WS_CK(c, cudaMemsetAsync(W->fT.p, 0, sizeof(__nv_bfloat16) * mp * kIn, s));
    k_params_bf16<<<nb(kHid * kHid, 256), 256, 0, s>>>(W->P.p, W->W1.p, W->W2.p, W->W3.p, W->W2t.p, W->W3t.p);
    WS_CK(c, cudaGetLastError());
    WS_CK(c, cudaStreamSynchronize(s));
    c.ws = std::unique_ptr<WarmStart, void (*)(WarmStart*)>(W.release(), ws_destroy);
    return IPC_OK;
}

ipc_status ipc_ws_features(ipc_ctx* ctx, const double* x_dev, const double* v_dev, const double* xm_dev,
                           void* feats_dev) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!c.ws) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_features: call ipc_ws_create first");
    if (!x_dev || !v_dev || (!xm_dev && c.nmv > 0)) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_features: NULL input");
    WarmStart& W = *c.ws;
    WS_CK(c, cudaSetDevice(c.device));
    // contact force at (x, xm) from the contact pass
    const bool f32 = c.P.precision == IPC_PREC_MIXED;
    WS_CK(c, run_candidates(c, x_dev, xm_dev));
    void* cg = f32 ? (void*)W.cgrad32.p : (void*)W.cgrad64.p;
    WS_CK(c, contact_eval(c, x_dev, xm_dev, nullptr, cg, false, nullptr));
    FeatScales S;
    S.inv_pos = (float)(1.0 / W.pos_scale);
    S.inv_disp = (float)(1.0 / W.disp_scale);
    S.inv_force = (float)(1.0 / W.force_scale);
    S.h = (float)c.prm.h;
    for (int q = 0; q < 3; ++q) {
        S.lo[q] = (float)W.lo[q];
        S.inv_ext[q] = (float)(W.hi[q] > W.lo[q] ? 1.0 / (W.hi[q] - W.lo[q]) : 1.0);
    }
    const uint8_t* dir = c.newton ? c.newton->dir.p : nullptr;
    DBuf<uint8_t> dtmp;
    if (!dir) {
        WS_CK(c, dtmp.upload(c.h_dir.data(), c.h_dir.size(), c.stream));
        dir = dtmp.p;
    }
    if (f32)
        k_features<float><<<nb(W.mp, 256), 256, 0, c.stream>>>(x_dev, v_dev, c.X.p, dir, W.surf.p, W.cgrad32.p, W.n, W.mp, S, W.f.p, W.fT.p);
    else
        k_features<double><<<nb(W.mp, 256), 256, 0, c.stream>>>(x_dev, v_dev, c.X.p, dir, W.surf.p, W.cgrad64.p, W.n, W.mp, S, W.f.p, W.fT.p);
    WS_CK(c, cudaGetLastError());
    if (feats_dev)
        WS_CK(c, cudaMemcpyAsync(feats_dev, W.f.p, sizeof(__nv_bfloat16) * W.n * kIn, cudaMemcpyDeviceToDevice, c.stream));
    WS_CK(c, cudaStreamSynchronize(c.stream));
    return IPC_OK;
}

// copy caller features [n][32] BF16 into the padded row-major and transposed buffers
namespace gmcp {
namespace {
__global__ void k_load_feats(const __nv_bfloat16* __restrict__ src, int64_t n, int64_t mp,
                             __nv_bfloat16* __restrict__ f, __nv_bfloat16* __restrict__ fT) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= mp) return;
    __align__(16) __nv_bfloat16 v[kIn];
    for (int q = 0; q < kIn / 8; ++q)
        reinterpret_cast<uint4*>(v)[q] = m < n ? reinterpret_cast<const uint4*>(src + m * kIn)[q] : make_uint4(0, 0, 0, 0);
    for (int q = 0; q < kIn / 8; ++q) reinterpret_cast<uint4*>(f + m * kIn)[q] = reinterpret_cast<const uint4*>(v)[q];
    for (int i = 0; i < kIn; ++i) fT[(int64_t)i * mp + m] = v[i];
}
}  // namespace
}  // namespace gmcp

static ipc_status ws_take_feats(Ctx& c, WarmStart& W, const void* feats_dev) {
    if (!feats_dev) return IPC_OK;
    k_load_feats<<<nb(W.mp, 256), 256, 0, c.stream>>>((const __nv_bfloat16*)feats_dev, W.n, W.mp, W.f.p, W.fT.p);
    WS_CK(c, cudaGetLastError());
    return IPC_OK;
}

ipc_status ipc_ws_forward(ipc_ctx* ctx, const void* feats_dev, float* out_dev) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!c.ws) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_forward: call ipc_ws_create first");
    if (!out_dev) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_forward: NULL output");
    WarmStart& W = *c.ws;
    WS_CK(c, cudaSetDevice(c.device));
    ipc_status st = ws_take_feats(c, W, feats_dev);
    if (st != IPC_OK) return st;
    WS_CK(c, ws_hidden(c, W, false));
    k_head_fwd<<<nb(W.n, 256), 256, 0, c.stream>>>(W.h3.p, W.P.p, W.n, out_dev);
    WS_CK(c, cudaGetLastError());
    bool bad = false;
    WS_CK(c, ws_check_err(c, W, &bad));
    if (bad) return ws_fail(c, IPC_ERR_TIMEOUT, "ipc_ws_forward: a tensor-core wait hit its iteration cap");
    return IPC_OK;
}

ipc_status ipc_ws_grads(ipc_ctx* ctx, const void* feats_dev, const float* target_dev, const float* mask_dev,
                        double* loss_host, float* grads_host) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!c.ws) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_grads: call ipc_ws_create first");
    if (!target_dev || !mask_dev) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_grads: NULL target or mask");
    WarmStart& W = *c.ws;
    WS_CK(c, cudaSetDevice(c.device));
    ipc_status st = ws_take_feats(c, W, feats_dev);
    if (st != IPC_OK) return st;
    double loss = 0.0;
    WS_CK(c, ws_backward(c, W, target_dev, mask_dev, &loss));
    if (grads_host)
        WS_CK(c, cudaMemcpyAsync(grads_host, W.G.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, c.stream));
    bool bad = false;
    WS_CK(c, ws_check_err(c, W, &bad));
    if (bad) return ws_fail(c, IPC_ERR_TIMEOUT, "ipc_ws_grads: a tensor-core wait hit its iteration cap");
    if (loss_host) *loss_host = loss;
    return IPC_OK;
}

ipc_status ipc_ws_train_step(ipc_ctx* ctx, const void* feats_dev, const float* target_dev, const float* mask_dev,
                             double* loss_host) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!c.ws) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_train_step: call ipc_ws_create first");
    if (!target_dev || !mask_dev) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_train_step: NULL target or mask");
    WarmStart& W = *c.ws;
    WS_CK(c, cudaSetDevice(c.device));
    ipc_status st = ws_take_feats(c, W, feats_dev);
    if (st != IPC_OK) return st;
    double loss = 0.0;
    WS_CK(c, ws_backward(c, W, target_dev, mask_dev, loss_host ? &loss : nullptr));
    W.step += 1;
    const float c1 = (float)(1.0 - std::pow(W.beta1, (double)W.step));
    const float c2 = (float)(1.0 - std::pow(W.beta2, (double)W.step));
    k_adam<<<nb(kNParam, 256), 256, 0, c.stream>>>(W.P.p, W.G.p, W.M1.p, W.M2.p, kNParam, (float)W.lr, (float)W.beta1,
                                                   (float)W.beta2, (float)(1.0 - W.beta1), (float)(1.0 - W.beta2),
                                                   (float)W.eps, c1, c2);
    k_params_bf16<<<nb(kHid * kHid, 256), 256, 0, c.stream>>>(W.P.p, W.W1.p, W.W2.p, W.W3.p, W.W2t.p, W.W3t.p);
    WS_CK(c, cudaGetLastError());
    bool bad = false;
    WS_CK(c, ws_check_err(c, W, &bad));
    if (bad) return ws_fail(c, IPC_ERR_TIMEOUT, "ipc_ws_train_step: a tensor-core wait hit its iteration cap");
    if (loss_host) *loss_host = loss;
    return IPC_OK;
}

ipc_status ipc_ws_get_params(ipc_ctx* ctx, float* params_host) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!c.ws || !params_host) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_get_params: no network or NULL output");
    WS_CK(c, cudaSetDevice(c.device));
    WS_CK(c, cudaMemcpyAsync(params_host, c.ws->P.p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, c.stream));
    WS_CK(c, cudaStreamSynchronize(c.stream));
    return IPC_OK;
}

ipc_status ipc_ws_predict(ipc_ctx* ctx, const double* x_dev, const double* v_dev, const double* xm_dev,
                          double* dx_dev) {
    if (!ctx) return IPC_ERR_ARG;
    Ctx& c = ctx_of(ctx);
    if (!c.ws) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_predict: call ipc_ws_create first");
    if (!dx_dev) return ws_fail(c, IPC_ERR_ARG, "ipc_ws_predict: NULL output");
    ipc_status st = ipc_ws_features(ctx, x_dev, v_dev, xm_dev, nullptr);
    if (st != IPC_OK) return st;
    WarmStart& W = *c.ws;
    WS_CK(c, ws_hidden(c, W, false));
    k_head_fwd<<<nb(W.n, 256), 256, 0, c.stream>>>(W.h3.p, W.P.p, W.n, W.y.p);
    k_predict<<<nb(3 * W.n, 256), 256, 0, c.stream>>>(W.y.p, v_dev, W.n, c.prm.h, W.disp_scale, dx_dev);
    WS_CK(c, cudaGetLastError());
    bool bad = false;
    WS_CK(c, ws_check_err(c, W, &bad));
    if (bad) return ws_fail(c, IPC_ERR_TIMEOUT, "ipc_ws_predict: a tensor-core wait hit its iteration cap");
    return IPC_OK;
}

}  // extern "C"

// scan.cu -- device-wide exclusive prefix sum of int32 counts.
//
// Three-phase scan: each 1024-thread block scans 4096 items (4 per thread,
// warp shuffles for the intra-block part), block totals are scanned
// recursively, then added back.  out[n] receives the grand total.  Integer
// arithmetic only, so the result does not depend on scheduling.
#include "gmcp_internal.cuh"

namespace gmcp {
namespace {

constexpr int kThreads = 1024;
constexpr int kPerThread = 4;
constexpr int kPerBlock = kThreads * kPerThread;

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__global__ void k_scan_blocks(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                              int32_t* __restrict__ block_sums, int64_t n) {
    pass_dep_wait();
    __shared__ int warp_tot[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kPerThread;
    int v[kPerThread];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int incl = warp_incl_scan(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int t = warp_tot[lane];
        int ti = warp_incl_scan(t);
        warp_tot[lane] = ti - t;  // exclusive offset of each warp
    }
    __syncthreads();
    int run = incl - s + warp_tot[warp];
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == kThreads - 1) block_sums[blockIdx.x] = run;
}

__global__ void k_add_offsets(int32_t* __restrict__ out, const int32_t* __restrict__ offs, int64_t n) {
    pass_dep_wait();
    const int64_t base = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kPerThread;
    const int add = offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kPerThread; ++i)
        if (base + i < n) out[base + i] += add;
}

__global__ void k_write_total(const int32_t* in, int32_t* out, int64_t n) {
    pass_dep_wait();
    out[n] = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

// exclusive scan of n items; tmp must hold 2 * scan_tmp_size(n) ints
cudaError_t scan_rec(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + kPerBlock - 1) / kPerBlock;
    int32_t* sums = tmp;                  // [nb]
    int32_t* sums_scan = tmp + nb + 1;    // [nb]
    launch_dep(k_scan_blocks, (unsigned)nb, kThreads, 0, s, in, out, sums, n);
    GMCP_CUDA_TRY(cudaGetLastError());
    if (nb > 1) {
        GMCP_CUDA_TRY(scan_rec(sums, sums_scan, nb, sums_scan + nb + 1, s));
        launch_dep(k_add_offsets, (unsigned)nb, kThreads, 0, s, out, sums_scan, n);
        GMCP_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace

size_t scan_tmp_size(int64_t n) {
    size_t total = 0;
    int64_t m = n;
    while (true) {
        int64_t nb = (m + kPerBlock - 1) / kPerBlock;
        total += (size_t)nb + 1;
        if (nb <= 1) break;
        m = nb;
    }
    return total + 8;
}

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp,
                               size_t tmp_n, cudaStream_t s) {
    if (tmp_n < 2 * scan_tmp_size(n)) return cudaErrorInvalidValue;
    GMCP_CUDA_TRY(scan_rec(in, out, n, tmp, s));
    launch_dep(k_write_total, 1, 1, 0, s, in, out, n);
    return cudaGetLastError();
}

}  // namespace gmcp

// peaks.cu -- CUDA-core arithmetic peaks of the device, measured.
//
// Not part of the method: the benchmark divides the contact pass's FP32 and
// FP64 work by these rates to report roofline fractions against what this
// GPU actually sustains, rather than against a nominal figure.  Each thread
// runs kChains independent fused multiply-add chains (enough independent
// work to cover the pipe latency), every SM holds several resident blocks,
// and the kernel is timed with CUDA events on the caller's stream after an
// untimed launch.  One FMA counts as two floating-point operations.
#include <cstdint>
#include <string>

#include "gmcp_internal.cuh"

namespace gmcp {
namespace {

constexpr int kChains = 16;
__device__ double g_peak_sink;   // keeps the chains live; written only if a result is exactly zero

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T a, T b) {
    T v[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = (T)(threadIdx.x + j) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) v[j] = fma(v[j], a, b);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += v[j];
    if (s == (T)0) g_peak_sink = (double)s;
}

}  // namespace
}  // namespace gmcp

using namespace gmcp;

extern "C" ipc_status ipc_alu_peak(int32_t kind, int32_t device, void* stream, double* tflops_host) {
    if ((kind != 0 && kind != 1) || !tflops_host) return IPC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // FP64 runs far fewer FMAs per clock: fewer iterations keep its launch
    // about as long as the FP32 one
    const int iters = kind == 0 ? 4096 : 128;
    const int blocks = sms * 8, threads = 256;
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(e0, s);
        if (kind == 0) k_fma_chains<float><<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-4f);
        else k_fma_chains<double><<<blocks, threads, 0, s>>>(iters, 0.999, 1e-4);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (rep == 1 && e == cudaSuccess) e = cudaEventRecord(e1, s);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_global_error(std::string("ipc_alu_peak: ") + cudaGetErrorString(e));
        return IPC_ERR_CUDA;
    }
    const double fmas = (double)blocks * threads * iters * kChains;
    *tflops_host = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return IPC_OK;
}

// faceclip.cu -- the paper's face samples of Sec. 4.1 ("Face samples") for
// a list of (slave triangle, master triangle) pairs, one thread per pair
// (the arithmetic is in faceclip.cuh, shared with the contact pass's
// clipped-overlap mode).  Compiled without FMA contraction.
#include <cmath>
#include <string>

#include "faceclip.cuh"
#include "gmcp_internal.cuh"

namespace {

using namespace gmcp::fclip;

__global__ void k_face_clip(const double* __restrict__ xs, const int32_t* __restrict__ ts, int64_t nts,
                            int64_t nvs, const double* __restrict__ xm, const int32_t* __restrict__ tm,
                            int64_t ntm, int64_t nvm, const int32_t* __restrict__ pairs, int64_t n,
                            double* __restrict__ out, int32_t* __restrict__ count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t a_t = pairs[2 * k], b_t = pairs[2 * k + 1];
    count[k] = 0;
    if (a_t < 0 || a_t >= nts || b_t < 0 || b_t >= ntm) { count[k] = -1; return; }
    int64_t vs[3], vm[3];
    for (int c = 0; c < 3; ++c) {
        vs[c] = ts[3 * a_t + c];
        vm[c] = tm[3 * b_t + c];
        if (vs[c] < 0 || vs[c] >= nvs || vm[c] < 0 || vm[c] >= nvm) { count[k] = -1; return; }
    }
    double* o = out + 96 * k;   // 12 samples x 8
    int ns = 0;
    count[k] = clip_samples(at(xs, vs[0]), at(xs, vs[1]), at(xs, vs[2]), at(xm, vm[0]), at(xm, vm[1]),
                            at(xm, vm[2]), [&](const double* bs, const double* bm, double g, double w) {
                                double* os = o + 8 * ns++;
                                os[0] = bs[0]; os[1] = bs[1]; os[2] = bs[2];
                                os[3] = bm[0]; os[4] = bm[1]; os[5] = bm[2];
                                os[6] = g;
                                os[7] = w;
                            });
}

ipc_status fc_fail(ipc_status st, const std::string& msg) {
    gmcp::set_global_error(msg);
    return st;
}

}  // namespace

extern "C" ipc_status ipc_face_clip_samples(const double* xs_dev, int64_t nvs, const int32_t* ts_dev, int64_t nts,
                                            const double* xm_dev, int64_t nvm, const int32_t* tm_dev, int64_t ntm,
                                            const int32_t* pairs_dev, int64_t n, double* samples_dev,
                                            int32_t* count_dev, void* stream) {
    if (n < 0) return fc_fail(IPC_ERR_ARG, "ipc_face_clip_samples: negative pair count");
    if (n == 0) return IPC_OK;
    if (!xs_dev || !ts_dev || !xm_dev || !tm_dev || !pairs_dev || !samples_dev || !count_dev)
        return fc_fail(IPC_ERR_ARG, "ipc_face_clip_samples: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    k_face_clip<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(xs_dev, ts_dev, nts, nvs, xm_dev, tm_dev, ntm, nvm,
                                                            pairs_dev, n, samples_dev, count_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fc_fail(IPC_ERR_CUDA, std::string("ipc_face_clip_samples: ") + cudaGetErrorString(e));
    return IPC_OK;
}

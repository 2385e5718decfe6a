// FP64 FMA throughput probe: the ALU peak against which the plain FP64 walk
// (an FP64-arithmetic-bound kernel on GB300) is reported.  Not part of the
// projectors; the paper has no counterpart.
#include <cuda_runtime.h>

#include "../../include/tetproj.h"
#include "kernels.cuh"

namespace tp {

constexpr int kFmaChains = 8;
constexpr int kFmaThreads = 256;

// Eight independent FMA chains per thread (enough in flight to cover the FP64
// pipe's latency); the result is written only on an impossible value, which
// the compiler cannot prove, so no chain is removed.
__global__ void __launch_bounds__(kFmaThreads) k_fma64(int64_t iters, double a, double b,
                                                       double *sink) {
    double x[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = 1e-3 * threadIdx.x + k;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += x[k];
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace tp

extern "C" tetproj_status tetproj_fma64_probe(int64_t iters, double *sink, double *flops,
                                              void *stream) {
    if (iters < 1 || !sink || !flops) return TETPROJ_ERR_ARG;
    const int blocks = 8 * tp::device_sm_count();
    tp::k_fma64<<<blocks, tp::kFmaThreads, 0, (cudaStream_t)stream>>>(iters, 0.999999, 1e-6, sink);
    tp::note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return TETPROJ_ERR_CUDA;
    *flops = 2.0 * tp::kFmaChains * (double)iters * (double)blocks * tp::kFmaThreads;
    return TETPROJ_OK;
}

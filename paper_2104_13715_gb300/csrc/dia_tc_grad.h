// Tensor-core weight gradient and the evaluation built on it (dia_tc_grad.cu).
#pragma once

#include <cuda_runtime.h>

#include "dia_eval.cuh"

namespace dia {

constexpr int kTcGradMaxM = 31;

int tc_grad_smem_bytes();
// After the tensor-core forward pass has written D = I - M (valid region,
// pitch Wv): amax[0..1] (zeroed by the caller) <- max |R|, max |g|; G <- g =
// dl/dM (0 where masked); partial rows [0, sms) <- loss, dL/dB0, pixel count,
// curvature sums; rows [sms, 2 sms) <- dL/dK from the tensor-core kernel.
// np = red_size(m*m).  *status is set to 1 if a bounded wait ran out.
cudaError_t launch_tc_grad_eval(const EvalArgs &ea, int m, const float *D, float *G,
                                unsigned *amax, double *partials, int np, int sms,
                                int *status, cudaStream_t s);

}  // namespace dia

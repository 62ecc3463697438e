// Table of the fused evaluation kernels, one instantiation per odd kernel side.
#pragma once

#include <cuda_runtime.h>

namespace dia {

struct KernelInfo {
    int mk, nw, qf, th, nt, smem, np, kp;
    const void *fn[2];   // [kModeGrad], [kModeForward]
};

// Fills `out` for kernel side mk (odd, 1..31); false if there is none.
bool kernel_info(int mk, KernelInfo *out);

}  // namespace dia

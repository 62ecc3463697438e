// Table of the fused evaluation kernels: one instantiation per odd kernel
// side and tile variant (see gen_instances.py).
#pragma once

#include <cuda_runtime.h>

namespace dia {

constexpr int kMaxKernelSide = 31;

struct KernelInfo {
    int mk, variant, nw, qf, minb, th, nt, smem, np, kp, f2;
    const void *fn[2];      // [kModeGrad], [kModeForward]: constant background B0
    const void *fn_bg[2];   // the same with the polynomial background (Eq. 18)
};

// Kernel of side mk (odd, 1..31) in its currently selected tile variant.
bool kernel_info(int mk, KernelInfo *out);
// A specific variant; false if there is none.
bool kernel_info_variant(int mk, int variant, KernelInfo *out);
// Number of tile variants for side mk (0 if unsupported).
int kernel_variants(int mk);
// Process-wide choice of variant for side mk (default 0).
bool select_variant(int mk, int variant);
int selected_variant(int mk);

}  // namespace dia

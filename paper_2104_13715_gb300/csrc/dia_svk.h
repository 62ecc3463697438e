// Fused evaluation with a spatially varying kernel (dia_svk.cu): each kernel
// pixel a polynomial of degree dk in the coordinates of Eq. 19.
#pragma once

#include <cuda_runtime.h>

#include "dia_eval.cuh"

namespace dia {

constexpr int kSvkMaxDeg = 2;                                        // largest kernel degree
constexpr int kSvkMaxNc = (kSvkMaxDeg + 1) * (kSvkMaxDeg + 2) / 2;  // coefficient kernels

struct SvkArgs {
    int kdeg;   // kernel degree dk
    int nc;     // coefficient kernels (dk+1)(dk+2)/2
    int np;     // partials per CTA: red_size(nc * m * m)
};

// Output rows per tile of the kernel (tiles are tile_rows x 128 pixels).
int svk_tile_rows();
// Sets the shared-memory attribute of both modes; CTAs per SM and smem bytes.
cudaError_t svk_prepare(int mk, int *occ, int *smem);
// One launch over a.n_tiles tiles (a.tiles_x, a.n_tiles in this kernel's
// tiling); mode kModeGrad writes per-CTA partials, kModeForward the
// difference image / clip mask.  Kpad: nc blocks of m rows x kp floats, then
// kBgMax + 1 background slots.
cudaError_t launch_eval_svk(const EvalArgs &a, const SvkArgs &v, int mk, int mode, int grid,
                            cudaStream_t s);

}  // namespace dia

// Small-kernel (m = 1, 3, 5) fused evaluation: warp-private strips streamed
// through a cp.async row ring (dia_small.cu).  Same per-CTA partials as the
// tiled kernel, so the same reduction follows it.
#pragma once

#include <cuda_runtime.h>

#include "dia_eval.cuh"

namespace dia {

// Work split of one launch: strips of band_rows output rows by 128 columns.
struct SmallGeom {
    int col_blocks, band_rows, n_strips;
    int kp;   // row pitch of Kpad
    int np;   // partials per CTA (red_size(m*m))
};

// True when the small kernel can evaluate these arguments: m in {1, 3, 5},
// constant background, float64 accumulation, 16-byte aligned images with a
// row pitch of a multiple of 4 floats (and of 16 bytes for a mask).
bool small_kernel_ok(const EvalArgs &a, int mk);
// Shared-memory bytes per CTA for these arguments' maps.
int small_kernel_smem(const EvalArgs &a);
// Sets the kernel's shared-memory attribute and returns its CTAs per SM.
cudaError_t small_kernel_prepare(const EvalArgs &a, int mk, int *occ);
SmallGeom small_geometry(const EvalArgs &a, int mk, int kp, int np, int grid);
// Gradient-mode evaluation over the whole valid region into a.partials
// (grid rows of np doubles); honours a.done_flag.
cudaError_t launch_eval_small(const EvalArgs &a, int mk, int kp, int np, int grid,
                              cudaStream_t s);

}  // namespace dia

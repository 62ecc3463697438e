// Tensor-core weight gradient (dia_tc_grad.cu).
#pragma once

#include <cuda_runtime.h>

#include "dia_eval.cuh"

namespace dia {

constexpr int kTcGradMaxM = 31;
constexpr int kTcGradTileRows = 128;   // g tile rows (the padded height is a multiple)
constexpr int kTcGradTileCols = 64;    // g tile columns (the padded width is a multiple)

int tc_grad_smem_bytes();
// dL/dK from the g map G (valid region padded with zeros to Hp x Wp, pitch
// gld: Hp a multiple of kTcGradTileRows, Wp of kTcGradTileCols, gld >= Wp a
// multiple of 4, G 16-byte aligned) and R (H x W, pitch ld), with amax[0..1]
// = max |R|, max |g| (float bits) already reduced: partial rows [0, rows)
// (np = red_size(m*m) doubles each) get dK at 1 .. m*m and 0 elsewhere.
// *status is set to 1 if a bounded wait ran out.
// done (nullable): nonzero -> the kernel returns at once (a converged fit's graph).
cudaError_t launch_tc_grad(const float *R, int H, int W, int ld, int m, const float *G, int gld,
                           int Hp, int Wp, const unsigned *amax, double *partials, int np,
                           int rows, int *status, long long wait_cycles, cudaStream_t s,
                           const int *done = nullptr);
// the kernel's shared-memory attribute, once per process (call before a capture)
cudaError_t tc_grad_prepare();

}  // namespace dia

// Batched evaluation kernels of kernel-side group 0.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_0(int mode) {
    return mode == kModeGrad ? (const void *)&eval_batch_kernel<0, kModeGrad>
                             : (const void *)&eval_batch_kernel<0, kModeForward>;
}
}  // namespace dia

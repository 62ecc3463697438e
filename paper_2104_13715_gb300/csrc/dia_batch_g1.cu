// Batched evaluation kernels of kernel-side group 1.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_1(int mode) {
    return mode == kModeGrad ? (const void *)&eval_batch_kernel<1, kModeGrad>
                             : (const void *)&eval_batch_kernel<1, kModeForward>;
}
}  // namespace dia

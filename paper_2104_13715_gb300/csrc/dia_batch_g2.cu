// Batched evaluation kernels of kernel-side group 2.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_2(int mode) {
    return mode == kModeGrad ? (const void *)&eval_batch_kernel<2, kModeGrad>
                             : (const void *)&eval_batch_kernel<2, kModeForward>;
}
}  // namespace dia

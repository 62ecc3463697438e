// Batched evaluation kernels of kernel-side group 3.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_3(int mode) {
    return mode == kModeGrad ? (const void *)&eval_batch_kernel<3, kModeGrad>
                             : (const void *)&eval_batch_kernel<3, kModeForward>;
}
}  // namespace dia

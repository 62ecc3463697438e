// Batched evaluation kernels of kernel-side group 1, polynomial background.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_bg_1(int mode) {
    return mode == kModeGrad ? (const void *)&eval_batch_kernel<1, kModeGrad, 1>
                             : (const void *)&eval_batch_kernel<1, kModeForward, 1>;
}
}  // namespace dia

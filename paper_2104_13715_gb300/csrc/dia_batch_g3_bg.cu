// Batched evaluation kernels of kernel-side group 3, polynomial background.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_bg_3(int mode) {
    return mode == kModeGrad ? (const void *)&eval_batch_kernel<3, kModeGrad, 1>
                             : (const void *)&eval_batch_kernel<3, kModeForward, 1>;
}
}  // namespace dia

// Batched evaluation kernels of kernel-side group 0, polynomial background.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_bg_0(int mode) {
    return mode == kModeGrad ? (const void *)&eval_batch_kernel<0, kModeGrad, 1>
                             : (const void *)&eval_batch_kernel<0, kModeForward, 1>;
}
}  // namespace dia

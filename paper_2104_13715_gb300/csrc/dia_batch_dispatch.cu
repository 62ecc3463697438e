// Pointers of the batched evaluation kernels by kernel-side group.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_0(int mode);
const void *batch_kernel_ptr_1(int mode);
const void *batch_kernel_ptr_2(int mode);
const void *batch_kernel_ptr_3(int mode);

const void *batch_kernel_ptr(int group, int mode) {
    switch (group) {
        case 0: return batch_kernel_ptr_0(mode);
        case 1: return batch_kernel_ptr_1(mode);
        case 2: return batch_kernel_ptr_2(mode);
        default: return batch_kernel_ptr_3(mode);
    }
}
}  // namespace dia

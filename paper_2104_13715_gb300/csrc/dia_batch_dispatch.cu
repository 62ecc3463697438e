// Pointers of the batched evaluation kernels by kernel-side group.
#include "dia_batch.cuh"

namespace dia {
const void *batch_kernel_ptr_0(int mode);
const void *batch_kernel_ptr_1(int mode);
const void *batch_kernel_ptr_2(int mode);
const void *batch_kernel_ptr_3(int mode);
const void *batch_kernel_ptr_bg_0(int mode);
const void *batch_kernel_ptr_bg_1(int mode);
const void *batch_kernel_ptr_bg_2(int mode);
const void *batch_kernel_ptr_bg_3(int mode);

const void *batch_kernel_ptr(int group, int mode, int bg) {
    switch (group) {
        case 0: return bg ? batch_kernel_ptr_bg_0(mode) : batch_kernel_ptr_0(mode);
        case 1: return bg ? batch_kernel_ptr_bg_1(mode) : batch_kernel_ptr_1(mode);
        case 2: return bg ? batch_kernel_ptr_bg_2(mode) : batch_kernel_ptr_2(mode);
        default: return bg ? batch_kernel_ptr_bg_3(mode) : batch_kernel_ptr_3(mode);
    }
}
}  // namespace dia

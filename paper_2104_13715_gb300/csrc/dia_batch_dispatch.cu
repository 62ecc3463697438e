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

// One block per group: an order-preserving compaction by block-wide prefix
// sums over chunks of the block size.
constexpr int kCompactThreads = 1024;

__global__ void __launch_bounds__(kCompactThreads)
    compact_items_kernel(const BatchItem *items, const EvalArgs *eas, const int *gbeg,
                         BatchItem *act, int *n_act) {
    __shared__ int warp_cnt[kCompactThreads / 32];
    __shared__ int base;
    const int g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b0 = gbeg[g], b1 = gbeg[g + 1];
    if (tid == 0) base = 0;
    __syncthreads();
    for (int c0 = b0; c0 < b1; c0 += kCompactThreads) {
        const int i = c0 + tid;
        bool keep = false;
        BatchItem it;
        if (i < b1) {
            it = items[i];
            const int *df = eas[it.pair].done_flag;
            keep = df == nullptr || *((volatile const int *)df) == 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) {
            if (w < warp) before += warp_cnt[w];
            total += warp_cnt[w];
        }
        if (keep) act[b0 + base + before + __popc(bal & ((1u << lane) - 1u))] = it;
        __syncthreads();   // every thread has read base and warp_cnt
        if (tid == 0) base += total;
        __syncthreads();
    }
    if (tid == 0) n_act[g] = base;
}

cudaError_t launch_compact_items(const BatchItem *items, const EvalArgs *eas, const int *gbeg,
                                 BatchItem *act, int *n_act, cudaStream_t s) {
    compact_items_kernel<<<4, kCompactThreads, 0, s>>>(items, eas, gbeg, act, n_act);
    return cudaGetLastError();
}

const void *batch_kernel_ptr(int group, int mode, int bg) {
    switch (group) {
        case 0: return bg ? batch_kernel_ptr_bg_0(mode) : batch_kernel_ptr_0(mode);
        case 1: return bg ? batch_kernel_ptr_bg_1(mode) : batch_kernel_ptr_1(mode);
        case 2: return bg ? batch_kernel_ptr_bg_2(mode) : batch_kernel_ptr_2(mode);
        default: return bg ? batch_kernel_ptr_bg_3(mode) : batch_kernel_ptr_3(mode);
    }
}
}  // namespace dia

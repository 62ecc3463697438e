// Batched fused-evaluation kernel (see dia_batch.cu).  Each kernel-side group
// is instantiated in its own translation unit (dia_batch_gN.cu).
#pragma once

#include "dia_eval.cuh"

namespace dia {

constexpr int kBW = 8;             // warps per CTA of the batched kernel
constexpr int kBQF = 4;            // output rows per warp in the forward pass
constexpr int kBTH = kBW * kBQF;   // tile rows
constexpr int kChunkTiles = 2;     // tiles per work item

// per kernel side: prefetch flag and backward split of the batched kernel
#define DIA_BATCH_SIDES(X)                                                                    \
    X(1, 0, 0) X(3, 0, 0) X(5, 0, 0) X(7, 0, 0) X(9, 0, 1) X(11, 1, 1) X(13, 1, 1) X(15, 0, 0) \
        X(17, 0, 1) X(19, 1, 1) X(21, 0, 0) X(23, 0, 0) X(25, 0, 1) X(27, 0, 0) X(29, 0, 0)   \
            X(31, 0, 0)

constexpr int batch_max_smem() {
    int mx = 0;
#define DIA_SMEM(MKV, PFV, SPV) \
    mx = EvalShape<MKV, kBW, kBQF, SPV>::SMEM > mx ? EvalShape<MKV, kBW, kBQF, SPV>::SMEM : mx;
    DIA_BATCH_SIDES(DIA_SMEM)
#undef DIA_SMEM
    return mx;
}
constexpr int kBatchSmem = batch_max_smem();

constexpr int np_of(int mk) { return red_size(mk * mk); }

struct BatchItem {
    int pair, t0, t1, pad;
    long long part_off;
};

// Kernel-side groups: 0 = {1,3,5,7}, 1 = {9,11,13,15}, 2 = {17,19,21,23},
// 3 = {25,27,29,31}.
__host__ __device__ constexpr int batch_group(int mk) { return mk <= 7 ? 0 : mk <= 15 ? 1 : mk <= 23 ? 2 : 3; }

// BG = 1: pairs may have a polynomial background (EvalArgs::bg_deg > 0)
template <int GROUP, int MODE, int BG = 0>
__global__ void __launch_bounds__(kBW * 32, 1)
    eval_batch_kernel(const EvalArgs *eas, const int *mks, const BatchItem *items, int n_items,
                      int *counter, double *partials) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ EvalArgs s_ea;
    __shared__ int s_it;
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_it;
        if (it >= n_items) break;
        const BatchItem item = items[it];
        if (threadIdx.x == 0) s_ea = eas[item.pair];
        __syncthreads();
        const bool skip = MODE == kModeGrad && s_ea.done_flag != nullptr &&
                          *((volatile const int *)s_ea.done_flag) != 0;
        if (!skip) {
            double *out = MODE == kModeGrad ? partials + item.part_off : nullptr;
            switch (mks[item.pair]) {
#define DIA_CASE(MKV, PFV, SPV)                                                              \
    case MKV:                                                                                \
        if constexpr (batch_group(MKV) == GROUP)                                             \
            process_tiles<MKV, kBW, kBQF, PFV, SPV, MODE, 0, BG>(s_ea, smem, item.t0, item.t1, 1, out); \
        break;
                DIA_BATCH_SIDES(DIA_CASE)
#undef DIA_CASE
                default: break;
            }
        }
        __syncthreads();   // s_ea, s_it are rewritten for the next item
    }
}

// kernel pointers of a group (defined in dia_batch_gN.cu, dia_batch_gN_bg.cu)
const void *batch_kernel_ptr(int group, int mode, int bg);

}  // namespace dia

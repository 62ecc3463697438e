// Batched fused-evaluation kernel (see dia_batch.cu).  Each kernel-side group
// is instantiated in its own translation unit (dia_batch_gN.cu).
#pragma once

#include "dia_eval.cuh"

namespace dia {

constexpr int kBW = 8;             // warps per CTA of the batched kernel
constexpr int kBQF = 4;            // output rows per warp in the forward pass
constexpr int kBTH = kBW * kBQF;   // tile rows
constexpr int kMaxChunkTiles = 32;  // longest run of tiles in one work item

// per kernel side: prefetch flag, backward split and packed-float2 forward
// (F2: bitwise the scalar forward) of the batched kernel
#define DIA_BATCH_SIDES(X)                                                                   \
    X(1, 0, 0, 0) X(3, 0, 0, 0) X(5, 0, 0, 0) X(7, 0, 0, 1) X(9, 0, 1, 1) X(11, 1, 1, 1)     \
        X(13, 1, 1, 1) X(15, 0, 0, 1) X(17, 0, 1, 1) X(19, 1, 1, 1) X(21, 0, 0, 1)           \
            X(23, 0, 0, 1) X(25, 0, 1, 1) X(27, 0, 0, 1) X(29, 0, 0, 1) X(31, 0, 0, 1)


constexpr int np_of(int mk) { return red_size(mk * mk); }

// Work-item size of the batched evaluation: tiles per item for kernel side
// mk under variant v of its group, about c_v * 441 / mk^2 tiles (equal work
// per item across sides) with c = 2, 1, 4, 8 for v = 0..3, within [1, 32].
constexpr int kBatchVariants = 4;
inline int batch_chunk(int mk, int v) {
    const double c = v == 1 ? 1.0 : v == 2 ? 4.0 : v == 3 ? 8.0 : 2.0;
    int t = (int)(c * 441.0 / (double)(mk * mk) + 0.5);
    return t < 1 ? 1 : (t > kMaxChunkTiles ? kMaxChunkTiles : t);
}

struct BatchItem {
    int pair, t0, t1, pad;
    long long part_off;
};

// Kernel-side groups: 0 = {1,3,5,7}, 1 = {9,11,13,15}, 2 = {17,19,21,23},
// 3 = {25,27,29,31}.
__host__ __device__ constexpr int batch_group(int mk) { return mk <= 7 ? 0 : mk <= 15 ? 1 : mk <= 23 ? 2 : 3; }

// shared memory of the kernel of group g (its largest side)
constexpr int batch_group_smem(int g) {
    int mx = 0;
#define DIA_SMEM_G(MKV, PFV, SPV, F2V)                                                            \
    if (batch_group(MKV) == g && EvalShape<MKV, kBW, kBQF, SPV, F2V>::SMEM > mx)                \
        mx = EvalShape<MKV, kBW, kBQF, SPV, F2V>::SMEM;
    DIA_BATCH_SIDES(DIA_SMEM_G)
#undef DIA_SMEM_G
    return mx;
}

// BG = 1: pairs may have a polynomial background (EvalArgs::bg_deg > 0)
// n_items: device count of the items to walk (the compacted list of the
// pairs still running, or every item for the final forward pass)
// groups 0 and 1 (m <= 15) fit two CTAs per SM (registers <= 128)
template <int GROUP, int MODE, int BG = 0>
__global__ void __launch_bounds__(kBW * 32, GROUP <= 1 ? 2 : 1)
    eval_batch_kernel(const EvalArgs *eas, const int *mks, const BatchItem *items,
                      const int *n_items_ptr, int *counter, double *partials) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ EvalArgs s_ea;
    __shared__ int s_it;
    const int n_items = *n_items_ptr;
    constexpr int kEaWords = (int)(sizeof(EvalArgs) / 4);
    static_assert(sizeof(EvalArgs) % 4 == 0, "EvalArgs is copied as words");
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_it;
        if (it >= n_items) break;
        const BatchItem item = items[it];
        // the pair's descriptor, copied by the first warps word by word
        if (threadIdx.x < kEaWords)
            reinterpret_cast<int *>(&s_ea)[threadIdx.x] =
                reinterpret_cast<const int *>(eas + item.pair)[threadIdx.x];
        __syncthreads();
        const bool skip = MODE == kModeGrad && s_ea.done_flag != nullptr &&
                          *((volatile const int *)s_ea.done_flag) != 0;
        if (!skip) {
            double *out = MODE == kModeGrad ? partials + item.part_off : nullptr;
            switch (mks[item.pair]) {
#define DIA_CASE(MKV, PFV, SPV, F2V)                                                         \
    case MKV:                                                                                \
        if constexpr (batch_group(MKV) == GROUP)                                             \
            process_tiles<MKV, kBW, kBQF, PFV, SPV, MODE, F2V, BG>(s_ea, smem, item.t0, item.t1, 1, out); \
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

// Work items of the pairs that are still running, per kernel-side group, in
// their planned order (largest first): block g compacts items[gbeg[g],
// gbeg[g+1]) into act[gbeg[g] ...] and writes the count to n_act[g].
cudaError_t launch_compact_items(const BatchItem *items, const EvalArgs *eas, const int *gbeg,
                                 BatchItem *act, int *n_act, cudaStream_t s);

}  // namespace dia

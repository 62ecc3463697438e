// Tensor-core form of the forward model image (Sec. 2.1, Eq. 2) for sm_103a:
// tcgen05.mma with bf16 operands in shared memory, float32 accumulators in
// tensor memory, three split-precision products per contraction.
//
// The correlation as a GEMM.  An output tile is NO = 32 rows (i) x 128 columns
// (j) from valid-region pixel (y0, x0); its R window is 64 rows (y) x 160
// columns (x) from full-image pixel (y0, x0).  With i' = NO - 1 - i (output rows
// in reverse order),
//   D[j][i'] = sum_b sum_y A_b[j][y] B_b[i'][y],
//   A_b[j][y]  = R[y0 + y][x0 + j + b]          (the R window shifted by b columns)
//   B_b[i'][y] = K[y + i' - (NO - 1)][b]         (0 outside [0, m)),
// so D[j][i'] = M[y0 + i][x0 + j] - B0.  The R window is stored column-major in
// 8-row chunks, T[y / 8][x][y % 8], so the 8 x 8 core matrices of A_b (rows j, K
// index y) are contiguous 128-byte blocks for every column shift b: A_b is the
// same array with its start moved by b * 16 bytes, and R is staged once per
// tile.  B_b is a Hankel matrix in (i', y) of the vector kb[s] = K[s - (NO - 1)][b]:
// one array Zk_b[c][t][e] = kb[8c + t + e] holds all of its core matrices (core
// matrix (I, Y) is block I + Y; both descriptor strides 128 bytes), built once per
// CTA for every b.
//
// Precision: x = hi + lo with hi = bf16(x), lo = bf16(x - hi) for R and K; the
// three products hi*hi + hi*lo + lo*hi are accumulated in float32 (the omitted
// lo*lo term is below 2^-16 of each product).
//
// Persistent CTAs (one per SM), warp-specialised: the R window of the next
// tile arrives by TMA (cp.async.bulk.tensor, 2-D tiled map, zero fill outside
// the image; cp.async when the rows are not 16-byte aligned or the image is
// smaller than one 160 x 64 box); warps 0-3 split
// tile k's window into T[k & 1] (signalled on tfull) and, one tile behind, read the
// accumulators of the previous tile from tensor memory and write D = I - M
// (signalled on aempty); warp 4 owns the tensor memory (two 32-column
// accumulators) and, on one lane, issues each tile's m x (K steps) x 3 MMAs and
// commits them to tempty (T buffer free) and afull (accumulators ready).  Every
// wait is bounded and any failed wait aborts the whole CTA.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/dia.h"
#include "dia_ops.cuh"
#include "dia_tc_ptx.cuh"

namespace dia {

namespace {

constexpr int kTcNO = 32;                  // output rows per tile (MMA N)
constexpr int kTcW = 128;                  // output columns per tile (MMA M)
constexpr int kTcXT = kTcW + 32;           // R window columns (m <= 33)
constexpr int kTcYT = 64;                  // R window rows (NO + m - 1 <= 64)
constexpr int kTcYC = kTcYT / 8;           // 8-row chunks of the window
constexpr int kTcKC = 12;                  // 16-byte chunks of one Zk_b (>= (NO + YT) / 8 + 1)
constexpr int kTcMaxM = 31;
constexpr int kTcProducers = 128;          // warps 0-3
constexpr int kTcThreads = kTcProducers + 32;

struct TcSmem {
    float f[kTcYT][kTcXT];                        // next tile's R window (cp.async)
    __nv_bfloat16 t[2][2][kTcYC][kTcXT][8];       // [buffer][hi|lo][y / 8][x][y % 8]
    __nv_bfloat16 zk[2][kTcMaxM][kTcKC * 64];     // [hi|lo][b][c][t][e]
    uint64_t tfull[2];    // T buffer staged (128 producer arrivals)
    uint64_t tempty[2];   // T buffer read by its MMAs (tcgen05.commit)
    uint64_t afull[2];    // accumulators final (tcgen05.commit)
    uint64_t aempty[2];   // accumulators read back (128 producer arrivals)
    uint64_t wfull;       // the TMA window copy landed (1 arrival + 40960 bytes)
    uint32_t tslot;
    int mma_abort;        // set by the MMA warp when a wait of its own ran out
    int prod_abort;       // set by a producer (read by the MMA warp's waits)
};

// Barrier 1 over the 128 producer threads with an OR reduction of `fail`: every
// producer gets the same answer, so they all leave the pipeline together.
__device__ __forceinline__ bool producers_any(bool fail) {
    uint32_t any;
    asm volatile("{\n\t.reg .pred q, p;\n\tsetp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(any) : "r"((uint32_t)fail), "n"(kTcProducers) : "memory");
    return any != 0;
}

// cp.async of the R window of the tile at (y0, x0) into f (zeros outside the
// image and past the window rows a kernel tap reaches); 16-byte copies when
// rows are 16-byte aligned
__device__ __forceinline__ void tc_prefetch(float (*f)[kTcXT], const float *R, int H, int W,
                                            int ld, int y0, int x0, int ylim, bool vec) {
    if (vec) {
        for (int i = threadIdx.x; i < kTcYT * (kTcXT / 4); i += kTcProducers) {
            const int yy = i / (kTcXT / 4), c4 = i % (kTcXT / 4);
            const int gy = y0 + yy, gx = x0 + 4 * c4;
            int bytes = 0;
            const float *src = R;
            if (yy < ylim && gy < H && gx < W) {
                bytes = (W - gx >= 4) ? 16 : 4 * (W - gx);
                src = R + (size_t)gy * ld + gx;
            }
            cp_async16(&f[yy][4 * c4], src, bytes);
        }
    } else {
        for (int i = threadIdx.x; i < kTcYT * kTcXT; i += kTcProducers) {
            const int yy = i / kTcXT, x = i % kTcXT;
            const int gy = y0 + yy, gx = x0 + x;
            const bool in = yy < ylim && gy < H && gx < W;
            cp_async4(&f[yy][x], in ? R + (size_t)gy * ld + gx : R, in ? 4 : 0);
        }
    }
    cp_async_commit();
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

struct TcArgs {
    const float *R, *I;
    int H, W, ld, m;
    int Hv, Wv, tiles_x, n_tiles;
    const float *Kpad;   // m rows of kp floats, then B0
    int kp;
    float *diff_out;     // (Hv x Wv) D = I - M
    int *status;         // set to 1 if a wait ran out
    int use_tma;         // 1: the window by TMA through `tmap`
    long long wait_cycles;   // limit of each pipeline wait (SM clock cycles)
};

constexpr uint32_t kTcWindowBytes = kTcYT * kTcXT * 4;

// one elected thread: the window of the tile at (y0, x0) into f by TMA
__device__ __forceinline__ void tc_tma_window(TcSmem &S, const CUtensorMap *tmap, int y0, int x0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(su32(&S.wfull)), "r"(kTcWindowBytes) : "memory");
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3}], [%4];"
                 :: "r"(su32(&S.f[0][0])), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x0), "r"(y0),
                    "r"(su32(&S.wfull))
                 : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1)
    tc_forward_kernel(const TcArgs a, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m, h = m / 2;
    const int nks = (kTcNO + m - 1 + 15) / 16;   // K steps of 16 window rows

    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&S.tslot)), "r"(64));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.tfull[i], kTcProducers);
            mbar_init(&S.tempty[i], 1);
            mbar_init(&S.afull[i], 1);
            mbar_init(&S.aempty[i], kTcProducers);
        }
        mbar_init(&S.wfull, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        S.mma_abort = 0;
        S.prod_abort = 0;
    }
    // Zk_b[c][t][e] = K[8c + t + e - (NO - 1)][b] (0 outside the kernel)
    for (int i = tid; i < m * kTcKC * 64; i += kTcThreads) {
        const int b = i / (kTcKC * 64), q = i % (kTcKC * 64);
        const int c = q / 64, t = (q / 8) % 8, e = q % 8;
        const int ar = 8 * c + t + e - (kTcNO - 1);
        const float v = (ar >= 0 && ar < m) ? a.Kpad[ar * a.kp + b] : 0.f;
        split_bf16(v, S.zk[0][b][q], S.zk[1][b][q]);
    }
    const float B0 = a.Kpad[m * a.kp];
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = S.tslot;

    if (warp == 4) {
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(kTcW, kTcNO);
            // A_b (ks): T + ((2 ks) XT + b) 16 bytes; B_b (ks): Zk_b + 2 ks 128 bytes
            const uint64_t dt0 = tc_desc(su32(&S.t[0][0][0][0][0]), kTcXT * 16, 128);
            const uint64_t dz0 = tc_desc(su32(&S.zk[0][0][0]), 128, 128);
            constexpr uint32_t kTbuf = sizeof(S.t[0]), kTsplit = sizeof(S.t[0][0]);
            constexpr uint32_t kZsplit = sizeof(S.zk[0]), kZb = sizeof(S.zk[0][0]);
            int k = 0;
            for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++k) {
                const int buf = k & 1;
                if (!tc_wait(&S.tfull[buf], (uint32_t)((k >> 1) & 1), &S.prod_abort,
                             a.wait_cycles) ||
                    (k >= 2 && !tc_wait(&S.aempty[buf], (uint32_t)(((k - 2) >> 1) & 1),
                                        &S.prod_abort, a.wait_cycles))) {
                    *reinterpret_cast<volatile int *>(&S.mma_abort) = 1;
                    atomicExch(a.status, 1);
                    // the MMAs already issued (tiles < k) must finish before the
                    // tensor memory is released: their last commit arrives on
                    // afull of tile k - 1 (waited with the long limit)
                    if (k > 0) {
                        const int never = 0;
                        tc_wait(&S.afull[(k - 1) & 1], (uint32_t)(((k - 1) >> 1) & 1), &never);
                    }
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t acc = tmem + (uint32_t)(buf * kTcNO);
                for (int b = 0; b < m; ++b) {
                    const uint64_t tb = dt0 + ((buf * kTbuf + b * 16) >> 4);
                    const uint64_t zb = dz0 + ((b * kZb) >> 4);
                    for (int ks = 0; ks < nks; ++ks) {
                        const uint64_t ahi = tb + ((2 * ks * kTcXT * 16) >> 4), alo = ahi + (kTsplit >> 4);
                        const uint64_t bhi = zb + ((2 * ks * 128) >> 4), blo = bhi + (kZsplit >> 4);
                        tc_mma(acc, ahi, bhi, idesc, (b > 0 || ks > 0) ? 1 : 0);
                        tc_mma(acc, ahi, blo, idesc, 1);
                        tc_mma(acc, alo, bhi, idesc, 1);
                    }
                }
                tc_commit(&S.tempty[buf]);
                tc_commit(&S.afull[buf]);
            }
        }
        __syncwarp();
    } else {
        // returns false if the accumulators did not arrive
        auto epilogue = [&](int kk, int tile) {
            const int buf = kk & 1;
            bool ok = tc_wait(&S.afull[buf], (uint32_t)((kk >> 1) & 1), &S.mma_abort,
                              a.wait_cycles);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) return false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t v[kTcNO];
            const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * kTcNO);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                           "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                           "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
                           "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                           "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]),
                           "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                         : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&S.aempty[buf]);
            const int y0 = (tile / a.tiles_x) * kTcNO, x0 = (tile % a.tiles_x) * kTcW;
            const int x = x0 + 32 * warp + lane;
            if (x < a.Wv) {
#pragma unroll
                for (int ip = 0; ip < kTcNO; ++ip) {
                    const int y = y0 + kTcNO - 1 - ip;
                    if (y < a.Hv) {
                        const float Iv = __ldg(a.I + (size_t)(y + h) * a.ld + (x + h));
                        a.diff_out[(size_t)y * a.Wv + x] = Iv - (__uint_as_float(v[ip]) + B0);
                    }
                }
            }
            return true;
        };
        const bool vec = ((a.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.R) & 15) == 0);
        const int ylim = kTcNO + m - 1;   // window rows with a nonzero kernel weight
        auto origin = [&](int tile, int &y0, int &x0) {
            y0 = (tile / a.tiles_x) * kTcNO;
            x0 = (tile % a.tiles_x) * kTcW;
        };
        int y0, x0;
        int tma_issued = 0;   // TMA windows requested (thread 0), each consumed in order
        if ((int)blockIdx.x < a.n_tiles) {
            origin(blockIdx.x, y0, x0);
            if (a.use_tma) {
                if (tid == 0) tc_tma_window(S, &tmap, y0, x0);
                tma_issued = 1;
            } else {
                tc_prefetch(S.f, a.R, a.H, a.W, a.ld, y0, x0, ylim, vec);
            }
        }
        bool fail = false;
        int k = 0, prev = -1;
        for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++k) {
            const int buf = k & 1;
            // the window has landed (TMA: the transaction count of wfull; cp.async:
            // each thread's own copies, then everyone's at the barrier)
            if (a.use_tma)
                fail = fail || !tc_wait(&S.wfull, (uint32_t)(k & 1), &S.mma_abort, a.wait_cycles);
            else
                cp_async_wait<0>();
            if (k >= 2 && !fail)
                fail = !tc_wait(&S.tempty[buf], (uint32_t)(((k - 2) >> 1) & 1), &S.mma_abort,
                                a.wait_cycles);
            if (producers_any(fail)) {
                fail = true;
                break;
            }
            // T[buf][.][yc][x][e] = split(f[8 yc + e][x])
#pragma unroll 2
            for (int u = tid; u < kTcYC * kTcXT; u += kTcProducers) {
                const int yc = u / kTcXT, x = u % kTcXT;
                __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) split_bf16(S.f[8 * yc + e][x], hi[e], lo[e]);
                *reinterpret_cast<uint4 *>(&S.t[buf][0][yc][x][0]) = *reinterpret_cast<const uint4 *>(hi);
                *reinterpret_cast<uint4 *>(&S.t[buf][1][yc][x][0]) = *reinterpret_cast<const uint4 *>(lo);
            }
            asm volatile("fence.proxy.async.shared::cta;");
            mbar_arrive(&S.tfull[buf]);
            // every producer has read f: request the next tile's window
            if (producers_any(fail)) {
                fail = true;
                break;
            }
            if (tile + (int)gridDim.x < a.n_tiles) {
                origin(tile + gridDim.x, y0, x0);
                if (a.use_tma) {
                    if (tid == 0) tc_tma_window(S, &tmap, y0, x0);
                    ++tma_issued;
                } else {
                    tc_prefetch(S.f, a.R, a.H, a.W, a.ld, y0, x0, ylim, vec);
                }
            }
            if (prev >= 0 && !epilogue(k - 1, prev)) fail = true;
            prev = tile;
        }
        if (!fail && prev >= 0 && !epilogue(k - 1, prev)) fail = true;
        cp_async_wait<0>();
        // after a failure, the last window requested must land (or its wait run
        // out) before the CTA's shared memory is released
        if (fail && a.use_tma && tid == 0 && tma_issued > 0) {
            const int never = 0;
            tc_wait(&S.wfull, (uint32_t)((tma_issued - 1) & 1), &never);
        }
        if (fail) {
            *reinterpret_cast<volatile int *>(&S.prod_abort) = 1;
            if (lane == 0) atomicExch(a.status, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(64));
}

}  // namespace

int tc_smem_bytes() { return (int)sizeof(TcSmem); }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to
// the driver library); nullptr if unavailable
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

cudaError_t launch_tc_forward(const float *R, const float *I, int H, int W, int ld, int m,
                              const float *Kpad, int kp, float *diff_out, int *status,
                              cudaStream_t s, long long wait_cycles) {
    if (m < 1 || m > kTcMaxM || (m & 1) == 0) return cudaErrorInvalidValue;
    // 2-D tiled map of R (x innermost): 160 x 64 float boxes, zero fill outside;
    // needs a 16-byte aligned base and row pitch; images smaller than one box
    // take the cp.async path
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    int use_tma = 0;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc && (ld % 4) == 0 && (reinterpret_cast<uintptr_t>(R) % 16) == 0 && W >= kTcXT &&
        H >= kTcYT) {
        const cuuint64_t gdim[2] = {(cuuint64_t)W, (cuuint64_t)H};
        const cuuint64_t gstride[1] = {(cuuint64_t)ld * 4};
        const cuuint32_t box[2] = {(cuuint32_t)kTcXT, (cuuint32_t)kTcYT};
        const cuuint32_t estride[2] = {1, 1};
        if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(R), gdim, gstride,
                box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            use_tma = 1;
    }
    TcArgs a;
    a.R = R;
    a.I = I;
    a.H = H;
    a.W = W;
    a.ld = ld;
    a.m = m;
    a.Hv = H - 2 * (m / 2);
    a.Wv = W - 2 * (m / 2);
    a.tiles_x = (a.Wv + kTcW - 1) / kTcW;
    a.n_tiles = a.tiles_x * ((a.Hv + kTcNO - 1) / kTcNO);
    a.Kpad = Kpad;
    a.kp = kp;
    a.diff_out = diff_out;
    a.status = status;
    a.use_tma = use_tma;
    a.wait_cycles = wait_cycles > 0 ? wait_cycles : kTcWaitCycles;
    int dev = 0, sms = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int smem = tc_smem_bytes();
    e = cudaFuncSetAttribute(tc_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = a.n_tiles < sms ? a.n_tiles : sms;
    tc_forward_kernel<<<grid, kTcThreads, smem, s>>>(a, tmap);
    return cudaGetLastError();
}

}  // namespace dia

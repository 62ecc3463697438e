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
// smaller than one 160 x 64 box); warps 0-3 split tile k's window into
// T[k & 1] (signalled on tfull); warp 8 owns the tensor memory (two 32-column
// accumulators) and, on one lane, issues each tile's m x (K steps) x 3 MMAs and
// commits them to tempty (T buffer free) and afull (accumulators ready); warps
// 4-7 read the accumulators back (signalled on aempty) and write D = I - M or,
// in loss mode, g = dl/dM with the loss sums, their loads issued 8 rows at a
// time.  Every wait is bounded and any failed wait aborts the whole CTA.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>
#include <atomic>
#include <mutex>

#include "../../include/dia.h"
#include "dia_ops.cuh"
#include "dia_tc_ptx.cuh"

namespace dia {

namespace {

constexpr int kTcNO = 32;                  // output rows per tile (MMA N)
constexpr int kTcCols = 2 * kTcNO;         // tensor-memory columns: two accumulator buffers
constexpr int kTcW = 128;                  // output columns per tile (MMA M)
constexpr int kTcXT = kTcW + 32;           // R window columns (m <= 33)
constexpr int kTcYT = 64;                  // R window rows (NO + m - 1 <= 64)
constexpr int kTcYC = kTcYT / 8;           // 8-row chunks of the window
constexpr int kTcKC = 12;                  // 16-byte chunks of one Zk_b (>= (NO + YT) / 8 + 1)
constexpr int kTcMaxM = 31;
constexpr int kTcProducers = 128;          // warps 0-3
constexpr int kTcEpi = 128;                // warps 4-7
constexpr int kTcMmaWarp = 8;
constexpr int kTcThreads = kTcProducers + kTcEpi + 32;

struct TcSmem {
    float f[kTcYT][kTcXT];                        // next tile's R window (cp.async)
    __nv_bfloat16 t[2][2][kTcYC][kTcXT][8];       // [buffer][hi|lo][y / 8][x][y % 8]
    __nv_bfloat16 zk[2][kTcMaxM][kTcKC * 64];     // [hi|lo][b][c][t][e]
    uint64_t tfull[2];    // T buffer staged (128 producer arrivals)
    uint64_t tempty[2];   // T buffer read by its MMAs (tcgen05.commit)
    uint64_t afull[2];    // accumulators final (tcgen05.commit)
    uint64_t aempty[2];   // accumulators read back (128 epilogue arrivals)
    uint64_t wfull;       // the TMA window copy landed (1 arrival + 40960 bytes)
    uint64_t drain;       // every MMA issued has completed
    double red[4][5];     // loss mode: per epilogue warp loss, dL/dB0, count, curvature sums
    uint32_t tslot;
    int abort;            // set by any role whose wait ran out (every wait watches it)
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
    int *status;         // [0] 1 if a wait ran out, 2 if a bounds check failed; [1] its index
    int use_tma;         // 1: the window by TMA through `tmap`
    long long wait_cycles;   // limit of each pipeline wait (SM clock cycles)
    // loss mode (gmap != nullptr; diff_out unused): g = dl/dM into gmap (pitch
    // gld; 0 where masked and, inside the tiles, outside the valid region),
    // this CTA's partial row (loss, dL/dB0, pixel count, curvature sums at
    // their red_size(nk) slots, 0 elsewhere) and max |R|, max |g| into amax
    float *gmap;
    int gld;
    const uint8_t *mask;
    const float *var, *flat;
    LossParams lp;
    double *partials;
    int np, nk;
    unsigned *amax;
    // extents for the kernel's own bounds checks: elements addressable in
    // R / I / mask / var / flat, in the output (D or g map), partial rows
    size_t n_img, n_out;
    int rows;
    const int *done;     // nullable: nonzero -> return at once (a converged fit's graph)
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

// One tile's MMAs: for every kernel column b, NKS K steps x 3 split products
// into the accumulator at acc.  Descriptor starts advance by adds on the encoded
// address field (b: 16 bytes of the window, one Zk_b array; ks: two 8-row
// chunks of the window, two 128-byte Zk blocks), so the issue loop stays
// short: at N = 32 the instruction issue, not the tensor pipe, bounds it.
template <int NKS>
__device__ __forceinline__ void tc_issue_tile(uint32_t acc, uint64_t tbuf, uint64_t dz0,
                                              uint32_t idesc, int m) {
    // only the low word (encoded start address, LBO) changes; the start field
    // (address / 16 < 2^14 for shared memory) never carries into the LBO field
    constexpr uint32_t kTsplit = (uint32_t)(kTcYC * kTcXT * 8 * 2) >> 4;
    constexpr uint32_t kZsplit = (uint32_t)(kTcMaxM * kTcKC * 64 * 2) >> 4;
    constexpr uint32_t kZb = (uint32_t)(kTcKC * 64 * 2) >> 4;
    const uint32_t thi = (uint32_t)(tbuf >> 32), zhi = (uint32_t)(dz0 >> 32);
    const uint32_t tlo0 = (uint32_t)tbuf, zlo0 = (uint32_t)dz0;
    auto d64 = [](uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; };
    for (int b = 0; b < m; ++b) {
        const uint32_t tb = tlo0 + (uint32_t)b;          // 16 bytes per column
        const uint32_t zb = zlo0 + (uint32_t)b * kZb;
#pragma unroll
        for (int ks = 0; ks < NKS; ++ks) {
            const uint32_t ahi = tb + (uint32_t)((2 * ks * kTcXT * 16) >> 4), alo = ahi + kTsplit;
            const uint32_t bhi = zb + (uint32_t)((2 * ks * 128) >> 4), blo = bhi + kZsplit;
            if (ks == 0)
                tc_mma(acc, d64(ahi, thi), d64(bhi, zhi), idesc, b > 0 ? 1 : 0);
            else
                tc_mma_acc(acc, d64(ahi, thi), d64(bhi, zhi), idesc);
            tc_mma_acc(acc, d64(ahi, thi), d64(blo, zhi), idesc);
            tc_mma_acc(acc, d64(alo, thi), d64(bhi, zhi), idesc);
        }
    }
}

// 32 consecutive tensor-memory columns of this warp's 32 lanes into v
__device__ __forceinline__ void tc_ld32(uint32_t (&v)[32], uint32_t ta) {
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
}

__device__ __forceinline__ void tc_set_abort(TcSmem &S, int *status) {
    *reinterpret_cast<volatile int *>(&S.abort) = 1;
    atomicExch(status, 1);
}

// LK < 0: D = I - M; LK = 3 rho + var_model: loss mode for that loss, the
// per-pixel arithmetic without branches (masked and outside pixels select 0)
template <int LK>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_forward_kernel(const TcArgs a, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    if (a.done != nullptr && *reinterpret_cast<const volatile int *>(a.done) != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m, h = m / 2;
    const int nks = (kTcNO + m - 1 + 15) / 16;   // K steps of 16 window rows

    if (warp == kTcMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&S.tslot)), "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.tfull[i], kTcProducers);
            mbar_init(&S.tempty[i], 1);
            mbar_init(&S.afull[i], 1);
            mbar_init(&S.aempty[i], kTcEpi);
        }
        mbar_init(&S.wfull, 1);
        mbar_init(&S.drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        S.abort = 0;
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

    if (warp == kTcMmaWarp) {
        // ---- MMA issue (one lane) ----
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(kTcW, kTcNO);
            // A_b (ks): T + ((2 ks) XT + b) 16 bytes; B_b (ks): Zk_b + 2 ks 128 bytes
            const uint64_t dt0 = tc_desc(su32(&S.t[0][0][0][0][0]), kTcXT * 16, 128);
            const uint64_t dz0 = tc_desc(su32(&S.zk[0][0][0]), 128, 128);
            constexpr uint32_t kTbuf = sizeof(S.t[0]);
            static_assert(sizeof(S.t[0][0]) == kTcYC * kTcXT * 8 * 2 &&
                          sizeof(S.zk[0]) == kTcMaxM * kTcKC * 64 * 2 &&
                          sizeof(S.zk[0][0]) == kTcKC * 64 * 2, "tc_issue_tile strides");
            int k = 0;
            for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++k) {
                const int buf = k & 1;
                if (!tc_wait(&S.tfull[buf], (uint32_t)((k >> 1) & 1), &S.abort, a.wait_cycles) ||
                    (k >= 2 && !tc_wait(&S.aempty[buf], (uint32_t)(((k - 2) >> 1) & 1), &S.abort,
                                        a.wait_cycles))) {
                    tc_set_abort(S, a.status);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t acc0 = tmem + (uint32_t)(buf * kTcNO);
                const uint64_t tbuf = dt0 + ((buf * kTbuf) >> 4);
                if (nks == 2)
                    tc_issue_tile<2>(acc0, tbuf, dz0, idesc, m);
                else if (nks == 3)
                    tc_issue_tile<3>(acc0, tbuf, dz0, idesc, m);
                else
                    tc_issue_tile<4>(acc0, tbuf, dz0, idesc, m);
                tc_commit(&S.tempty[buf]);
                tc_commit(&S.afull[buf]);
            }
            // every MMA issued completes before the shared and tensor memory go
            tc_commit(&S.drain);
            const int never = 0;
            tc_wait(&S.drain, 0, &never);
        }
        __syncwarp();
    } else if (warp >= kTcProducers / 32) {
        // ---- epilogue: tensor memory lanes 32 (warp - 4) .. + 31 = output columns ----
        const int ew = warp - kTcProducers / 32;
        float gmax = 0.f;
        double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        bool ok = true;
        int k = 0;
        for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++k) {
            const int buf = k & 1;
            ok = tc_wait(&S.afull[buf], (uint32_t)((k >> 1) & 1), &S.abort, a.wait_cycles);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t v[kTcNO];
            tc_ld32(v, tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(buf * kTcNO));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&S.aempty[buf]);
            const int y0 = (tile / a.tiles_x) * kTcNO, x0 = (tile % a.tiles_x) * kTcW;
            const int x = x0 + 32 * ew + lane;
            const bool xin = x < a.Wv;
            // 8 rows at a time: every load of the group is issued before the
            // first is used (pixels outside the valid region read pixel 0)
            if constexpr (LK >= 0) {
                LossParams lq = a.lp;
                lq.rho = LK / 3;
                lq.var_model = LK % 3;
                float l = 0.f, gs = 0.f, cnt = 0.f, kr = 0.f, ks = 0.f;
#pragma unroll
                for (int c = 0; c < kTcNO / 8; ++c) {
                    float Iv[8], vm[8], Fv[8], rv[8];
                    uint32_t mk[8];
                    bool in[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int y = y0 + kTcNO - 1 - (8 * c + e);
                        in[e] = xin && y < a.Hv;
                        size_t off = in[e] ? (size_t)(y + h) * a.ld + (x + h) : 0;
                        if (off >= a.n_img) {
                            tc_report_bad(a.status, 2, off);
                            off = 0;
                        }
                        mk[e] = a.mask ? (uint32_t)a.mask[off] : 1u;
                        Iv[e] = __ldg(a.I + off);
                        vm[e] = a.var ? __ldg(a.var + off) : a.lp.var_scalar;
                        Fv[e] = a.flat ? __ldg(a.flat + off) : 1.0f;
                        rv[e] = __ldg(a.R + off);
                    }
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int ip = 8 * c + e;
                        const int y = y0 + kTcNO - 1 - ip;
                        const bool use = in[e] && mk[e] != 0;
                        float g, z, kap;
                        const float ell = pixel_loss(lq, Iv[e], __uint_as_float(v[ip]) + B0, vm[e],
                                                     Fv[e], g, z, kap);
                        const float gv = use ? g : 0.f;
                        l += use ? ell : 0.f;
                        gs += gv;
                        cnt += use ? 1.f : 0.f;
                        kr = fmaf(use ? kap * rv[e] : 0.f, rv[e], kr);
                        ks += use ? kap : 0.f;
                        gmax = fmaxf(gmax, fabsf(gv));
                        const size_t gi = (size_t)y * a.gld + x;
                        if (gi < a.n_out)
                            a.gmap[gi] = gv;
                        else
                            tc_report_bad(a.status, 2, gi);
                    }
                }
                acc[0] += l;
                acc[1] += gs;
                acc[2] += cnt;
                acc[3] += kr;
                acc[4] += ks;
            } else if (xin) {
#pragma unroll
                for (int c = 0; c < kTcNO / 8; ++c) {
                    float Iv[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int y = y0 + kTcNO - 1 - (8 * c + e);
                        const size_t off = (size_t)(y + h) * a.ld + (x + h);
                        Iv[e] = (y < a.Hv && off < a.n_img) ? __ldg(a.I + off) : 0.f;
                    }
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int ip = 8 * c + e;
                        const int y = y0 + kTcNO - 1 - ip;
                        const size_t di = (size_t)y * a.Wv + x;
                        if (y < a.Hv) {
                            if (di < a.n_out)
                                a.diff_out[di] = Iv[e] - (__uint_as_float(v[ip]) + B0);
                            else
                                tc_report_bad(a.status, 2, di);
                        }
                    }
                }
            }
        }
        if (!ok && lane == 0) tc_set_abort(S, a.status);
        if constexpr (LK >= 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                gmax = fmaxf(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
#pragma unroll
                for (int q = 0; q < 5; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            }
            if (lane == 0) {
                if (gmax > 0.f) atomicMax(a.amax + 1, __float_as_uint(gmax));
#pragma unroll
                for (int q = 0; q < 5; ++q) S.red[ew][q] = acc[q];
            }
        }
    } else {
        // ---- producers: the window of each tile, split into T[k & 1] ----
        const bool vec = ((a.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.R) & 15) == 0);
        const int ylim = kTcNO + m - 1;   // window rows with a nonzero kernel weight
        float rmax = 0.f;                 // loss mode: max |R| over the windows
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
        int k = 0;
        for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++k) {
            const int buf = k & 1;
            // the window has landed (TMA: the transaction count of wfull; cp.async:
            // each thread's own copies, then everyone's at the barrier)
            if (a.use_tma)
                fail = fail || !tc_wait(&S.wfull, (uint32_t)(k & 1), &S.abort, a.wait_cycles);
            else
                cp_async_wait<0>();
            if (k >= 2 && !fail)
                fail = !tc_wait(&S.tempty[buf], (uint32_t)(((k - 2) >> 1) & 1), &S.abort,
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
                for (int e = 0; e < 8; ++e) {
                    const float rv = S.f[8 * yc + e][x];
                    rmax = fmaxf(rmax, fabsf(rv));
                    split_bf16(rv, hi[e], lo[e]);
                }
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
        }
        cp_async_wait<0>();
        // after a failure, the last window requested must land (or its wait run
        // out) before the CTA's shared memory is released
        if (fail && a.use_tma && tid == 0 && tma_issued > 0) {
            const int never = 0;
            tc_wait(&S.wfull, (uint32_t)((tma_issued - 1) & 1), &never);
        }
        if (fail && lane == 0) tc_set_abort(S, a.status);
        if (a.gmap != nullptr) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            if (lane == 0 && rmax > 0.f) atomicMax(a.amax, __float_as_uint(rmax));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (a.gmap != nullptr && (int)blockIdx.x < a.rows) {
        double *out = a.partials + (size_t)blockIdx.x * a.np;
        const int c0 = red_count(a.nk);
        for (int k = tid; k < a.np; k += kTcThreads) {
            int q = -1;
            if (k == 0) q = 0;
            else if (k == a.nk + 1) q = 1;
            else if (k >= c0 && k < c0 + 3) q = 2 + (k - c0);
            double t = 0.0;
            if (q >= 0)
                for (int w = 0; w < 4; ++w) t += S.red[w][q];
            out[k] = t;
        }
    }
    if (warp == kTcMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
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

static cudaError_t tc_forward_launch(TcArgs &a, const float *R, int H, int W, int ld, int m,
                                     cudaStream_t s, int rows);

cudaError_t launch_tc_forward(const float *R, const float *I, int H, int W, int ld, int m,
                              const float *Kpad, int kp, float *diff_out, int *status,
                              cudaStream_t s, long long wait_cycles) {
    if (m < 1 || m > kTcMaxM || (m & 1) == 0) return cudaErrorInvalidValue;
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.I = I;
    a.Kpad = Kpad;
    a.kp = kp;
    a.diff_out = diff_out;
    a.status = status;
    a.wait_cycles = wait_cycles > 0 ? wait_cycles : kTcWaitCycles;
    a.n_out = (size_t)(H - 2 * (m / 2)) * (W - 2 * (m / 2));
    return tc_forward_launch(a, R, H, W, ld, m, s, 0);
}

cudaError_t launch_tc_forward_gmap(const EvalArgs &ea, int m, const float *Kpad, int kp,
                                   float *gmap, int gld, int gmap_rows, double *partials, int np,
                                   int rows, unsigned *amax, int *status, cudaStream_t s,
                                   long long wait_cycles, const int *done) {
    const int hv = ea.H - 2 * (m / 2);
    if (m < 1 || m > kTcMaxM || (m & 1) == 0 || !gmap || !partials || !amax || rows < 1 ||
        gld < ((ea.W - 2 * (m / 2) + kTcW - 1) / kTcW) * kTcW ||
        gmap_rows < (hv + kTcNO - 1) / kTcNO * kTcNO)
        return cudaErrorInvalidValue;
    TcArgs a;
    memset(&a, 0, sizeof(a));
    a.I = ea.I;
    a.Kpad = Kpad;
    a.kp = kp;
    a.status = status;
    a.wait_cycles = wait_cycles > 0 ? wait_cycles : kTcWaitCycles;
    a.gmap = gmap;
    a.gld = gld;
    a.mask = ea.mask;
    a.var = ea.var;
    a.flat = ea.flat;
    a.lp = ea.lp;
    a.partials = partials;
    a.np = np;
    a.nk = m * m;
    a.amax = amax;
    a.n_out = (size_t)gmap_rows * gld;
    a.done = done;
    return tc_forward_launch(a, ea.R, ea.H, ea.W, ea.ld, m, s, rows);
}

// the shared-memory attribute of tc_forward_kernel<lk>, set once per process
// (before any graph capture when tc_forward_prepare is called first)
static cudaError_t tc_forward_attr(int lk) {
    static std::atomic<int> done[10];
    std::atomic<int> &d = done[lk + 1];
    if (d.load()) return cudaSuccess;
    const int smem = tc_smem_bytes();
    cudaError_t e = cudaErrorInvalidValue;
    switch (lk) {
#define DIA_TC_ATTR(L)                                                                          \
    case L:                                                                                     \
        e = cudaFuncSetAttribute(tc_forward_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 smem);                                                         \
        break;
        DIA_TC_ATTR(-1)
        DIA_TC_ATTR(0)
        DIA_TC_ATTR(1)
        DIA_TC_ATTR(2)
        DIA_TC_ATTR(3)
        DIA_TC_ATTR(4)
        DIA_TC_ATTR(5)
        DIA_TC_ATTR(6)
        DIA_TC_ATTR(7)
        DIA_TC_ATTR(8)
#undef DIA_TC_ATTR
        default: break;
    }
    if (e == cudaSuccess) d.store(1);
    return e;
}

cudaError_t tc_forward_prepare(int rho, int var_model) {
    if (rho < 0 || rho > 2 || var_model < 0 || var_model > 2) return cudaErrorInvalidValue;
    cudaError_t e = tc_forward_attr(-1);
    return e == cudaSuccess ? tc_forward_attr(3 * rho + var_model) : e;
}

// the launch itself: tensor map, tiling, grid (rows > 0: the loss mode's
// partial rows, those past the grid cleared)
static cudaError_t tc_forward_launch(TcArgs &a, const float *R, int H, int W, int ld, int m,
                                     cudaStream_t s, int rows) {
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
    a.R = R;
    a.H = H;
    a.W = W;
    a.ld = ld;
    a.m = m;
    a.Hv = H - 2 * (m / 2);
    a.Wv = W - 2 * (m / 2);
    a.tiles_x = (a.Wv + kTcW - 1) / kTcW;
    a.n_tiles = a.tiles_x * ((a.Hv + kTcNO - 1) / kTcNO);
    a.use_tma = use_tma;
    a.n_img = (size_t)(H - 1) * ld + W;
    int dev = 0, sms = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int smem = tc_smem_bytes();
    const int cap = rows > 0 ? (rows < sms ? rows : sms) : sms;
    const int grid = a.n_tiles < cap ? a.n_tiles : cap;
    a.rows = rows;
    int lk = -1;
    if (a.gmap) {
        if (a.lp.rho < 0 || a.lp.rho > 2 || a.lp.var_model < 0 || a.lp.var_model > 2)
            return cudaErrorInvalidValue;
        lk = 3 * a.lp.rho + a.lp.var_model;
    }
    switch (lk) {
#define DIA_TC_CASE(L)                                                                          \
    case L:                                                                                     \
        e = tc_forward_attr(L);                                                                 \
        if (e == cudaSuccess) tc_forward_kernel<L><<<grid, kTcThreads, smem, s>>>(a, tmap);    \
        break;
        DIA_TC_CASE(-1)
        DIA_TC_CASE(0)
        DIA_TC_CASE(1)
        DIA_TC_CASE(2)
        DIA_TC_CASE(3)
        DIA_TC_CASE(4)
        DIA_TC_CASE(5)
        DIA_TC_CASE(6)
        DIA_TC_CASE(7)
        DIA_TC_CASE(8)
#undef DIA_TC_CASE
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e == cudaSuccess && rows > grid)
        e = cudaMemsetAsync(a.partials + (size_t)grid * a.np, 0, (size_t)(rows - grid) * a.np * 8, s);
    return e;
}

}  // namespace dia

// Fused DIA evaluation kernel: forward convolution, per-pixel loss and the
// kernel/background gradient in one pass over the image (sm_103a).
//
// Model (Sec. 2.1, Eq. 2): for an output pixel p = (y, x) of the valid region,
//   M_p = sum_{a,b} K[a][b] R[y+a][x+b] + B0        (valid-region coordinates)
// Loss (Sec. 2.3 Eq. 7, Sec. 2.4 Eq. 10-11): l_p = rho(z_p) + ln sigma_p with
// z = (I - M)/sigma and sigma^2 from the fixed map or the CCD / EMCCD models
// (Eq. 5, Eq. 6).  Gradient: dL/dK[a][b] = sum_p g_p R[y+a][x+b],
// dL/dB0 = sum_p g_p with g_p = dl_p/dM_p.
//
// One CTA owns a TH x TW tile of output pixels at a time (persistent loop over
// tiles).  Per tile:
//   1. the R tile plus its (m-1) halo is staged in shared memory with
//      cp.async, double-buffered so the next tile's copy overlaps compute;
//   2. forward: warp w computes rows [w*QF, (w+1)*QF) of the tile, lane l the
//      four columns [4l, 4l+4); each R row is loaded once into a register
//      window and reused by all QF output rows and all m kernel columns;
//      K is read from shared memory as warp-uniform (broadcast) float4 loads;
//   3. epilogue: M stays in registers, the loss terms and g_p are formed in
//      float32 and g_p is written to a shared-memory tile (never to HBM);
//   4. backward: with m = NW*KF + RM, warp w owns kernel rows [w*KF, (w+1)*KF)
//      over the whole tile plus the RM last rows on its own QF-row slice
//      (equal work per warp); lanes split the columns; each R row window is
//      reused by every kernel row it feeds, the m column offsets and the
//      four pixels of the lane;
//   5. per-lane float32 sums (at most 4096 pixels each) are reduced over the
//      warp and added in float64 to per-CTA shared accumulators.
// At the end each CTA writes m*m + 5 float64 partials (loss, dK, dB0, pixel
// count, and two curvature sums for the optimiser's diagonal preconditioner);
// a separate kernel sums them in a fixed order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dia {

constexpr int kTW = 128;  // tile width: 32 lanes x 4 pixels

enum EvalMode { kModeGrad = 0, kModeForward = 1 };

struct LossParams {
    int rho;          // 0 gauss, 1 huber, 2 cauchy
    int var_model;    // 0 fixed, 1 ccd, 2 emccd
    float s0sq;       // sigma0^2
    float inv_gain;   // 1/G
    float excess;     // E
    float huber_c;
    float var_scalar;
    float var_floor;
};

struct EvalArgs {
    const float *R;
    const float *I;
    const uint8_t *mask;   // nullable
    const float *var;      // nullable
    const float *flat;     // nullable
    int H, W, ld;
    int Hv, Wv;            // valid region
    int tiles_x, n_tiles;
    const float *Kpad;     // m rows of KP floats (zero padded), then B0
    double *partials;      // [gridDim.x][m*m + 5]
    float *diff_out;       // forward mode: D = I - M over the valid region (nullable)
    uint8_t *mask_out;     // forward mode: clip |z| > kappa (nullable)
    float clip_kappa;
    const int *done_flag;  // nullable: nonzero -> return at once
    LossParams lp;
};

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }

// Pixel loss and g = dl/dM (float32).  Returns the loss; writes g, z and a
// non-negative curvature weight kappa ~ d2l/dM2 (Gauss-Newton / IRLS weight
// rho'(z)/z / v, plus the Fisher term (v'/v)^2 / 2 of a model-dependent
// variance) used only to precondition the optimiser.
__device__ __forceinline__ float pixel_loss(const LossParams &lp, float I, float M, float vmap,
                                            float F, float &g, float &z, float &kappa) {
    float v, dv;
    if (lp.var_model == 0) {
        v = vmap;
        dv = 0.f;
    } else {
        const float invGF = lp.inv_gain / F;
        if (lp.var_model == 1) {
            v = lp.s0sq / (F * F) + M * invGF;
            dv = invGF;
        } else {
            v = lp.excess * M * invGF;
            dv = lp.excess * invGF;
        }
        if (v < lp.var_floor) {
            v = lp.var_floor;
            dv = 0.f;
        }
    }
    const float inv_v = 1.0f / v;
    const float inv_s = sqrtf(inv_v);
    const float r = I - M;
    z = r * inv_s;
    // dz/dM = -1/s - z v'/(2v)
    const float dz = -inv_s - 0.5f * z * dv * inv_v;
    float rho, rho1, wz;  // wz = rho'(z)/z
    if (lp.rho == 0) {
        rho = 0.5f * z * z;
        rho1 = z;
        wz = 1.f;
    } else if (lp.rho == 1) {
        const float c = lp.huber_c, az = fabsf(z);
        if (az <= c) {
            rho = 0.5f * z * z;
            rho1 = z;
            wz = 1.f;
        } else {
            rho = c * (az - 0.5f * c);
            rho1 = copysignf(c, z);
            wz = c / az;
        }
    } else {
        const float q = z * z;
        rho = log1pf(q);
        wz = 2.0f / (1.0f + q);
        rho1 = z * wz;
    }
    float ell = rho;
    g = rho1 * dz;
    kappa = wz * inv_v;
    if (lp.var_model != 0) {
        ell += 0.5f * logf(v);
        g += 0.5f * dv * inv_v;
        kappa += 0.5f * (dv * inv_v) * (dv * inv_v);
    }
    return ell;
}

// Asynchronous global -> shared copies (cp.async); a source size below the
// copy size fills the rest with zeros.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Stage the R tile (rows ty0.., columns tx0.., RROWS x RP) into dst; zeros
// outside the image.  16-byte copies when rows are 16-byte aligned.
template <int RROWS, int RP, int NT>
__device__ __forceinline__ void stage_tile(float *dst, const EvalArgs &a, int ty0, int tx0,
                                           bool vec) {
    if (vec) {
        constexpr int CH = RP / 4;
        for (int i = threadIdx.x; i < RROWS * CH; i += NT) {
            const int r = i / CH, c4 = i - r * CH;
            const int gy = ty0 + r, gx = tx0 + 4 * c4;
            int bytes = 0;
            const float *src = a.R;
            if (gy < a.H && gx < a.W) {
                bytes = (a.W - gx >= 4) ? 16 : 4 * (a.W - gx);
                src = a.R + (size_t)gy * a.ld + gx;
            }
            cp_async16(dst + r * RP + 4 * c4, src, bytes);
        }
    } else {
        for (int i = threadIdx.x; i < RROWS * RP; i += NT) {
            const int r = i / RP, c = i - r * RP;
            const int gy = ty0 + r, gx = tx0 + c;
            const bool in = gy < a.H && gx < a.W;
            cp_async4(dst + i, in ? a.R + (size_t)gy * a.ld + gx : a.R, in ? 4 : 0);
        }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// SPLIT selects how the backward's kernel rows are shared among the warps:
// 0 = whole rows, ceil(MK/NW) or floor(MK/NW) per warp; 1 = MK = NW*KF + RM
// with KF whole rows per warp and the RM last rows split by tile-row slices.
template <int MK, int NW, int QF, int SPLIT>
struct EvalShape {
    static constexpr int TH = NW * QF;
    static constexpr int RROWS = TH + MK - 1;
    static constexpr int RP = round4(kTW + MK - 1);      // R tile pitch (floats)
    static constexpr int RWIN = round4(MK + 3);          // register window per lane
    static constexpr int KP = round4(MK);                // K row pitch (floats)
    // backward split: MK = NW*KF + RM; warp w owns kernel rows [w*KF, (w+1)*KF)
    // over the whole tile and the RM last rows on its own QF-row slice, so
    // every warp does the same work
    static constexpr int KF = SPLIT ? MK / NW : (MK + NW - 1) / NW;
    static constexpr int RM = SPLIT ? MK % NW : 0;
    static constexpr int QB = KF + RM;                   // dK rows held per lane
    static constexpr int NP = MK * MK + 5;               // partials per CTA
    static constexpr int NT = NW * 32;
    // shared memory layout (bytes)
    static constexpr int OFF_R = 0;
    static constexpr int SZ_R = RROWS * RP * 4;          // one R tile buffer (two are kept)
    static constexpr int GPAD = KF > 2 ? KF - 1 : 1;     // zero rows above and below the g tile
    static constexpr int OFF_G = OFF_R + 2 * SZ_R;
    // tiles between float64 flushes: each lane's float32 sums then cover at
    // most 4096 pixels
    static constexpr int FLUSH = (4096 / (4 * TH)) > 0 ? (4096 / (4 * TH)) : 1;
    static constexpr int SZ_G = (TH + 2 * GPAD) * kTW * 4;
    static constexpr int OFF_K = OFF_G + SZ_G;
    static constexpr int SZ_K = (MK * KP + 4) * 4;
    static constexpr int OFF_D = (OFF_K + SZ_K + 15) & ~15;
    // float64: dK rows with one owner, per-warp copies of the RM shared rows,
    // per-warp {loss, dB0, count, kR^2, k}
    static constexpr int OFF_D_RM = MK * MK;
    static constexpr int OFF_D_W5 = OFF_D_RM + NW * RM * MK;
    static constexpr int SZ_D = (OFF_D_W5 + 5 * NW) * 8;
    static constexpr int SMEM = OFF_D + SZ_D;
};

// Backward rows: dk[OFF+qb][b] += sum_rr sum_p g[y][x+p] R[r0+rr][x+b+p] with
// y = y0 + rr - qb, for NQ kernel rows.  Whole-tile rows (SLICE = false)
// rely on the zero rows around the g tile; slice rows (SLICE = true) keep
// y inside [y0, y0 + NS) and read a zero row otherwise.  Each R row window is
// loaded once and used by all NQ kernel rows, m column offsets and 4 pixels.
template <int MK, int QB, int OFF, int NQ, int RP, int RWIN, bool SLICE, int NS>
__device__ __forceinline__ void bwd_rows(const float *rrow, const float *g0, const float *gzero,
                                         int n_rr, float (&dk)[QB][MK]) {
#pragma unroll 1
    for (int rr = 0; rr < n_rr; ++rr) {
        float win[RWIN];
        const float4 *rp4 = reinterpret_cast<const float4 *>(rrow + rr * RP);
#pragma unroll
        for (int v4 = 0; v4 < RWIN / 4; ++v4) {
            const float4 t = rp4[v4];
            win[4 * v4 + 0] = t.x;
            win[4 * v4 + 1] = t.y;
            win[4 * v4 + 2] = t.z;
            win[4 * v4 + 3] = t.w;
        }
        float4 g4[NQ];
#pragma unroll
        for (int qb = 0; qb < NQ; ++qb) {
            const float *gp = g0 + (rr - qb) * kTW;
            if (SLICE && (rr - qb < 0 || rr - qb >= NS)) gp = gzero;
            g4[qb] = *reinterpret_cast<const float4 *>(gp);
        }
        // pixel p outer: consecutive FMAs update different accumulators
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
            for (int qb = 0; qb < NQ; ++qb) {
                const float gv = p == 0 ? g4[qb].x : p == 1 ? g4[qb].y : p == 2 ? g4[qb].z : g4[qb].w;
#pragma unroll
                for (int b = 0; b < MK; ++b) dk[OFF + qb][b] = fmaf(gv, win[b + p], dk[OFF + qb][b]);
            }
        }
    }
}

template <int MK, int NW, int QF, int MINB, int SPLIT, int MODE>
__global__ void __launch_bounds__(NW * 32, MINB) eval_kernel(const EvalArgs args) {
    using S = EvalShape<MK, NW, QF, SPLIT>;
    constexpr int TH = S::TH, RP = S::RP, RWIN = S::RWIN, KP = S::KP, QB = S::QB;
    constexpr int H2 = MK / 2;
    if (args.done_flag != nullptr && *((volatile const int *)args.done_flag) != 0) return;

    extern __shared__ __align__(16) unsigned char smem[];
    float *Rbuf0 = reinterpret_cast<float *>(smem + S::OFF_R);
    float *Rbuf1 = Rbuf0 + S::RROWS * RP;
    float *gs = reinterpret_cast<float *>(smem + S::OFF_G);
    float *Ks = reinterpret_cast<float *>(smem + S::OFF_K);
    double *acc64 = reinterpret_cast<double *>(smem + S::OFF_D);  // dK[MK*MK], then per warp
                                                                  // {loss, dB0, count, kR2, k}

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < MK * KP + 4; i += S::NT) Ks[i] = args.Kpad[i];
    if (MODE == kModeGrad) {
        for (int i = tid; i < S::OFF_D_W5 + 5 * NW; i += S::NT) acc64[i] = 0.0;
        for (int i = tid; i < S::GPAD * kTW; i += S::NT) {
            gs[i] = 0.f;
            gs[(S::GPAD + TH) * kTW + i] = 0.f;
        }
    }
    float *gt = gs + S::GPAD * kTW;   // g tile row 0
    __syncthreads();
    const float B0 = Ks[MK * KP];

    constexpr int KF = S::KF, RM = S::RM;
    // whole-tile kernel rows of this warp: [a_lo, a_lo + nq)
    const int a_lo = SPLIT ? warp * KF : (warp * MK) / NW;
    const int nq = SPLIT ? KF : ((warp + 1) * MK) / NW - a_lo;

    // per-lane float32 sums, flushed to the float64 CTA accumulators every
    // FLUSH tiles: dK rows owned by this warp, and loss / dB0 / count /
    // curvature sums of the lane's pixels
    float dk[QB][MK];
#pragma unroll
    for (int qb = 0; qb < QB; ++qb)
#pragma unroll
        for (int b = 0; b < MK; ++b) dk[qb][b] = 0.f;
    float lsum = 0.f, gsum = 0.f, cnt = 0.f, ksum = 0.f, kr2sum = 0.f;
    int since_flush = 0;
    auto flush = [&]() {
#pragma unroll
        for (int qb = 0; qb < QB; ++qb) {
            if (qb < KF && qb >= nq) continue;
            double *dst = (qb < KF) ? acc64 + (a_lo + qb) * MK
                                    : acc64 + S::OFF_D_RM + (warp * RM + (qb - KF)) * MK;
#pragma unroll
            for (int b = 0; b < MK; ++b) {
                const float sm = warp_sum(dk[qb][b]);
                if (lane == 0) dst[b] += (double)sm;
                dk[qb][b] = 0.f;
            }
        }
        const float l = warp_sum(lsum), g = warp_sum(gsum), c = warp_sum(cnt);
        const float k = warp_sum(ksum), kr = warp_sum(kr2sum);
        if (lane == 0) {
            double *w5 = acc64 + S::OFF_D_W5 + 5 * warp;
            w5[0] += (double)l;
            w5[1] += (double)g;
            w5[2] += (double)c;
            w5[3] += (double)kr;
            w5[4] += (double)k;
        }
        lsum = gsum = cnt = ksum = kr2sum = 0.f;
    };

    // ---- 1. R tiles (+ halo) are staged with cp.async, the next tile's copy
    // overlapping the current tile's compute (two buffers)
    const bool vec = ((args.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(args.R) & 15) == 0);
    if (blockIdx.x < args.n_tiles)
        stage_tile<S::RROWS, RP, S::NT>(Rbuf0, args, (blockIdx.x / args.tiles_x) * TH,
                                        (blockIdx.x % args.tiles_x) * kTW, vec);
    cp_async_commit();
    int buf = 0;
    for (int tile = blockIdx.x; tile < args.n_tiles; tile += gridDim.x, buf ^= 1) {
        const int ty0 = (tile / args.tiles_x) * TH;
        const int tx0 = (tile % args.tiles_x) * kTW;
        const int nxt = tile + gridDim.x;
        if (nxt < args.n_tiles)
            stage_tile<S::RROWS, RP, S::NT>(buf ? Rbuf0 : Rbuf1, args, (nxt / args.tiles_x) * TH,
                                            (nxt % args.tiles_x) * kTW, vec);
        cp_async_commit();
        cp_async_wait<1>();   // this tile's copies have landed
        __syncthreads();
        const float *Rs = buf ? Rbuf1 : Rbuf0;

        // ---- 2. forward: acc[q][p] = sum_{a,b} K[a][b] R[y0+q+a][x+p+b]
        float acc[QF][4];
#pragma unroll
        for (int q = 0; q < QF; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[q][p] = 0.f;

        const float *rbase = Rs + (warp * QF) * RP + 4 * lane;
        const float4 *K4 = reinterpret_cast<const float4 *>(Ks);
        // R rows r with every output row q of the warp active (kernel row a = r - q
        // in [0, MK)): no branch, all QF x 4 accumulators interleaved per K column
#pragma unroll 1
        for (int r = QF - 1; r <= MK - 1; ++r) {
            float win[RWIN];
            const float4 *rp4 = reinterpret_cast<const float4 *>(rbase + r * RP);
#pragma unroll
            for (int v4 = 0; v4 < RWIN / 4; ++v4) {
                const float4 t = rp4[v4];
                win[4 * v4 + 0] = t.x;
                win[4 * v4 + 1] = t.y;
                win[4 * v4 + 2] = t.z;
                win[4 * v4 + 3] = t.w;
            }
            // K columns in groups of 4 (warp-uniform broadcast loads)
#pragma unroll
            for (int b4 = 0; b4 < KP / 4; ++b4) {
                float4 kq[QF];
#pragma unroll
                for (int q = 0; q < QF; ++q) kq[q] = K4[(r - q) * (KP / 4) + b4];
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const int b = 4 * b4 + bb;
                    if (b < MK) {
#pragma unroll
                        for (int q = 0; q < QF; ++q) {
                            const float kv = bb == 0 ? kq[q].x : bb == 1 ? kq[q].y : bb == 2 ? kq[q].z : kq[q].w;
#pragma unroll
                            for (int p = 0; p < 4; ++p) acc[q][p] = fmaf(kv, win[p + b], acc[q][p]);
                        }
                    }
                }
            }
        }
        // the first and last QF-1 R rows feed only some output rows (with
        // MK < QF - 1 there is no interior and every row is done here once)
        constexpr bool kSplit = MK >= QF - 1;
        constexpr int kEdges = kSplit ? 2 * (QF - 1) : (QF + MK - 1);
#pragma unroll 1
        for (int e = 0; e < kEdges; ++e) {
            const int r = kSplit ? ((e < QF - 1) ? e : (MK + e - (QF - 1))) : e;
            float win[RWIN];
            const float4 *rp4 = reinterpret_cast<const float4 *>(rbase + r * RP);
#pragma unroll
            for (int v4 = 0; v4 < RWIN / 4; ++v4) {
                const float4 t = rp4[v4];
                win[4 * v4 + 0] = t.x;
                win[4 * v4 + 1] = t.y;
                win[4 * v4 + 2] = t.z;
                win[4 * v4 + 3] = t.w;
            }
#pragma unroll
            for (int q = 0; q < QF; ++q) {
                const int a = r - q;
                if (a >= 0 && a < MK) {
#pragma unroll
                    for (int b4 = 0; b4 < KP / 4; ++b4) {
                        const float4 kk = K4[a * (KP / 4) + b4];
                        const float kv[4] = {kk.x, kk.y, kk.z, kk.w};
#pragma unroll
                        for (int bb = 0; bb < 4; ++bb) {
                            const int b = 4 * b4 + bb;
                            if (b < MK) {
#pragma unroll
                                for (int p = 0; p < 4; ++p) acc[q][p] = fmaf(kv[bb], win[p + b], acc[q][p]);
                            }
                        }
                    }
                }
            }
        }

        // ---- 3. epilogue: loss terms, g -> shared tile
#pragma unroll
        for (int q = 0; q < QF; ++q) {
            const int yl = warp * QF + q;
            const int y = ty0 + yl;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int xl = 4 * lane + p;
                const int x = tx0 + xl;
                float gval = 0.f;
                if (y < args.Hv && x < args.Wv) {
                    const size_t off = (size_t)(y + H2) * args.ld + (x + H2);
                    const bool use = (args.mask == nullptr) || (args.mask[off] != 0);
                    const float M = acc[q][p] + B0;
                    const float Iv = __ldg(args.I + off);
                    const float vm = args.var ? __ldg(args.var + off) : args.lp.var_scalar;
                    const float F = args.flat ? __ldg(args.flat + off) : 1.0f;
                    float g, z, kap;
                    const float ell = pixel_loss(args.lp, Iv, M, vm, F, g, z, kap);
                    if (MODE == kModeGrad) {
                        if (use) {
                            const float rc = Rs[(yl + H2) * RP + xl + H2];
                            lsum += ell;
                            gsum += g;
                            cnt += 1.f;
                            ksum += kap;
                            kr2sum = fmaf(kap * rc, rc, kr2sum);
                            gval = g;
                        }
                    } else {
                        if (args.diff_out) args.diff_out[(size_t)y * args.Wv + x] = Iv - M;
                        if (args.mask_out && use && fabsf(z) > args.clip_kappa) args.mask_out[off] = 0;
                    }
                }
                if (MODE == kModeGrad) gt[yl * kTW + xl] = gval;
            }
        }
        if (MODE != kModeGrad) {
            __syncthreads();  // the R buffer is refilled two tiles later
            continue;
        }
        __syncthreads();  // g tile complete

        // ---- 4. backward: dK[a][b] += sum_{y,x} g[y][x] R[y+a][x+b], a in [a_lo, a_lo+nqb)
        const float *gzero = gs + 4 * lane;   // a zero row above the g tile
        if (KF > 0 && nq == KF)
            bwd_rows<MK, QB, 0, (KF > 0 ? KF : 1), RP, RWIN, false, TH>(
                Rs + a_lo * RP + 4 * lane, gt + 4 * lane, gzero, TH + KF - 1, dk);
        else if (KF > 1 && nq == KF - 1)   // SPLIT 0: the warps with one row fewer
            bwd_rows<MK, QB, 0, (KF > 1 ? KF - 1 : 1), RP, RWIN, false, TH>(
                Rs + a_lo * RP + 4 * lane, gt + 4 * lane, gzero, TH + KF - 2, dk);
        if (RM > 0) {
            const int ys = warp * QF;          // this warp's slice of the tile rows
            bwd_rows<MK, QB, KF, (RM > 0 ? RM : 1), RP, RWIN, true, QF>(
                Rs + (NW * KF + ys) * RP + 4 * lane, gt + ys * kTW + 4 * lane, gzero,
                QF + RM - 1, dk);
        }
        // ---- 5. float32 sums -> float64 every FLUSH tiles (each kernel row
        // is owned by one warp, so the warps write disjoint accumulators)
        if (++since_flush == S::FLUSH) {
            flush();
            since_flush = 0;
        }
        __syncthreads();  // R buffer and g tile are reused
    }
    cp_async_wait<0>();

    if (MODE == kModeGrad) {
        if (since_flush > 0) flush();
        __syncthreads();
        double *out = args.partials + (size_t)blockIdx.x * S::NP;
        for (int i = tid; i < (MK - RM) * MK; i += S::NT) out[1 + i] = acc64[i];
        for (int i = tid; i < RM * MK; i += S::NT) {   // shared rows: per-warp copies, fixed order
            double t = 0.0;
            for (int w = 0; w < NW; ++w) t += acc64[S::OFF_D_RM + w * RM * MK + i];
            out[1 + (MK - RM) * MK + i] = t;
        }
        if (tid < 5) {
            // tid 0: loss, 1: dB0, 2: pixel count, 3: sum kappa R^2, 4: sum kappa
            double t = 0.0;
            for (int w = 0; w < NW; ++w) t += acc64[S::OFF_D_W5 + 5 * w + tid];
            out[tid == 0 ? 0 : MK * MK + tid] = t;
        }
    }
}

}  // namespace dia

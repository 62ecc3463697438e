// Fused DIA evaluation kernel: forward convolution, per-pixel loss and the
// kernel/background gradient in one pass over the image (sm_103a).
//
// Model (Sec. 2.1, Eq. 2): for an output pixel p = (y, x) of the valid region,
//   M_p = sum_{a,b} K[a][b] R[y+a][x+b] + B_p       (valid-region coordinates)
// with B_p = B0, or the polynomial of Sec. 2.6 (Eq. 18) in the normalised
// coordinates of Eq. 19 (eta along x, xi along y):
//   B_p = sum_{i<=d} c_i(xi) eta^i,  c_i(xi) = sum_{j<=d-i} b_ij xi^j.
// Loss (Sec. 2.3 Eq. 8, Sec. 2.4 Eq. 12-13): l_p = rho(z_p) + ln sigma_p with
// z = (I - M)/sigma and sigma^2 from the fixed map or the CCD / EMCCD models
// (Eq. 6, Eq. 7).  Gradient: dL/dK[a][b] = sum_p g_p R[y+a][x+b],
// dL/db_ij = sum_p g_p eta_p^i xi_p^j with g_p = dl_p/dM_p (dL/dB0 = sum_p g_p).
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
//      float32 (a fixed scalar variance with 1/v and sqrt(1/v) formed once per
//      thread) and g_p is written to a shared-memory tile (never to HBM);
//   4. backward (SPLIT 0, 1): with m = NW*KF + RM, warp w owns kernel rows
//      [w*KF, (w+1)*KF) over the whole tile plus the RM last rows on its own
//      QF-row slice (equal work per warp); lanes split the columns; each R row
//      window is reused by every kernel row it feeds, the m column offsets and
//      the four pixels of the lane.  SPLIT 2 (own rows): each warp takes every
//      kernel row over its own QF output rows, g still in registers, in passes
//      of about 64 accumulators per lane;
//   5. dK: per-lane float32 sums over one tile, reduced over the warp by a
//      halving butterfly and added to per-warp Kahan-compensated float32
//      shared accumulators; loss sums: per-lane float32 over <= 4096 pixels,
//      then float64.  Everything is combined in float64 at the end.
// At the end each CTA writes m*m + kBgMax + 4 float64 partials (loss, dK, the
// kBgMax background slots, pixel count, and two curvature sums for the
// optimiser's diagonal preconditioner); a separate kernel sums them in a fixed
// order.  With a polynomial background the moments sum_p g eta^i xi^j of a
// tile are taken from the shared g tile after the epilogue (float32 over one
// tile and warp, then float64).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace dia {

constexpr int kTW = 128;  // tile width: 32 lanes x 4 pixels

// Polynomial background (Eq. 18): degree <= kBgMaxDeg, kBgMax coefficient
// slots b_00, b_01, ..., b_0d, b_10, ... (power of xi fastest) after K.
constexpr int kBgMaxDeg = 4;
constexpr int kBgMax = (kBgMaxDeg + 1) * (kBgMaxDeg + 2) / 2;
__host__ __device__ constexpr int n_background(int deg) { return (deg + 1) * (deg + 2) / 2; }
// degree whose coefficient count is nb (nb = n_background(d) for some d <= kBgMaxDeg)
__host__ __device__ inline int bg_degree_of(int nb) {
    int d = 0;
    while (d < kBgMaxDeg && n_background(d) < nb) ++d;
    return d;
}
// layout of the reduced vector / per-CTA partials: [0] loss, [1, nk] dK,
// [nk+1, nk+kBgMax] background coefficients, then pixel count, sum kappa R^2,
// sum kappa
__host__ __device__ constexpr int red_count(int nk) { return nk + kBgMax + 1; }
__host__ __device__ constexpr int red_size(int nk) { return nk + kBgMax + 4; }
// float64 per-warp accumulators: loss, dB0, count, kR^2, k, then the moments of
// the background coefficients 1 .. kBgMax-1
constexpr int kAccW = 5 + kBgMax - 1;

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
    const float *Kpad;     // m rows of KP floats (zero padded), then kBgMax + 1
                           // background slots (b_00 first)
    double *partials;      // [gridDim.x][red_size(m*m)]
    float *diff_out;       // forward mode: D = I - M over the valid region (nullable)
    uint8_t *mask_out;     // forward mode: clip |z| > kappa (nullable)
    float clip_kappa;
    const int *done_flag;  // nullable: nonzero -> return at once
    LossParams lp;
    int acc32;             // nonzero: float32 accumulation everywhere, no compensation
                           // (the comparison form of the precision study)
    int bg_deg;            // background degree (0: constant B0)
    float eta0, eta_s;     // eta = eta0 + eta_s * x for valid-region column x (Eq. 19)
    float xi0, xi_s;       // xi = xi0 + xi_s * y for valid-region row y
};

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }

// Background of degree deg for an H x W image with kernel half-width h: the
// Eq. 19 coordinates of valid-region pixel (y, x), i.e. full-image pixel
// (y + h, x + h): eta = (x + h - (W-1)/2) / W, xi = (y + h - (H-1)/2) / H.
inline void set_background(EvalArgs &a, int deg, int H, int W, int h) {
    a.bg_deg = deg;
    a.eta_s = (float)(1.0 / W);
    a.eta0 = (float)((h - 0.5 * (W - 1)) / W);
    a.xi_s = (float)(1.0 / H);
    a.xi0 = (float)((h - 0.5 * (H - 1)) / H);
}

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

// The pixel loss of a fixed scalar variance (var_model 0, no variance map)
// with inv_v = 1/v and inv_s = sqrt(1/v) formed once per thread by the same
// correctly rounded operations: for finite inputs it returns exactly what
// pixel_loss does (there dv = 0, so dz reduces to -inv_s).
__device__ __forceinline__ float pixel_loss_fixed(const LossParams &lp, float inv_v, float inv_s,
                                                  float I, float M, float &g, float &z,
                                                  float &kappa) {
    const float r = I - M;
    z = r * inv_s;
    const float dz = -inv_s;
    float rho, rho1, wz;
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
    g = rho1 * dz;
    kappa = wz * inv_v;
    return rho;
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

template <int RWIN>
__device__ __forceinline__ void load_win(float (&win)[RWIN], const float *row) {
    const float4 *rp4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int v4 = 0; v4 < RWIN / 4; ++v4) {
        const float4 t = rp4[v4];
        win[4 * v4 + 0] = t.x;
        win[4 * v4 + 1] = t.y;
        win[4 * v4 + 2] = t.z;
        win[4 * v4 + 3] = t.w;
    }
}

// Warp reduction of N per-lane values by halving: at each of the five
// butterfly stages a lane keeps one half of its values (chosen by its lane
// bit), adds the partner's copy of that half, and sends the other half.
// Afterwards lane L holds the warp sums of NF = ceil(N/32) entries, entry j
// being value index base(L) + j; halving_index() gives that index (or -1 for
// a padding slot).  75 values cost 75 shuffles instead of 375.
template <int N>
struct Halving {
    static constexpr int H1 = (N + 1) / 2, H2 = (H1 + 1) / 2, H3 = (H2 + 1) / 2, H4 = (H3 + 1) / 2,
                         H5 = (H4 + 1) / 2;
};

template <int N, int O>
__device__ __forceinline__ void halve(const float *v, float *w, bool up) {
    constexpr int H = (N + 1) / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float lo = v[i];
        const float hi = (i + H < N) ? v[i + H] : 0.f;
        const float keep = up ? hi : lo;
        const float send = up ? lo : hi;
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

template <int N>
__device__ __forceinline__ int halving_index(int lane, int j) {
    using Hv = Halving<N>;
    const int hs[5] = {Hv::H1, Hv::H2, Hv::H3, Hv::H4, Hv::H5};
    const int ns[5] = {N, Hv::H1, Hv::H2, Hv::H3, Hv::H4};   // sizes before each stage
    int p = j;
    for (int st = 4; st >= 0; --st) {
        if (lane & (16 >> st)) p += hs[st];
        if (p >= ns[st]) return -1;
    }
    return p;
}

// Kernel rows per pass of the own-rows backward (SPLIT = 2): about 64 float32
// dK accumulators per lane, MK rows split into ceil(MK*MK/64) nearly equal passes.
__host__ __device__ constexpr int own_rows_per_pass(int mk) {
    return (mk + (mk * mk + 63) / 64 - 1) / ((mk * mk + 63) / 64);
}

// SPLIT selects how the backward's kernel rows are shared among the warps:
// 0 = whole rows, ceil(MK/NW) or floor(MK/NW) per warp; 1 = MK = NW*KF + RM
// with KF whole rows per warp and the RM last rows split by tile-row slices;
// 2 = own rows: each warp takes every kernel row over the QF output rows of
// its forward pass, with g still in registers, in passes of NQ kernel rows
// (each R row window then serves up to QF*NQ*MK*4 FMAs; the price is one warp
// reduction of MK*MK values per tile).
template <int MK, int NW, int QF, int SPLIT, int F2 = 0>
struct EvalShape {
    static constexpr int TH = NW * QF;
    static constexpr int RROWS = TH + MK - 1;
    static constexpr int RP = round4(kTW + MK - 1);      // R tile pitch (floats)
    static constexpr int RWIN = round4(MK + 3);          // register window per lane
    static constexpr int KP = round4(MK);                // K row pitch (floats)
    // backward split: MK = NW*KF + RM; warp w owns kernel rows [w*KF, (w+1)*KF)
    // over the whole tile and the RM last rows on its own QF-row slice, so
    // every warp does the same work
    static constexpr int KF = SPLIT == 2 ? 0 : SPLIT ? MK / NW : (MK + NW - 1) / NW;
    static constexpr int RM = SPLIT == 1 ? MK % NW : 0;
    static constexpr int QB = SPLIT == 2 ? MK : KF + RM;   // dK rows summed per warp
    // own rows: kernel rows per pass, full passes, rows of the last (short) pass
    static constexpr int NQ = own_rows_per_pass(MK);
    static constexpr int NPF = MK / NQ;
    static constexpr int NQL = MK - NPF * NQ;
    static constexpr int NP = red_size(MK * MK);         // partials per CTA
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
    static constexpr int SZ_K = (MK * KP + kBgMax + 1) * 4;
    static constexpr int OFF_D = (OFF_K + SZ_K + 15) & ~15;
    // float64 per-warp {loss, dB0, count, kR^2, k, background moments}
    static constexpr int SZ_D = kAccW * NW * 8;
    // float32 Kahan pairs (sum, compensation) of each warp's QB x MK dK rows
    // (all MK x MK for the own-rows backward)
    static constexpr int NK = QB * MK;
    static constexpr int OFF_KS = OFF_D + SZ_D;
    static constexpr int SZ_KS = NW * 2 * NK * 4;
    // F2: float2 pairs (K[a][b], K[a-1][b]) for the paired forward
    static constexpr int OFF_K2 = (OFF_KS + SZ_KS + 15) & ~15;
    static constexpr int SZ_K2 = (F2 & 1) ? MK * KP * 8 : 0;
    static constexpr int SMEM = OFF_K2 + SZ_K2;
};

// Polynomial background (Eq. 18) of the tile's TH x kTW pixels, written to
// B_out (pitch kTW): each thread takes one row segment of 16 pixels, forms the
// row's c_i(xi) = sum_j b_ij xi^j by Horner in xi and then B = sum_i c_i eta^i
// by Horner in eta.  b: the coefficients in theta order (float32).  Kept out of
// line so that the tile loop's code stays as compact as without a background.
struct BgCoords {
    int deg;
    float eta0, eta_s, xi0, xi_s;
};

static __device__ __noinline__ void bg_tile(const BgCoords bc, const float *b, float *B_out, int TH,
                                     int ty0, int tx0, int tid, int nt) {
    const int d = bc.deg;
    for (int e = tid; e < TH * (kTW / 16); e += nt) {
        const int r = e / (kTW / 16), x0 = (e % (kTW / 16)) * 16;
        const float xi = fmaf((float)(ty0 + r), bc.xi_s, bc.xi0);
        float c[kBgMaxDeg + 1];
        int k = 0;
#pragma unroll
        for (int i = 0; i <= kBgMaxDeg; ++i) {
            c[i] = 0.f;
            if (i <= d) {
                for (int j = d - i; j >= 0; --j) c[i] = fmaf(c[i], xi, b[k + j]);
                k += d - i + 1;
            }
        }
        float *out = B_out + r * kTW + x0;
#pragma unroll 4
        for (int p = 0; p < 16; ++p) {
            const float eta = fmaf((float)(tx0 + x0 + p), bc.eta_s, bc.eta0);
            float v = c[kBgMaxDeg];
#pragma unroll
            for (int i = kBgMaxDeg - 1; i >= 0; --i) v = fmaf(v, eta, c[i]);
            out[p] = v;
        }
    }
}

// Moments sum_p g_p eta^i xi^j of the background coefficients (Eq. 18)
// over this warp's qf rows of the g tile (out-of-range and masked pixels hold
// g = 0): float32 per lane over its 4 pixels of each row, summed over the warp,
// added by lane 0 to the warp's float64 slots w[5 + c - 1], c the coefficient
// index for the pair's degree d (c = 0, dL/dB0, is summed in the epilogue).
// All kBgMax moments of the largest degree are formed in registers (fixed
// indices) and those with i + j <= d kept.  Out of line, like bg_tile.
static __device__ __noinline__ void bg_moments(const BgCoords bc, int acc32, const float *gt, int qf,
                                        int ty0, int tx0, double *w, int warp, int lane) {
    float mom[kBgMax];
#pragma unroll
    for (int k = 0; k < kBgMax; ++k) mom[k] = 0.f;
    for (int q = 0; q < qf; ++q) {
        const int yl = warp * qf + q;
        const float xi = fmaf((float)(ty0 + yl), bc.xi_s, bc.xi0);
        const float4 g4 = *reinterpret_cast<const float4 *>(gt + yl * kTW + 4 * lane);
        const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
        float sx[kBgMaxDeg + 1];   // sum over the lane's pixels of g eta^i
#pragma unroll
        for (int i = 0; i <= kBgMaxDeg; ++i) sx[i] = 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float eta = fmaf((float)(tx0 + 4 * lane + p), bc.eta_s, bc.eta0);
            float e = gv[p];
#pragma unroll
            for (int i = 0; i <= kBgMaxDeg; ++i) {
                sx[i] += e;
                e *= eta;
            }
        }
        int k = 0;
#pragma unroll
        for (int i = 0; i <= kBgMaxDeg; ++i) {
            float t = sx[i];
#pragma unroll
            for (int j = 0; j <= kBgMaxDeg - i; ++j) {
                mom[k++] += t;
                t *= xi;
            }
        }
    }
    const int d = bc.deg;
    int k = 0;
#pragma unroll
    for (int i = 0; i <= kBgMaxDeg; ++i) {
#pragma unroll
        for (int j = 0; j <= kBgMaxDeg - i; ++j, ++k) {
            if (k == 0) continue;
            const float v = warp_sum(mom[k]);
            if (lane == 0 && i + j <= d) {
                const int c = i * (d + 1) - i * (i - 1) / 2 + j;   // index for degree d
                double *slot = w + 5 + c - 1;
                *slot = acc32 ? (double)((float)*slot + v) : *slot + (double)v;
            }
        }
    }
}

// Backward rows: dk[OFF+qb][b] += sum_rr sum_p g[y][x+p] R[r0+rr][x+b+p] with
// y = y0 + rr - qb, for NQ kernel rows.  Whole-tile rows (SLICE = false)
// rely on the zero rows around the g tile; slice rows (SLICE = true) keep
// y inside [y0, y0 + NS) and read a zero row otherwise.  Each R row window is
// loaded once and used by all NQ kernel rows, m column offsets and 4 pixels.
template <int MK, int QB, int OFF, int NQ, int RP, int RWIN, bool SLICE, int NS>
__device__ __forceinline__ void bwd_row(const float (&win)[RWIN], const float *g0, const float *gzero,
                                        int rr, float (&dk)[QB * MK]) {
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
            for (int b = 0; b < MK; ++b)
                dk[(OFF + qb) * MK + b] = fmaf(gv, win[b + p], dk[(OFF + qb) * MK + b]);
        }
    }
}

// Backward rows: dk[OFF+qb][b] += sum_rr sum_p g[y][x+p] R[r0+rr][x+b+p] with
// y = y0 + rr - qb, for NQ kernel rows.  Whole-tile rows (SLICE = false)
// rely on the zero rows around the g tile; slice rows (SLICE = true) keep
// y inside [y0, y0 + NS) and read a zero row otherwise.  Each R row window is
// loaded once and used by all NQ kernel rows, m column offsets and 4 pixels;
// with PF the next row's window is loaded while the current one is used.
template <int MK, int QB, int OFF, int NQ, int RP, int RWIN, bool SLICE, int NS, int PF>
__device__ __forceinline__ void bwd_rows(const float *rrow, const float *g0, const float *gzero,
                                         int n_rr, float (&dk)[QB * MK]) {
    if (PF) {
        float wa[RWIN], wb[RWIN];
        load_win<RWIN>(wa, rrow);
#pragma unroll 1
        for (int rr = 0; rr < n_rr; rr += 2) {
            const bool two = rr + 1 < n_rr;
            if (two) load_win<RWIN>(wb, rrow + (rr + 1) * RP);
            bwd_row<MK, QB, OFF, NQ, RP, RWIN, SLICE, NS>(wa, g0, gzero, rr, dk);
            if (two) {
                if (rr + 2 < n_rr) load_win<RWIN>(wa, rrow + (rr + 2) * RP);
                bwd_row<MK, QB, OFF, NQ, RP, RWIN, SLICE, NS>(wb, g0, gzero, rr + 1, dk);
            }
        }
    } else {
#pragma unroll 1
        for (int rr = 0; rr < n_rr; ++rr) {
            float win[RWIN];
            load_win<RWIN>(win, rrow + rr * RP);
            bwd_row<MK, QB, OFF, NQ, RP, RWIN, SLICE, NS>(win, g0, gzero, rr, dk);
        }
    }
}

// Own-rows backward, one pass of NQ kernel rows: dk[j][b] += sum_q sum_p
// gq[q][p] R[r][x+p+b] with r = j + q rows below rrow (rrow: the R row of the
// warp's first output row plus the pass's first kernel row, at this lane's
// pixel column).  Every (j, q) pair with j + q = s uses the window of row s,
// loaded once; all indices are compile-time, so dk stays in registers.
template <int MK, int NQ, int QF, int RP, int RWIN>
__device__ __forceinline__ void own_pass(const float *rrow, const float (&gq)[QF][4],
                                         float (&dk)[NQ * MK]) {
#pragma unroll
    for (int i = 0; i < NQ * MK; ++i) dk[i] = 0.f;
#pragma unroll
    for (int s = 0; s < NQ + QF - 1; ++s) {
        float win[RWIN];
        load_win<RWIN>(win, rrow + s * RP);
        // pixel p outer: consecutive FMAs update different accumulators
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
            for (int q = 0; q < QF; ++q) {
                const int j = s - q;
                if (j >= 0 && j < NQ) {
#pragma unroll
                    for (int b = 0; b < MK; ++b)
                        dk[j * MK + b] = fmaf(gq[q][p], win[p + b], dk[j * MK + b]);
                }
            }
        }
    }
}

// Warp sum of N per-lane values (halving) added to this warp's float32 Kahan
// pairs sum[i], comp[i] (plain float32 sums with acc32); kidx from
// halving_index<N>.
template <int N>
__device__ __forceinline__ void warp_kahan_add(const float (&v)[N], const int (&kidx)[Halving<N>::H5],
                                               float *sum, float *comp, int acc32, int lane) {
    using Hv = Halving<N>;
    float w1[Hv::H1], w2[Hv::H2], w3[Hv::H3], w4[Hv::H4], w5[Hv::H5];
    halve<N, 16>(v, w1, lane & 16);
    halve<Hv::H1, 8>(w1, w2, lane & 8);
    halve<Hv::H2, 4>(w2, w3, lane & 4);
    halve<Hv::H3, 2>(w3, w4, lane & 2);
    halve<Hv::H4, 1>(w4, w5, lane & 1);
#pragma unroll
    for (int j = 0; j < Hv::H5; ++j) {
        const int ix = kidx[j];
        if (ix >= 0) {
            float *sm = sum + ix, *cm = comp + ix;
            if (acc32) {
                *sm += w5[j];
            } else {
                const float y = w5[j] - *cm;
                const float t = *sm + y;
                *cm = (t - *sm) - y;
                *sm = t;
            }
        }
    }
}

// The fused pass over tiles t_begin, t_begin + t_step, ... < t_end of one
// pair; the CTA's partial sums (m*m + 5 float64) go to `out`.  Called by
// the single-pair kernel (tiles strided over the grid) and by the batched
// kernel (a contiguous tile range of one pair per work item).
// BG = 1: the kernel also handles a polynomial background (args.bg_deg > 0);
// BG = 0 kernels take the constant B0 only.
template <int MK, int NW, int QF, int PF, int SPLIT, int MODE, int F2 = 0, int BG = 0>
__device__ __forceinline__ void process_tiles(const EvalArgs &args, unsigned char *smem, int t_begin,
                                              int t_end, int t_step, double *out) {
    using S = EvalShape<MK, NW, QF, SPLIT, F2>;
    static_assert(!(F2 & 1) || QF % 2 == 0, "the paired forward pairs output rows");
    constexpr int TH = S::TH, RP = S::RP, RWIN = S::RWIN, KP = S::KP, QB = S::QB;
    constexpr int H2 = MK / 2;

    float *Rbuf0 = reinterpret_cast<float *>(smem + S::OFF_R);
    float *Rbuf1 = Rbuf0 + S::RROWS * RP;
    float *gs = reinterpret_cast<float *>(smem + S::OFF_G);
    float *Ks = reinterpret_cast<float *>(smem + S::OFF_K);
    double *acc64 = reinterpret_cast<double *>(smem + S::OFF_D);  // per warp, kAccW each
    float *kahan = reinterpret_cast<float *>(smem + S::OFF_KS);    // per warp [NK sums | NK comps]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < MK * KP + kBgMax + 1; i += S::NT) Ks[i] = args.Kpad[i];
    float2 *K2 = reinterpret_cast<float2 *>(smem + S::OFF_K2);   // F2 only
    if constexpr ((F2 & 1) != 0) {
        for (int i = tid; i < MK * KP; i += S::NT) {
            const int a = i / KP;
            K2[i] = make_float2(args.Kpad[i], a > 0 ? args.Kpad[i - KP] : 0.f);
        }
    }
    if (MODE == kModeGrad) {
        for (int i = tid; i < kAccW * NW; i += S::NT) acc64[i] = 0.0;
        for (int i = tid; i < NW * 2 * S::NK; i += S::NT) kahan[i] = 0.f;
        for (int i = tid; i < S::GPAD * kTW; i += S::NT) {
            gs[i] = 0.f;
            gs[(S::GPAD + TH) * kTW + i] = 0.f;
        }
    }
    float *gt = gs + S::GPAD * kTW;   // g tile row 0
    __syncthreads();
    const bool poly = BG && args.bg_deg > 0;
    const BgCoords bc = {args.bg_deg, args.eta0, args.eta_s, args.xi0, args.xi_s};
    // the constant background, added in the epilogue; a polynomial one is added
    // to the accumulators before it
    const float B0 = poly ? 0.f : Ks[MK * KP];

    constexpr int KF = S::KF, RM = S::RM;
    // whole-tile kernel rows of this warp: [a_lo, a_lo + nq)
    const int a_lo = SPLIT ? warp * KF : (warp * MK) / NW;
    const int nq = SPLIT ? KF : ((warp + 1) * MK) / NW - a_lo;

    // per-lane float32 loss / dB0 / count / curvature sums, flushed to the
    // per-warp float64 accumulators every FLUSH tiles (<= 4096 px per lane)
    float lsum = 0.f, gsum = 0.f, cnt = 0.f, ksum = 0.f, kr2sum = 0.f;
    int since_flush = 0;
    auto flush = [&]() {
        const float l = warp_sum(lsum), g = warp_sum(gsum), c = warp_sum(cnt);
        const float k = warp_sum(ksum), kr = warp_sum(kr2sum);
        if (lane == 0) {
            double *w5 = acc64 + kAccW * warp;
            if (args.acc32) {   // float32 running sums (kept in the float64 slots)
                w5[0] = (double)((float)w5[0] + l);
                w5[1] = (double)((float)w5[1] + g);
                w5[2] = (double)((float)w5[2] + c);
                w5[3] = (double)((float)w5[3] + kr);
                w5[4] = (double)((float)w5[4] + k);
            } else {
                w5[0] += (double)l;
                w5[1] += (double)g;
                w5[2] += (double)c;
                w5[3] += (double)kr;
                w5[4] += (double)k;
            }
        }
        lsum = gsum = cnt = ksum = kr2sum = 0.f;
    };
    // dK of one tile: per-lane float32 sums over the tile's 4 x TH pixels,
    // reduced over the warp by halving and added (Kahan-compensated float32)
    // to this warp's shared accumulators
    constexpr int NK = S::NK;
    constexpr int NKO = SPLIT == 2 ? 1 : NK;   // values of the row-split backward's tile reduction
    constexpr int NF = Halving<NKO>::H5;
    float *ksum_w = kahan + warp * 2 * NK;
    int kidx[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) kidx[j] = halving_index<NKO>(lane, j);
    // own rows: the reduction index maps of a full pass and of the short last one
    constexpr int NQ = S::NQ, NQL = S::NQL, NQLH = NQL > 0 ? NQL : 1;
    constexpr int NFQ = SPLIT == 2 ? Halving<NQ * MK>::H5 : 1;
    constexpr int NFL = SPLIT == 2 ? Halving<NQLH * MK>::H5 : 1;
    int kidq[NFQ], kidl[NFL];
    if constexpr (SPLIT == 2) {
#pragma unroll
        for (int j = 0; j < NFQ; ++j) kidq[j] = halving_index<NQ * MK>(lane, j);
#pragma unroll
        for (int j = 0; j < NFL; ++j) kidl[j] = halving_index<NQLH * MK>(lane, j);
    }

    // a fixed scalar variance: 1/v and sqrt(1/v) once per thread
    const bool scalar_var = args.lp.var_model == 0 && args.var == nullptr;
    const float sv_inv_v = 1.0f / args.lp.var_scalar;
    const float sv_inv_s = sqrtf(sv_inv_v);

    // ---- 1. R tiles (+ halo) are staged with cp.async, the next tile's copy
    // overlapping the current tile's compute (two buffers)
    const bool vec = ((args.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(args.R) & 15) == 0);
    if (t_begin < t_end)
        stage_tile<S::RROWS, RP, S::NT>(Rbuf0, args, (t_begin / args.tiles_x) * TH,
                                        (t_begin % args.tiles_x) * kTW, vec);
    cp_async_commit();
    int buf = 0;
    for (int tile = t_begin; tile < t_end; tile += t_step, buf ^= 1) {
        const int ty0 = (tile / args.tiles_x) * TH;
        const int tx0 = (tile % args.tiles_x) * kTW;
        const int nxt = tile + t_step;
        if (nxt < t_end)
            stage_tile<S::RROWS, RP, S::NT>(buf ? Rbuf0 : Rbuf1, args, (nxt / args.tiles_x) * TH,
                                            (nxt % args.tiles_x) * kTW, vec);
        cp_async_commit();
        // a polynomial background: B over the tile into the g tile's rows (the
        // epilogue reads it back before writing g there)
        if (poly) bg_tile(bc, Ks + MK * KP, gt, TH, ty0, tx0, tid, S::NT);
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
        auto fwd_interior = [&](const float (&win)[RWIN], int r) {
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
        };
        if constexpr ((F2 & 1) != 0) {
            // output rows paired (2i, 2i+1): kernel rows a = r - 2i and a - 1 in one
            // packed FMA per column b, the R value broadcast to both halves
            float2 accp[QF / 2][4];
#pragma unroll
            for (int i = 0; i < QF / 2; ++i)
#pragma unroll
                for (int p = 0; p < 4; ++p) accp[i][p] = make_float2(0.f, 0.f);
            const float4 *K24 = reinterpret_cast<const float4 *>(K2);
#pragma unroll 1
            for (int r = QF - 1; r <= MK - 1; ++r) {
                float win[RWIN];
                load_win<RWIN>(win, rbase + r * RP);
#pragma unroll
                for (int b2 = 0; b2 < KP / 2; ++b2) {
                    float4 kk[QF / 2];
#pragma unroll
                    for (int i = 0; i < QF / 2; ++i) kk[i] = K24[((r - 2 * i) * KP) / 2 + b2];
#pragma unroll
                    for (int bb = 0; bb < 2; ++bb) {
                        const int b = 2 * b2 + bb;
                        if (b < MK) {
#pragma unroll
                            for (int i = 0; i < QF / 2; ++i) {
                                const float2 kv = bb == 0 ? make_float2(kk[i].x, kk[i].y)
                                                          : make_float2(kk[i].z, kk[i].w);
#pragma unroll
                                for (int p = 0; p < 4; ++p)
                                    accp[i][p] = __ffma2_rn(kv, make_float2(win[p + b], win[p + b]),
                                                            accp[i][p]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < QF / 2; ++i)
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    acc[2 * i][p] = accp[i][p].x;
                    acc[2 * i + 1][p] = accp[i][p].y;
                }
        } else if constexpr (PF != 0) {
            // the next row's window is loaded while the current one is used
            float wa[RWIN], wb[RWIN];
            if (QF - 1 <= MK - 1) load_win<RWIN>(wa, rbase + (QF - 1) * RP);
#pragma unroll 1
            for (int r = QF - 1; r <= MK - 1; r += 2) {
                const bool two = r + 1 <= MK - 1;
                if (two) load_win<RWIN>(wb, rbase + (r + 1) * RP);
                fwd_interior(wa, r);
                if (two) {
                    if (r + 2 <= MK - 1) load_win<RWIN>(wa, rbase + (r + 2) * RP);
                    fwd_interior(wb, r + 1);
                }
            }
        } else {
#pragma unroll 1
            for (int r = QF - 1; r <= MK - 1; ++r) {
                float win[RWIN];
                load_win<RWIN>(win, rbase + r * RP);
                fwd_interior(win, r);
            }
        }
        // the first and last QF-1 R rows feed only some output rows (with
        // MK < QF - 1 there is no interior and every row is done here once);
        // unrolled, so that each row's kernel rows are compile-time (no branches)
        constexpr bool kSplit = MK >= QF - 1;
        constexpr int kEdges = kSplit ? 2 * (QF - 1) : (QF + MK - 1);
#pragma unroll
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

        // ---- 3. epilogue: loss terms, g -> shared tile (two instances: a fixed
        // scalar variance with its reciprocals from registers, and the general form)
        auto epilogue = [&](auto sv_tag) {
            constexpr bool SV = decltype(sv_tag)::value;
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
                        const float M = acc[q][p] + (poly ? gt[yl * kTW + xl] : B0);
                        const float Iv = __ldg(args.I + off);
                        float g, z, kap, ell;
                        if constexpr (SV) {
                            ell = pixel_loss_fixed(args.lp, sv_inv_v, sv_inv_s, Iv, M, g, z, kap);
                        } else {
                            const float vm = args.var ? __ldg(args.var + off) : args.lp.var_scalar;
                            const float F = args.flat ? __ldg(args.flat + off) : 1.0f;
                            ell = pixel_loss(args.lp, Iv, M, vm, F, g, z, kap);
                        }
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
                    if (MODE == kModeGrad) {
                        // the own-rows backward keeps g in acc; the g tile serves the
                        // row-split backward and the background moments
                        if (SPLIT != 2 || poly) gt[yl * kTW + xl] = gval;
                        if constexpr (SPLIT == 2) acc[q][p] = gval;
                    }
                }
            }
        };
        if (scalar_var)
            epilogue(std::true_type{});
        else
            epilogue(std::false_type{});
        if (MODE != kModeGrad) {
            __syncthreads();  // the R buffer is refilled two tiles later
            continue;
        }
        if (SPLIT != 2 || poly) __syncthreads();  // g tile complete
        if (poly) bg_moments(bc, args.acc32, gt, QF, ty0, tx0, acc64 + kAccW * warp, warp, lane);

        // ---- 4. backward: dK[a][b] += sum_{y,x} g[y][x] R[y+a][x+b]
        if constexpr (SPLIT == 2) {
            // own rows: the warp's QF output rows, every kernel row, passes of NQ
            const float *rw = Rs + (warp * QF) * RP + 4 * lane;
#pragma unroll 1
            for (int ps = 0; ps < S::NPF; ++ps) {
                float dq[NQ * MK];
                own_pass<MK, NQ, QF, RP, RWIN>(rw + ps * NQ * RP, acc, dq);
                warp_kahan_add<NQ * MK>(dq, kidq, ksum_w + ps * NQ * MK, ksum_w + NK + ps * NQ * MK,
                                        args.acc32, lane);
            }
            if constexpr (NQL > 0) {
                float dl[NQLH * MK];
                own_pass<MK, NQLH, QF, RP, RWIN>(rw + S::NPF * NQ * RP, acc, dl);
                warp_kahan_add<NQLH * MK>(dl, kidl, ksum_w + S::NPF * NQ * MK,
                                          ksum_w + NK + S::NPF * NQ * MK, args.acc32, lane);
            }
        } else {
            float dk[NK];
#pragma unroll
            for (int i = 0; i < NK; ++i) dk[i] = 0.f;
            const float *gzero = gs + 4 * lane;   // a zero row above the g tile
            if (KF > 0 && nq == KF)
                bwd_rows<MK, QB, 0, (KF > 0 ? KF : 1), RP, RWIN, false, TH, PF>(
                    Rs + a_lo * RP + 4 * lane, gt + 4 * lane, gzero, TH + KF - 1, dk);
            else if (KF > 1 && nq == KF - 1)   // SPLIT 0: the warps with one row fewer
                bwd_rows<MK, QB, 0, (KF > 1 ? KF - 1 : 1), RP, RWIN, false, TH, PF>(
                    Rs + a_lo * RP + 4 * lane, gt + 4 * lane, gzero, TH + KF - 2, dk);
            if (RM > 0) {
                const int ys = warp * QF;          // this warp's slice of the tile rows
                bwd_rows<MK, QB, KF, (RM > 0 ? RM : 1), RP, RWIN, true, QF, 0>(
                    Rs + (NW * KF + ys) * RP + 4 * lane, gt + ys * kTW + 4 * lane, gzero,
                    QF + RM - 1, dk);
            }
            // ---- 5. warp-reduce this tile's dK and add it to the warp's accumulators
            warp_kahan_add<NK>(dk, kidx, ksum_w, ksum_w + NK, args.acc32, lane);
        }
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
        // rows with one owner warp (w, qb < nq(w)); the RM shared rows (every
        // row with the own-rows backward) summed over the warps' copies in a
        // fixed order
        for (int i = tid; i < MK * MK; i += S::NT) {
            const int a = i / MK, b = i - a * MK;
            // row qb of every warp's accumulators, summed in warp order
            auto all_warps = [&](int qb) {
                double t = 0.0;
                float t32 = 0.f;
                for (int w = 0; w < NW; ++w) {
                    const float *kw = kahan + w * 2 * NK;
                    t += (double)kw[qb * MK + b] - (double)kw[NK + qb * MK + b];
                    t32 += kw[qb * MK + b];
                }
                return args.acc32 ? (double)t32 : t;
            };
            double t;
            if constexpr (SPLIT == 2) {
                t = all_warps(a);
            } else if (a < MK - RM) {
                int w = SPLIT ? a / KF : 0;
                if (!SPLIT) {
                    while (w + 1 < NW && ((w + 1) * MK) / NW <= a) ++w;
                }
                const int qb = a - (SPLIT ? w * KF : (w * MK) / NW);
                const float *kw = kahan + w * 2 * NK;
                t = (double)kw[qb * MK + b] - (double)kw[NK + qb * MK + b];
            } else {
                t = all_warps(KF + (a - (MK - RM)));
            }
            out[1 + i] = t;
        }
        if (tid < kAccW) {
            // tid 0: loss, 1: dB0, 2: pixel count, 3: sum kappa R^2, 4: sum kappa,
            // 5 + c: background coefficient 1 + c
            double t = 0.0;
            float t32 = 0.f;
            for (int w = 0; w < NW; ++w) {
                t += acc64[kAccW * w + tid];
                t32 += (float)acc64[kAccW * w + tid];
            }
            const int o = tid == 0  ? 0
                          : tid == 1 ? MK * MK + 1
                          : tid < 5  ? red_count(MK * MK) + tid - 2
                                     : MK * MK + 1 + (tid - 4);
            out[o] = args.acc32 ? (double)t32 : t;
        }
    }
}

template <int MK, int NW, int QF, int PF, int SPLIT, int MODE, int F2 = 0, int BG = 0>
__global__ void __launch_bounds__(NW * 32, 1) eval_kernel(const EvalArgs args) {
    if (args.done_flag != nullptr && *((volatile const int *)args.done_flag) != 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    process_tiles<MK, NW, QF, PF, SPLIT, MODE, F2, BG>(
        args, smem, blockIdx.x, args.n_tiles, gridDim.x,
        MODE == kModeGrad ? args.partials + (size_t)blockIdx.x * EvalShape<MK, NW, QF, SPLIT, F2>::NP
                          : nullptr);
}

}  // namespace dia

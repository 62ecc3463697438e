// Fused evaluation with a spatially varying kernel.
//
// The paper names kernels that vary over the image as the natural extension
// of DIA (Sec. 1, citing Alard 2000 and Bramich et al. 2013) without fitting
// one.  Reading taken here (the Bramich et al. 2013 form): every kernel pixel
// is a polynomial of degree dk in the normalised coordinates of Eq. 19,
//   K_ab(x, y) = sum_{p+q <= dk} K_pq[a][b] eta^p xi^q,
// evaluated at the output pixel, so with phi_c = eta^p xi^q (c in the
// coefficient order of Eq. 18, power of xi fastest)
//   M = sum_c phi_c (R (x) K_c) + B,                       (Eq. 2 per term)
//   dL/dK_c[a][b] = sum_p g_p phi_c(p) R[y+a][x+b],   g = dl/dM (Eq. 8 / 13).
// theta = [K_0 (m*m), K_1, ..., K_{nc-1}, background coefficients], nc =
// (dk+1)(dk+2)/2.  M is still linear in theta.
//
// One CTA (8 warps) owns a 16 x 128 output tile at a time (persistent loop):
// the R tile with its (m-1) halo is staged in shared memory; warp w computes
// output rows 2w, 2w+1, lane l four columns; per coefficient c it forms the
// correlation with K_c from a register window of each R row and adds
// phi_c times it to M; the epilogue forms the loss and g in float32 (the same
// pixel terms as the constant-kernel kernels) and writes g to a shared tile.
// Backward, per c: the tile of g phi_c, then warp w accumulates the kernel
// rows a = w, w + 8, ... (lane: its four columns, every tile row; float32 over
// one tile), a warp sum and a float64 add into the CTA's accumulators.
// Background moments sum g eta^i xi^j are float32 per lane over one tile,
// then float64.  Per-CTA partials: loss, dK (nc m^2), the kBgMax background
// slots, pixel count and the two curvature sums, reduced in a fixed order by
// the same kernel as the other evaluations.
#include <cstdint>
#include <cuda_runtime.h>

#include "dia_eval.cuh"
#include "dia_svk.h"

namespace dia {

namespace {

constexpr int kVW = 8;               // warps
constexpr int kVNT = kVW * 32;
constexpr int kVTH = 2 * kVW;        // tile rows (2 per warp)

template <int MK>
struct SvkShape {
    static constexpr int RROWS = kVTH + MK - 1;
    static constexpr int RP = round4(kTW + MK - 1);
    static constexpr int RWIN = round4(MK + 3);
    static constexpr int KP = round4(MK);
    static constexpr int NK1 = MK * MK;
    // shared layout (bytes): R tile, g tile, g*phi tile, K blocks, float64
    // accumulators: per warp [loss, count, kR^2, kappa, bg moments kBgMax],
    // then dK (nc m^2; kernel row a is only written by warp a % 8)
    static constexpr int NW5 = 4 + kBgMax;
    static constexpr int OFF_R = 0;
    static constexpr int SZ_R = RROWS * RP * 4;
    static constexpr int OFF_G = OFF_R + SZ_R;
    static constexpr int SZ_G = kVTH * kTW * 4;
    static constexpr int OFF_GC = OFF_G + SZ_G;
    static constexpr int OFF_K = OFF_GC + SZ_G;
    static constexpr int SZ_K = kSvkMaxNc * MK * KP * 4 + (kBgMax + 1) * 4;
    static constexpr int OFF_D = (OFF_K + SZ_K + 15) & ~15;
    static constexpr int NACC = kVW * NW5 + kSvkMaxNc * NK1;
    static constexpr int SMEM = OFF_D + NACC * 8;
};

// eta^i (pe) and xi^j (px) for i, j <= 4 at valid-region pixel (y, x)
__device__ __forceinline__ void powers(const EvalArgs &a, int y, int x, float (&pe)[5],
                                       float (&px)[5]) {
    const float eta = fmaf((float)x, a.eta_s, a.eta0);
    const float xi = fmaf((float)y, a.xi_s, a.xi0);
    pe[0] = 1.f;
    px[0] = 1.f;
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        pe[i] = pe[i - 1] * eta;
        px[i] = px[i - 1] * xi;
    }
}

// basis function c of degree deg (coefficient order of Eq. 18)
__device__ __forceinline__ float basis(int deg, int c, const float (&pe)[5], const float (&px)[5]) {
    int k = 0;
    for (int i = 0; i <= deg; ++i)
        for (int j = 0; j <= deg - i; ++j, ++k)
            if (k == c) return pe[i] * px[j];
    return 0.f;
}

template <int MK, int MODE>
__global__ void __launch_bounds__(kVNT, 1) eval_svk_kernel(const EvalArgs a, const SvkArgs v) {
    if (a.done_flag != nullptr && *((volatile const int *)a.done_flag) != 0) return;
    using S = SvkShape<MK>;
    constexpr int RP = S::RP, RWIN = S::RWIN, KP = S::KP, NK1 = S::NK1, H2 = MK / 2;
    extern __shared__ __align__(16) unsigned char smem[];
    float *Rs = reinterpret_cast<float *>(smem + S::OFF_R);
    float *gt = reinterpret_cast<float *>(smem + S::OFF_G);
    float *gc = reinterpret_cast<float *>(smem + S::OFF_GC);
    float *Ks = reinterpret_cast<float *>(smem + S::OFF_K);
    double *acc64 = reinterpret_cast<double *>(smem + S::OFF_D);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nc = v.nc, kdeg = v.kdeg, nb = n_background(a.bg_deg);
    const int nkt = nc * NK1;

    for (int i = tid; i < nc * MK * KP + kBgMax + 1; i += kVNT) Ks[i] = a.Kpad[i];
    if (MODE == kModeGrad)
        for (int i = tid; i < S::NACC; i += kVNT) acc64[i] = 0.0;
    const float *bgc = Ks + nc * MK * KP;   // background coefficients
    const bool vec = ((a.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.R) & 15) == 0);

    for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int ty0 = (tile / a.tiles_x) * kVTH, tx0 = (tile % a.tiles_x) * kTW;
        __syncthreads();   // the previous tile's shared data is no longer read
        stage_tile<S::RROWS, RP, kVNT>(Rs, a, ty0, tx0, vec);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();

        // ---- forward and epilogue: rows 2 warp + q, columns 4 lane + p
        float lsum = 0.f, gsum = 0.f, cnt = 0.f, ksum = 0.f, kr2 = 0.f;
        float bgm[kBgMax];
#pragma unroll
        for (int i = 0; i < kBgMax; ++i) bgm[i] = 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int yl = 2 * warp + q, y = ty0 + yl;
            float pe[4][5], px[4][5];
#pragma unroll
            for (int p = 0; p < 4; ++p) powers(a, y, tx0 + 4 * lane + p, pe[p], px[p]);
            float M[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                // background (Eq. 18): sum_i b_i (basis i)
                float B = 0.f;
                for (int i = 0; i < nb; ++i) B = fmaf(bgc[i], basis(a.bg_deg, i, pe[p], px[p]), B);
                M[p] = B;
            }
            for (int c = 0; c < nc; ++c) {
                const float *Kc = Ks + c * MK * KP;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
                for (int aa = 0; aa < MK; ++aa) {
                    float win[RWIN];
                    load_win<RWIN>(win, Rs + (yl + aa) * RP + 4 * lane);
#pragma unroll
                    for (int b = 0; b < MK; ++b) {
                        const float kv = Kc[aa * KP + b];
#pragma unroll
                        for (int p = 0; p < 4; ++p) acc[p] = fmaf(kv, win[p + b], acc[p]);
                    }
                }
#pragma unroll
                for (int p = 0; p < 4; ++p) M[p] = fmaf(basis(kdeg, c, pe[p], px[p]), acc[p], M[p]);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int xl = 4 * lane + p, x = tx0 + xl;
                float gval = 0.f;
                if (y < a.Hv && x < a.Wv) {
                    const size_t off = (size_t)(y + H2) * a.ld + (x + H2);
                    const bool use = (a.mask == nullptr) || (a.mask[off] != 0);
                    const float Iv = __ldg(a.I + off);
                    const float vm = a.var ? __ldg(a.var + off) : a.lp.var_scalar;
                    const float F = a.flat ? __ldg(a.flat + off) : 1.0f;
                    float g, z, kap;
                    const float ell = pixel_loss(a.lp, Iv, M[p], vm, F, g, z, kap);
                    if (MODE == kModeGrad) {
                        if (use) {
                            const float rc = Rs[(yl + H2) * RP + xl + H2];
                            lsum += ell;
                            gsum += g;
                            cnt += 1.f;
                            ksum += kap;
                            kr2 = fmaf(kap * rc, rc, kr2);
                            for (int i = 1; i < nb; ++i)
                                bgm[i] = fmaf(g, basis(a.bg_deg, i, pe[p], px[p]), bgm[i]);
                            gval = g;
                        }
                    } else {
                        if (a.diff_out) a.diff_out[(size_t)y * a.Wv + x] = Iv - M[p];
                        if (a.mask_out && use && fabsf(z) > a.clip_kappa) a.mask_out[off] = 0;
                    }
                }
                if (MODE == kModeGrad) gt[yl * kTW + xl] = gval;
            }
        }
        if (MODE != kModeGrad) continue;
        // loss, count, curvature and background sums of this tile: warp sums,
        // float64 adds into this warp's own slots
        {
            const float l = warp_sum(lsum), c1 = warp_sum(cnt), kr = warp_sum(kr2),
                        k1 = warp_sum(ksum), g1 = warp_sum(gsum);
            float bw[kBgMax];
#pragma unroll
            for (int i = 1; i < kBgMax; ++i) bw[i] = warp_sum(bgm[i]);
            if (lane == 0) {
                double *w5 = acc64 + warp * S::NW5;
                w5[0] += (double)l;
                w5[1] += (double)c1;
                w5[2] += (double)kr;
                w5[3] += (double)k1;
                w5[4] += (double)g1;
#pragma unroll
                for (int i = 1; i < kBgMax; ++i) w5[4 + i] += (double)bw[i];
            }
        }

        // ---- backward, per coefficient c: dK_c[a][b] += sum g phi_c R
        for (int c = 0; c < nc; ++c) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int yl = 2 * warp + q;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int xl = 4 * lane + p;
                    float pe[5], px[5];
                    powers(a, ty0 + yl, tx0 + xl, pe, px);
                    gc[yl * kTW + xl] = gt[yl * kTW + xl] * basis(kdeg, c, pe, px);
                }
            }
            __syncthreads();
            for (int aa = warp; aa < MK; aa += kVW) {
                float dk[MK];
#pragma unroll
                for (int b = 0; b < MK; ++b) dk[b] = 0.f;
#pragma unroll 1
                for (int yl = 0; yl < kVTH; ++yl) {
                    const float4 g4 = *reinterpret_cast<const float4 *>(gc + yl * kTW + 4 * lane);
                    float win[RWIN];
                    load_win<RWIN>(win, Rs + (yl + aa) * RP + 4 * lane);
                    const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int b = 0; b < MK; ++b) dk[b] = fmaf(gv[p], win[p + b], dk[b]);
                }
#pragma unroll
                for (int b = 0; b < MK; ++b) {
                    const float s = warp_sum(dk[b]);
                    if (lane == 0) acc64[kVW * S::NW5 + c * NK1 + aa * MK + b] += (double)s;
                }
            }
            __syncthreads();   // gc is rewritten for the next c
        }
    }
    if (MODE != kModeGrad) return;
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * v.np;
    for (int k = tid; k < v.np; k += kVNT) {
        // 0 loss, 1..nkt dK, nkt+1 dB0, nkt+2.. background slots, then count,
        // kR^2, kappa (red_count(nkt) onwards); per-warp slots summed in warp order
        int slot = -1;
        double t = 0.0;
        if (k == 0) slot = 0;
        else if (k <= nkt) t = acc64[kVW * S::NW5 + (k - 1)];
        else if (k <= nkt + kBgMax) slot = 4 + (k - nkt - 1);
        else if (k == red_count(nkt)) slot = 1;
        else if (k == red_count(nkt) + 1) slot = 2;
        else if (k == red_count(nkt) + 2) slot = 3;
        if (slot >= 0)
            for (int w = 0; w < kVW; ++w) t += acc64[w * S::NW5 + slot];
        out[k] = t;
    }
}

struct SvkFns {
    const void *fn[2];
    int smem;
};

template <int MK>
SvkFns svk_fns() {
    return {{(const void *)&eval_svk_kernel<MK, kModeGrad>,
             (const void *)&eval_svk_kernel<MK, kModeForward>},
            SvkShape<MK>::SMEM};
}

bool svk_lookup(int mk, SvkFns *o) {
    switch (mk) {
        case 1: *o = svk_fns<1>(); return true;
        case 3: *o = svk_fns<3>(); return true;
        case 5: *o = svk_fns<5>(); return true;
        case 7: *o = svk_fns<7>(); return true;
        case 9: *o = svk_fns<9>(); return true;
        case 11: *o = svk_fns<11>(); return true;
        case 13: *o = svk_fns<13>(); return true;
        case 15: *o = svk_fns<15>(); return true;
        case 17: *o = svk_fns<17>(); return true;
        case 19: *o = svk_fns<19>(); return true;
        case 21: *o = svk_fns<21>(); return true;
        case 23: *o = svk_fns<23>(); return true;
        case 25: *o = svk_fns<25>(); return true;
        case 27: *o = svk_fns<27>(); return true;
        case 29: *o = svk_fns<29>(); return true;
        case 31: *o = svk_fns<31>(); return true;
        default: return false;
    }
}

}  // namespace

int svk_tile_rows() { return kVTH; }

cudaError_t svk_prepare(int mk, int *occ, int *smem) {
    SvkFns f;
    if (!svk_lookup(mk, &f)) return cudaErrorInvalidValue;
    for (int md = 0; md < 2; ++md) {
        cudaError_t e = cudaFuncSetAttribute(f.fn[md], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             f.smem);
        if (e != cudaSuccess) return e;
    }
    *smem = f.smem;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, f.fn[kModeGrad], kVNT, f.smem);
}

cudaError_t launch_eval_svk(const EvalArgs &a, const SvkArgs &v, int mk, int mode, int grid,
                            cudaStream_t s) {
    SvkFns f;
    if (!svk_lookup(mk, &f)) return cudaErrorInvalidValue;
    void *params[] = {(void *)&a, (void *)&v};
    return cudaLaunchKernel(f.fn[mode], dim3(grid), dim3(kVNT), params, f.smem, s);
}

}  // namespace dia

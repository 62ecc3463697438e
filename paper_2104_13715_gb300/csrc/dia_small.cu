// Fused evaluation for small kernels (m = 1, 3, 5): the memory-bound end of
// the method (Sec. 5.3's kernel-size sweep starts at these sides).
//
// Per pixel the work is 2 m^2 FMAs (forward, Eq. 2, and the weight gradient
// dL/dK[a][b] = sum_p g_p R[y+a][x+b]) plus the loss epilogue (Eq. 8 / Eq. 13),
// against 8-17 bytes of input, so the kernel must stream R, I and the optional
// maps from HBM at full rate while issuing as few instructions per pixel as
// possible.  Design (differs from the tiled kernel used for m >= 7):
//
//   * warp-private work: a warp owns a strip of S output rows of one block of
//     128 full-image columns; lane l owns columns cb + 4l .. cb + 4l + 3 of
//     every row of the strip (columns outside the valid region are masked);
//   * staging: each warp keeps a private ring of D row slots in shared memory,
//     filled by cp.async (16-byte chunks, zero-filled outside the image) D rows
//     ahead of use; slot t holds R row i0 - h + t and the target, mask, variance
//     and flat rows of output row i0 + t - 2h.  Only __syncwarp between stages:
//     no CTA barrier inside the strip;
//   * registers: the 4 + 2h window columns of the last m R rows are a register
//     ring (the row loop is unrolled by m so ring slots are compile-time); the
//     forward sum, g = dl/dM, and the m^2 weight-gradient FMAs of each pixel run
//     on the same registers (M is never stored, no g tile);
//   * sums: float32 per lane over one strip (<= 4 S <= 4096 pixels), then a halving
//     butterfly over the warp and float64 per lane; one CTA-wide float64 sum at
//     the end gives the same per-CTA partials as the tiled kernel (loss, dK,
//     dB0, pixel count, curvature sums), reduced by the same fixed-order kernel.
#include <cstdint>
#include <cuda_runtime.h>

#include "dia_eval.cuh"
#include "dia_small.h"

namespace dia {

namespace {

constexpr int kSW = 8;            // warps per CTA
constexpr int kSNT = kSW * 32;
constexpr int kSDepth = 8;        // row slots per warp ring
constexpr int kSColBlock = 128;   // full-image columns per strip

// shared-memory bytes of one row slot: R (136 floats from cb - 4), I, and
// the optional var / flat rows (128 floats each from cb), mask (128 bytes)
__host__ __device__ inline int slot_bytes(int has_mask, int has_var, int has_flat) {
    return 136 * 4 + 128 * 4 + (has_var ? 512 : 0) + (has_flat ? 512 : 0) + (has_mask ? 128 : 0);
}

__device__ __forceinline__ void cpa16(void *dst, const void *src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cpa_wait_depth() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kSDepth - 1));
}
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

struct SlotLayout {
    int off_I, off_var, off_flat, off_mask, bytes;
};

// Stage slot t of the strip (R row i0 - h + t; target-side rows of output
// row i0 + t - 2h when that row lies in the strip) into `slot`.
template <int MK>
__device__ __forceinline__ void stage_slot(unsigned char *slot, const SlotLayout &sl,
                                           const EvalArgs &a, int cb, int i0, int i1, int t,
                                           int lane) {
    constexpr int h = MK / 2;
    const int rr = i0 - h + t;                 // R row (in [0, H) while t < i1 - i0 + 2h)
    const int io = i0 + t - 2 * h;             // output row of the target-side rows
    if (rr >= i1 + h) return;                  // past the strip: nothing to stage
    float *Rs = reinterpret_cast<float *>(slot);
    // R: 34 chunks of 4 floats from column cb - 4
    for (int c = lane; c < 34; c += 32) {
        const int gx = cb - 4 + 4 * c;
        int bytes = 0;
        const float *src = a.R;
        if (gx >= 0 && gx < a.W) {
            bytes = (a.W - gx >= 4) ? 16 : 4 * (a.W - gx);
            src = a.R + (size_t)rr * a.ld + gx;
        }
        cpa16(Rs + 4 * c, src, bytes);
    }
    if (io < i0) return;
    const int gx = cb + 4 * lane;
    const bool in = gx < a.W;
    const int bytes = in ? ((a.W - gx >= 4) ? 16 : 4 * (a.W - gx)) : 0;
    const size_t off = (size_t)io * a.ld + (in ? gx : 0);
    cpa16(slot + sl.off_I + 16 * lane, a.I + off, bytes);
    if (a.var) cpa16(slot + sl.off_var + 16 * lane, a.var + off, bytes);
    if (a.flat) cpa16(slot + sl.off_flat + 16 * lane, a.flat + off, bytes);
    if (a.mask && lane < 8) {
        const int mx = cb + 16 * lane;
        const bool min_ = mx < a.W;
        const int mb = min_ ? ((a.W - mx >= 16) ? 16 : (a.W - mx)) : 0;
        cpa16(slot + sl.off_mask + 16 * lane, a.mask + (size_t)io * a.ld + (min_ ? mx : 0), mb);
    }
}

// The window columns 4l + 4 - h .. 4l + 7 + h of a staged R row (4 + 2h floats)
template <int MK>
__device__ __forceinline__ void read_window(const float *Rs, int lane, float (&w)[4 + 2 * (MK / 2)]) {
    constexpr int h = MK / 2;
    const float4 c = *reinterpret_cast<const float4 *>(Rs + 4 * lane + 4);
    if constexpr (h == 0) {
        w[0] = c.x; w[1] = c.y; w[2] = c.z; w[3] = c.w;
    } else if constexpr (h == 1) {
        w[0] = Rs[4 * lane + 3];
        w[1] = c.x; w[2] = c.y; w[3] = c.z; w[4] = c.w;
        w[5] = Rs[4 * lane + 8];
    } else {
        const float2 l2 = *reinterpret_cast<const float2 *>(Rs + 4 * lane + 2);
        const float2 r2 = *reinterpret_cast<const float2 *>(Rs + 4 * lane + 8);
        w[0] = l2.x; w[1] = l2.y;
        w[2] = c.x; w[3] = c.y; w[4] = c.z; w[5] = c.w;
        w[6] = r2.x; w[7] = r2.y;
    }
}

template <int MK>
__global__ void __launch_bounds__(kSNT, 2) eval_small_kernel(const EvalArgs a, const SmallGeom g) {
    if (a.done_flag != nullptr && *((volatile const int *)a.done_flag) != 0) return;
    constexpr int h = MK / 2, NWIN = 4 + 2 * h, NK = MK * MK;
    // per-lane float32 sums: dK (NK), then loss, dB0, count, kR^2, kappa
    constexpr int NS = NK + 5, NF = Halving<NS>::H5;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    SlotLayout sl;
    sl.off_I = 136 * 4;
    sl.off_var = sl.off_I + 512;
    sl.off_flat = sl.off_var + (a.var ? 512 : 0);
    sl.off_mask = sl.off_flat + (a.flat ? 512 : 0);
    sl.bytes = slot_bytes(a.mask != nullptr, a.var != nullptr, a.flat != nullptr);
    unsigned char *ring = smem + (size_t)warp * kSDepth * sl.bytes;

    // kernel rows in shared memory (read back as warp-uniform float4
    // broadcasts, 8 floats per row) after the warps' rings; constant background
    float *Ks = reinterpret_cast<float *>(smem + (size_t)kSW * kSDepth * sl.bytes);
    for (int i = tid; i < MK * 8; i += kSNT) {
        const int aa = i / 8, b = i % 8;
        Ks[i] = b < MK ? a.Kpad[aa * g.kp + b] : 0.f;
    }
    const float B0 = a.Kpad[MK * g.kp];
    __syncthreads();

    int kidx[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) kidx[j] = halving_index<NS>(lane, j);
    double acc[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) acc[j] = 0.0;

    const int gw = blockIdx.x * kSW + warp, tw = gridDim.x * kSW;
    for (int s = gw; s < g.n_strips; s += tw) {
        const int cb = (s % g.col_blocks) * kSColBlock;
        const int i0 = h + (s / g.col_blocks) * g.band_rows;
        const int i1 = min(i0 + g.band_rows, a.H - h);
        const int T = (i1 - i0) + 2 * h;     // slots of this strip
        // columns of this lane in the valid region
        const int j0 = cb + 4 * lane;
        float s32[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) s32[k] = 0.f;

        __syncwarp();   // the previous strip's last reads of the ring are done
#pragma unroll 1
        for (int t = 0; t < kSDepth; ++t) {
            if (t < T) stage_slot<MK>(ring + t * sl.bytes, sl, a, cb, i0, i1, t, lane);
            cpa_commit();
        }
        float win[MK][NWIN];
#pragma unroll
        for (int r = 0; r < MK; ++r)
#pragma unroll
            for (int c = 0; c < NWIN; ++c) win[r][c] = 0.f;

#pragma unroll 1
        for (int t0 = 0; t0 < T; t0 += MK) {
#pragma unroll
            for (int u = 0; u < MK; ++u) {
                const int t = t0 + u;
                if (t < T) {
                    cpa_wait_depth();
                    __syncwarp();
                    unsigned char *slot = ring + (t % kSDepth) * sl.bytes;
                    read_window<MK>(reinterpret_cast<const float *>(slot), lane, win[u]);
                    float Iv[4], Vv[4], Fv[4];
                    uint32_t mk4 = 0xffffffffu;
                    const bool row_out = t >= 2 * h;
                    if (row_out) {
                        const float4 i4 = *reinterpret_cast<const float4 *>(slot + sl.off_I + 16 * lane);
                        Iv[0] = i4.x; Iv[1] = i4.y; Iv[2] = i4.z; Iv[3] = i4.w;
                        if (a.var) {
                            const float4 v4 = *reinterpret_cast<const float4 *>(slot + sl.off_var + 16 * lane);
                            Vv[0] = v4.x; Vv[1] = v4.y; Vv[2] = v4.z; Vv[3] = v4.w;
                        }
                        if (a.flat) {
                            const float4 f4 = *reinterpret_cast<const float4 *>(slot + sl.off_flat + 16 * lane);
                            Fv[0] = f4.x; Fv[1] = f4.y; Fv[2] = f4.z; Fv[3] = f4.w;
                        }
                        if (a.mask) mk4 = *reinterpret_cast<const uint32_t *>(slot + sl.off_mask + 4 * lane);
                    }
                    __syncwarp();   // every lane has read slot t
                    if (t + kSDepth < T)
                        stage_slot<MK>(slot, sl, a, cb, i0, i1, t + kSDepth, lane);
                    cpa_commit();
                    if (row_out) {
                        // window rows a = 0..MK-1 of this output row sit in ring
                        // slots (u + 1 + a) % MK (the newest row in slot u)
                        // two partial sums per pixel (even / odd kernel rows)
                        // so the forward has eight independent FMA chains
                        float M[4], M2[4];
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            M[p] = B0;
                            M2[p] = 0.f;
                        }
#pragma unroll
                        for (int aa = 0; aa < MK; ++aa) {
                            const int rs = (u + 1 + aa) % MK;
                            float kk[8];
                            const float4 k0 = *reinterpret_cast<const float4 *>(Ks + 8 * aa);
                            kk[0] = k0.x; kk[1] = k0.y; kk[2] = k0.z; kk[3] = k0.w;
                            if (MK > 4) {
                                const float4 k1 = *reinterpret_cast<const float4 *>(Ks + 8 * aa + 4);
                                kk[4] = k1.x; kk[5] = k1.y; kk[6] = k1.z; kk[7] = k1.w;
                            }
#pragma unroll
                            for (int b = 0; b < MK; ++b)
#pragma unroll
                                for (int p = 0; p < 4; ++p) {
                                    if (aa & 1)
                                        M2[p] = fmaf(kk[b], win[rs][p + b], M2[p]);
                                    else
                                        M[p] = fmaf(kk[b], win[rs][p + b], M[p]);
                                }
                        }
#pragma unroll
                        for (int p = 0; p < 4; ++p) M[p] += M2[p];
                        float gp[4];
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const int j = j0 + p;
                            const bool use = j >= h && j < a.W - h && ((mk4 >> (8 * p)) & 0xffu) != 0;
                            float gv = 0.f;
                            if (use) {
                                float z, kap;
                                const float ell = pixel_loss(a.lp, Iv[p], M[p],
                                                             a.var ? Vv[p] : a.lp.var_scalar,
                                                             a.flat ? Fv[p] : 1.0f, gv, z, kap);
                                const float rc = win[(u + 1 + h) % MK][p + h];
                                s32[NK] += ell;
                                s32[NK + 1] += gv;
                                s32[NK + 2] += 1.f;
                                s32[NK + 3] = fmaf(kap * rc, rc, s32[NK + 3]);
                                s32[NK + 4] += kap;
                            }
                            gp[p] = gv;
                        }
#pragma unroll
                        for (int aa = 0; aa < MK; ++aa) {
                            const int rs = (u + 1 + aa) % MK;
#pragma unroll
                            for (int b = 0; b < MK; ++b)
#pragma unroll
                                for (int p = 0; p < 4; ++p)
                                    s32[aa * MK + b] = fmaf(gp[p], win[rs][p + b], s32[aa * MK + b]);
                        }
                    }
                }
            }
        }
        cpa_wait_all();
        // warp sums of this strip, float64 per lane
        {
            using Hv = Halving<NS>;
            float w1[Hv::H1], w2[Hv::H2], w3[Hv::H3], w4[Hv::H4], w5[Hv::H5];
            halve<NS, 16>(s32, w1, lane & 16);
            halve<Hv::H1, 8>(w1, w2, lane & 8);
            halve<Hv::H2, 4>(w2, w3, lane & 4);
            halve<Hv::H3, 2>(w3, w4, lane & 2);
            halve<Hv::H4, 1>(w4, w5, lane & 1);
#pragma unroll
            for (int j = 0; j < NF; ++j) acc[j] += (double)w5[j];
        }
    }

    // CTA sum in a fixed order (warp 0, 1, ...), then the per-CTA partials in
    // the layout of the tiled kernel
    __syncthreads();
    double *red = reinterpret_cast<double *>(smem);   // kSW x NS (the rings are done)
#pragma unroll
    for (int j = 0; j < NF; ++j)
        if (kidx[j] >= 0) red[warp * NS + kidx[j]] = acc[j];
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * g.np;
    for (int k = tid; k < g.np; k += kSNT) {
        // k: 0 loss, 1..NK dK, NK+1 dB0, NK+2..NK+kBgMax other background slots (0),
        // red_count pixel count, +1 kR^2, +2 kappa
        int src = -1;
        if (k == 0) src = NK;
        else if (k <= NK) src = k - 1;
        else if (k == NK + 1) src = NK + 1;
        else if (k == red_count(NK)) src = NK + 2;
        else if (k == red_count(NK) + 1) src = NK + 3;
        else if (k == red_count(NK) + 2) src = NK + 4;
        double v = 0.0;
        if (src >= 0)
            for (int w = 0; w < kSW; ++w) v += red[w * NS + src];
        out[k] = v;
    }
}

template <int MK>
const void *small_fn() {
    return (const void *)&eval_small_kernel<MK>;
}

}  // namespace

bool small_kernel_ok(const EvalArgs &a, int mk) {
    if (mk != 1 && mk != 3 && mk != 5) return false;
    if (a.bg_deg != 0 || a.acc32) return false;
    // every 16-byte cp.async source must be aligned: 16-byte bases, rows a
    // multiple of 16 bytes (of 4 floats; of 16 mask bytes)
    auto al = [](const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    if (!al(a.R) || !al(a.I) || !al(a.var) || !al(a.flat) || !al(a.mask)) return false;
    if (a.ld % 4 != 0) return false;
    if (a.mask && a.ld % 16 != 0) return false;
    return true;
}

int small_kernel_smem(const EvalArgs &a) {
    return kSW * kSDepth * slot_bytes(a.mask != nullptr, a.var != nullptr, a.flat != nullptr) +
           5 * 8 * 4;   // + the kernel rows
}

cudaError_t small_kernel_prepare(const EvalArgs &a, int mk, int *occ) {
    const void *fn = mk == 1 ? small_fn<1>() : mk == 3 ? small_fn<3>() : small_fn<5>();
    const int smem = small_kernel_smem(a);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fn, kSNT, smem);
}

SmallGeom small_geometry(const EvalArgs &a, int mk, int kp, int np, int grid) {
    SmallGeom g;
    const int h = mk / 2, Hv = a.H - 2 * h;
    g.kp = kp;
    g.np = np;
    g.col_blocks = (a.W + kSColBlock - 1) / kSColBlock;
    const long long warps = (long long)grid * kSW;
    long long bands = warps / g.col_blocks;
    if (bands < 1) bands = 1;
    // at most 1024 rows per strip: each lane's float32 sums cover <= 4096 px
    if (bands < (Hv + 1023) / 1024) bands = (Hv + 1023) / 1024;
    if (bands > Hv) bands = Hv;
    g.band_rows = (int)((Hv + bands - 1) / bands);
    const int nb = (Hv + g.band_rows - 1) / g.band_rows;
    g.n_strips = g.col_blocks * nb;
    return g;
}

cudaError_t launch_eval_small(const EvalArgs &a, int mk, int kp, int np, int grid,
                              cudaStream_t s) {
    const SmallGeom g = small_geometry(a, mk, kp, np, grid);
    const int smem = small_kernel_smem(a);
    const void *fn = mk == 1 ? small_fn<1>() : mk == 3 ? small_fn<3>() : small_fn<5>();
    void *params[] = {(void *)&a, (void *)&g};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSNT), params, smem, s);
}

}  // namespace dia

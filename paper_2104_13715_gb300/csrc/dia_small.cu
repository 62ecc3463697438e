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
//   * sums: float32 per lane over one strip (<= 64 rows, <= 256 pixels; for
//     m <= 3 in two levels, per m-row chunk then per strip), then a float64
//     halving butterfly over the warp and float64 per lane across strips; one
//     CTA-wide float64 sum at the end gives the same per-CTA partials as the
//     tiled kernel (loss, dK, dB0, pixel count, curvature sums), reduced by the
//     same fixed-order kernel.
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
// the same, issued only where `pred` holds (a predicated instruction, no branch)
__device__ __forceinline__ void cpa16_if(void *dst, const void *src, int bytes, bool pred) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
                 "@p cp.async.cg.shared.global [%0], [%1], 16, %2;\n\t}\n"
                 ::"r"(d), "l"(src), "r"(bytes), "r"((int)pred));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cpa_wait_depth() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kSDepth - 1));
}
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// The halving warp reduction of dia_eval.cuh on float64 values.
template <int N, int O>
__device__ __forceinline__ void halve_d(const double *v, double *w, bool up) {
    constexpr int H = (N + 1) / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const double lo = v[i];
        const double hi = (i + H < N) ? v[i + H] : 0.0;
        const double keep = up ? hi : lo;
        const double send = up ? lo : hi;
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

struct SlotLayout {
    int off_I, off_var, off_flat, off_mask, bytes;
};

// Per-lane copy plan of one strip (row independent): the R chunk of the
// lane's own columns (chunk lane + 1 of the slot's 34) and, for lanes 0 and
// 1, the halo chunks 0 and 33; the target-side chunk (columns cb + 4 lane)
// and, for lanes 0-7, a 16-byte mask chunk.  Byte counts below 16 zero-fill.
struct StripCopy {
    int rx1, rb1;   // R column and bytes of chunk lane + 1
    int rc2, rx2, rb2;   // chunk index (0 or 33), column and bytes (lanes 0, 1)
    int ix, ib;     // target-side column and bytes
    int mx, mb;     // mask column and bytes (lanes 0-7)
};

__device__ __forceinline__ StripCopy strip_copy(const EvalArgs &a, int cb, int lane) {
    StripCopy c;
    c.rx1 = cb + 4 * lane;
    c.rb1 = (c.rx1 < a.W) ? ((a.W - c.rx1 >= 4) ? 16 : 4 * (a.W - c.rx1)) : 0;
    if (c.rb1 == 0) c.rx1 = 0;
    c.rc2 = lane == 0 ? 0 : 33;
    c.rx2 = cb - 4 + 4 * c.rc2;
    c.rb2 = (lane < 2 && c.rx2 >= 0 && c.rx2 < a.W) ? ((a.W - c.rx2 >= 4) ? 16 : 4 * (a.W - c.rx2)) : 0;
    if (c.rb2 == 0) c.rx2 = 0;
    c.ix = c.rx1;
    c.ib = c.rb1;
    c.mx = cb + 16 * lane;
    c.mb = (lane < 8 && c.mx < a.W) ? ((a.W - c.mx >= 16) ? 16 : (a.W - c.mx)) : 0;
    if (c.mb == 0) c.mx = 0;
    return c;
}

// Running source pointers of one strip's staging: the next R row to stage
// (chunk lane + 1 and the halo chunk of lanes 0, 1) and the next target-side
// row (advanced by one row pitch per staged slot).
struct StripPtr {
    const float *r1, *r2, *ti, *tv, *tf;
    const uint8_t *tm;
};

// Stage the next slot (R row i0 - h + t, and the target-side rows of output
// row i0 + t - 2h once t >= 2h) into `slot` and advance the pointers.
template <int MK, int FAST>
__device__ __forceinline__ void stage_next(unsigned char *slot, const SlotLayout &sl,
                                           const StripCopy &cp, StripPtr &sp, size_t ld, int t,
                                           int lane, bool hv, bool hf, bool hm) {
    constexpr int h = MK / 2;
    float *Rs = reinterpret_cast<float *>(slot);
    cpa16(Rs + 4 * (lane + 1), sp.r1, cp.rb1);
    cpa16_if(Rs + 4 * cp.rc2, sp.r2, cp.rb2, lane < 2);
    sp.r1 += ld;
    sp.r2 += ld;
    if (t < 2 * h) return;                              // no output row yet
    cpa16(slot + sl.off_I + 16 * lane, sp.ti, cp.ib);
    sp.ti += ld;
    if (!FAST && hv) {
        cpa16(slot + sl.off_var + 16 * lane, sp.tv, cp.ib);
        sp.tv += ld;
    }
    if (!FAST && hf) {
        cpa16(slot + sl.off_flat + 16 * lane, sp.tf, cp.ib);
        sp.tf += ld;
    }
    if (hm) {
        cpa16_if(slot + sl.off_mask + 16 * lane, sp.tm, cp.mb, lane < 8);
        sp.tm += ld;
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

// FAST = 1: the Gaussian loss with a fixed scalar variance (the chi^2 of the
// memory-bound workloads): a branch-free epilogue with the mask folded into a
// per-pixel weight w in {0, 1}: z = (I - M)/s, sum w z^2 (loss = half of it),
// g = -w z / s, count, and sum w R^2 (the curvature sums are 1/v times
// these).  FAST = 0: any loss and variance model through pixel_loss.
// HM: a mask is given.
template <int MK, int FAST, int HM>
__global__ void __launch_bounds__(kSNT, MK <= 1 ? 3 : 2) eval_small_kernel(const EvalArgs a,
                                                                          const SmallGeom g) {
    if (a.done_flag != nullptr && *((volatile const int *)a.done_flag) != 0) return;
    constexpr int h = MK / 2, NWIN = 4 + 2 * h, NK = MK * MK;
    // per-lane float32 sums: dK (NK), then loss, dB0, count, kR^2, kappa
    constexpr int NS = NK + 5, NF = Halving<NS>::H5;
    constexpr bool KREG = MK <= 3;   // kernel taps in registers (else shared memory)
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
    float kreg[KREG ? NK : 1];
    if constexpr (KREG) {
#pragma unroll
        for (int i = 0; i < NK; ++i) kreg[i] = Ks[(i / MK) * 8 + i % MK];
    }

    int kidx[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) kidx[j] = halving_index<NS>(lane, j);
    double acc[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) acc[j] = 0.0;

    // a fixed scalar variance: its reciprocal and root once per thread
    const bool scalar_var = a.lp.var_model == 0 && a.var == nullptr;
    const float sv_inv_v = 1.0f / a.lp.var_scalar;
    const float sv_inv_s = sqrtf(sv_inv_v);

    const int gw = blockIdx.x * kSW + warp, tw = gridDim.x * kSW;
    for (int s = gw; s < g.n_strips; s += tw) {
        const int cb = (s % g.col_blocks) * kSColBlock;
        const int i0 = h + (s / g.col_blocks) * g.band_rows;
        const int i1 = min(i0 + g.band_rows, a.H - h);
        const int T = (i1 - i0) + 2 * h;     // slots of this strip
        const StripCopy cp = strip_copy(a, cb, lane);
        const size_t ld = (size_t)a.ld;
        StripPtr sp;
        sp.r1 = a.R + (size_t)(i0 - h) * ld + cp.rx1;
        sp.r2 = a.R + (size_t)(i0 - h) * ld + cp.rx2;
        sp.ti = a.I + (size_t)i0 * ld + cp.ix;
        sp.tv = a.var ? a.var + (size_t)i0 * ld + cp.ix : nullptr;
        sp.tf = a.flat ? a.flat + (size_t)i0 * ld + cp.ix : nullptr;
        sp.tm = HM ? a.mask + (size_t)i0 * ld + cp.mx : nullptr;
        const bool hv = a.var != nullptr, hf = a.flat != nullptr;
        // valid-region columns of this lane's four pixels (1) or not (0)
        float vcol[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int j = cb + 4 * lane + p;
            vcol[p] = (j >= h && j < a.W - h) ? 1.f : 0.f;
        }
        // float32 sums over the strip (<= 64 rows): dK first, then loss, dB0,
        // count, kR^2, kappa; for m <= 3 two-level (`in` over one chunk of MK
        // rows, then `out`), for m = 5 directly into `out` (registers)
        constexpr bool TWO = MK <= 3;
        float out[NS], inb[TWO ? NS : 1];
#pragma unroll
        for (int k = 0; k < NS; ++k) out[k] = 0.f;
#pragma unroll
        for (int k = 0; k < (TWO ? NS : 1); ++k) inb[k] = 0.f;
        float *const in = TWO ? inb : out;

        __syncwarp();   // the previous strip's last reads of the ring are done
        unsigned char *slot_st = ring;   // next slot to fill
#pragma unroll 1
        for (int t = 0; t < kSDepth; ++t) {
            if (t < T) stage_next<MK, FAST>(slot_st, sl, cp, sp, ld, t, lane, hv, hf, HM);
            cpa_commit();
            slot_st += sl.bytes;
        }
        unsigned char *slot = ring;      // slot of row t (refilled with row t + D)
        unsigned char *const ring_end = ring + kSDepth * sl.bytes;
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
                    read_window<MK>(reinterpret_cast<const float *>(slot), lane, win[u]);
                    float Iv[4], Vv[4], Fv[4];
                    uint32_t mk4 = 0xffffffffu;
                    const bool row_out = t >= 2 * h;
                    if (row_out) {
                        const float4 i4 = *reinterpret_cast<const float4 *>(slot + sl.off_I + 16 * lane);
                        Iv[0] = i4.x; Iv[1] = i4.y; Iv[2] = i4.z; Iv[3] = i4.w;
                        if (!FAST && hv) {
                            const float4 v4 = *reinterpret_cast<const float4 *>(slot + sl.off_var + 16 * lane);
                            Vv[0] = v4.x; Vv[1] = v4.y; Vv[2] = v4.z; Vv[3] = v4.w;
                        }
                        if (!FAST && hf) {
                            const float4 f4 = *reinterpret_cast<const float4 *>(slot + sl.off_flat + 16 * lane);
                            Fv[0] = f4.x; Fv[1] = f4.y; Fv[2] = f4.z; Fv[3] = f4.w;
                        }
                        if (HM) mk4 = *reinterpret_cast<const uint32_t *>(slot + sl.off_mask + 4 * lane);
                    }
                    __syncwarp();   // every lane has read slot t
                    if (t + kSDepth < T) stage_next<MK, FAST>(slot, sl, cp, sp, ld, t + kSDepth, lane, hv, hf, HM);
                    cpa_commit();
                    slot += sl.bytes;
                    if (slot == ring_end) slot = ring;
                    if (row_out) {
                        // window rows a = 0..MK-1 of this output row sit in ring
                        // slots (u + 1 + a) % MK (the newest row in slot u); for
                        // m = 5 two partial sums per pixel (even / odd kernel
                        // rows) give eight independent FMA chains
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
                            if constexpr (KREG) {
#pragma unroll
                                for (int b = 0; b < MK; ++b) kk[b] = kreg[aa * MK + b];
                            } else {
                                const float4 k0 = *reinterpret_cast<const float4 *>(Ks + 8 * aa);
                                const float4 k1 = *reinterpret_cast<const float4 *>(Ks + 8 * aa + 4);
                                kk[0] = k0.x; kk[1] = k0.y; kk[2] = k0.z; kk[3] = k0.w;
                                kk[4] = k1.x; kk[5] = k1.y; kk[6] = k1.z; kk[7] = k1.w;
                            }
#pragma unroll
                            for (int b = 0; b < MK; ++b)
#pragma unroll
                                for (int p = 0; p < 4; ++p) {
                                    if (MK > 3 && (aa & 1))
                                        M2[p] = fmaf(kk[b], win[rs][p + b], M2[p]);
                                    else
                                        M[p] = fmaf(kk[b], win[rs][p + b], M[p]);
                                }
                        }
                        if (MK > 3) {
#pragma unroll
                            for (int p = 0; p < 4; ++p) M[p] += M2[p];
                        }
                        float gp[4];
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float rc = win[(u + 1 + h) % MK][p + h];
                            float w = vcol[p];
                            if (HM) w = ((mk4 >> (8 * p)) & 0xffu) ? w : 0.f;
                            if constexpr (FAST != 0) {
                                const float z = (Iv[p] - M[p]) * sv_inv_s;
                                const float zw = z * w;
                                in[NK] = fmaf(zw, z, in[NK]);
                                gp[p] = zw * -sv_inv_s;
                                in[NK + 1] += gp[p];
                                in[NK + 2] += w;
                                in[NK + 3] = fmaf(w * rc, rc, in[NK + 3]);
                            } else {
                                float gv = 0.f;
                                if (w != 0.f) {
                                    float z, kap;
                                    const float ell =
                                        scalar_var
                                            ? pixel_loss_fixed(a.lp, sv_inv_v, sv_inv_s, Iv[p], M[p], gv, z, kap)
                                            : pixel_loss(a.lp, Iv[p], M[p], hv ? Vv[p] : a.lp.var_scalar,
                                                         hf ? Fv[p] : 1.0f, gv, z, kap);
                                    in[NK] += ell;
                                    in[NK + 1] += gv;
                                    in[NK + 2] += 1.f;
                                    in[NK + 3] = fmaf(kap * rc, rc, in[NK + 3]);
                                    in[NK + 4] += kap;
                                }
                                gp[p] = gv;
                            }
                        }
#pragma unroll
                        for (int aa = 0; aa < MK; ++aa) {
                            const int rs = (u + 1 + aa) % MK;
#pragma unroll
                            for (int b = 0; b < MK; ++b)
#pragma unroll
                                for (int p = 0; p < 4; ++p)
                                    in[aa * MK + b] = fmaf(gp[p], win[rs][p + b], in[aa * MK + b]);
                        }
                    }
                }
            }
            // end of a chunk of MK rows: into the strip sums
            if constexpr (TWO) {
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    out[k] += inb[k];
                    inb[k] = 0.f;
                }
            }
        }
        cpa_wait_all();
        // warp sums of this strip in float64 (halving butterfly), per lane
        {
            if constexpr (FAST != 0) {
                // loss = sum w z^2 / 2; curvature weight 1/v per used pixel
                out[NK] *= 0.5f;
                out[NK + 3] *= sv_inv_v;
                out[NK + 4] = out[NK + 2] * sv_inv_v;
            }
            double d0[NS];
#pragma unroll
            for (int k = 0; k < NS; ++k) d0[k] = (double)out[k];
            using Hv = Halving<NS>;
            double w1[Hv::H1], w2[Hv::H2], w3[Hv::H3], w4[Hv::H4], w5[Hv::H5];
            halve_d<NS, 16>(d0, w1, lane & 16);
            halve_d<Hv::H1, 8>(w1, w2, lane & 8);
            halve_d<Hv::H2, 4>(w2, w3, lane & 4);
            halve_d<Hv::H3, 2>(w3, w4, lane & 2);
            halve_d<Hv::H4, 1>(w4, w5, lane & 1);
#pragma unroll
            for (int j = 0; j < NF; ++j) acc[j] += w5[j];
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
const void *small_fn(int fast, int hm) {
    if (fast) return hm ? (const void *)&eval_small_kernel<MK, 1, 1> : (const void *)&eval_small_kernel<MK, 1, 0>;
    return hm ? (const void *)&eval_small_kernel<MK, 0, 1> : (const void *)&eval_small_kernel<MK, 0, 0>;
}

// the kernel instance for these arguments
const void *small_pick(const EvalArgs &a, int mk) {
    const int fast = a.lp.rho == 0 && a.lp.var_model == 0 && a.var == nullptr;
    const int hm = a.mask != nullptr;
    return mk == 1 ? small_fn<1>(fast, hm) : mk == 3 ? small_fn<3>(fast, hm) : small_fn<5>(fast, hm);
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
    const void *fn = small_pick(a, mk);
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
    // at most 64 rows per strip: each lane's float32 sums cover <= 256 px
    if (bands < (Hv + 63) / 64) bands = (Hv + 63) / 64;
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
    const void *fn = small_pick(a, mk);
    void *params[] = {(void *)&a, (void *)&g};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kSNT), params, smem, s);
}

}  // namespace dia

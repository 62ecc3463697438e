// Tensor-core form of the weight gradient (the correlation of dl/dM with R,
// Sec. 2.3) and of the evaluation built on it, for sm_103a.
//
// With g = dl/dM over the valid region (0 where masked), for an output tile
// of 64 rows (i) x 128 columns (j) at valid-region pixel (y0, x0) and its R
// window W[y][x] = R[y0 + y][x0 + x] (full-image coordinates, 96 x 160):
//   dL/dK[a][b] = sum_{i,j} g[y0+i][x0+j] W[i+a][j+b] = sum_i P_b[i+a][i],
//   P_b[y][i]   = sum_j W[y][j+b] g[i][j],
// one GEMM per kernel column b (M = window row y, N = tile row i, K = tile
// column j) followed by sums along the diagonals y - i = a.  The window is
// stored in 8-row chunks, T[y/8][x][y%8], so A_b = W[.][. + b] is an MN-major
// operand whose start moves by b * 16 bytes (no copy per b), exactly the
// layout of the forward pass's window; the g tile is a K-major operand.
// M = 128 rows are multiplied, of which the first 64 + m - 1 hold window rows
// (the rest read the other split's data and are ignored).
//
// Precision: g and R are scaled by powers of two (per launch, from their
// largest magnitudes) into the range of float16 and split x = hi + lo in
// float16 (22 significant bits together); the products hi*hi + hi*lo + lo*hi
// are accumulated in float32 in tensor memory (the dropped lo*lo term and the
// split leave about 2^-21 of each product), then the diagonal sums in float32
// per tile and float64 across tiles.
//
// Per tile: the producer warps stage both operands in shared memory; the MMA
// warp issues the products for up to 8 kernel columns at a time into 8 x 64
// tensor-memory columns; the producer warps holding window rows (lanes
// y < 64 + m - 1) read them back and add each value to the diagonal it lies
// on (shared-memory atomics, one accumulator set per warp, so the sums do not
// depend on timing).  Every wait is bounded.
#include <cuda_fp16.h>
#include <cstdint>
#include <cstring>

#include "../../include/dia.h"
#include "dia_ops.cuh"
#include "dia_tc_ptx.cuh"
#include "dia_tc_grad.h"

namespace dia {

namespace {

constexpr int kGI = 64;             // tile rows (MMA N)
constexpr int kGJ = 128;            // tile columns (MMA K)
constexpr int kGXT = kGJ + 32;      // window columns (m <= 33)
constexpr int kGYC = 12;            // 8-row chunks of the window: 96 >= 64 + m - 1
constexpr int kGB = 8;              // kernel columns per round (8 x 64 TMEM columns)
constexpr int kGMaxM = 31;
constexpr int kGProd = 128;         // warps 0-3
constexpr int kGThreads = kGProd + 32;
constexpr int kGDiagWarps = 3;      // warps whose TMEM lanes hold window rows (< 96)

struct GradSmem {
    __half t[2][kGYC][kGXT][8];            // window [hi|lo][y/8][x][y%8]
    __half g[2][kGI / 8][kGJ / 8][8][8];   // g tile [hi|lo][i/8][j/8][i%8][j%8]
    float s32[kGDiagWarps][kGMaxM][kGMaxM];   // per-warp float32 diagonal sums of a tile [b][a]
    double s64[kGDiagWarps][kGMaxM][kGMaxM];  // per-warp float64 totals [b][a]
    uint64_t mb;                           // a round of MMAs completed
    uint32_t tslot;
};

// 2^e with |x| 2^e in [2^13, 2^14) for the largest magnitude x (1 if x == 0)
__device__ __forceinline__ float pow2_scale(float amax) {
    if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
    int e;
    frexpf(amax, &e);   // amax = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, 14 - e);
}

__device__ __forceinline__ void split_f16(float x, __half &hi, __half &lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

struct GradArgs {
    const float *R;
    int H, W, ld, m;
    const float *G;        // valid-region g map (Hv x Wv, pitch Wv), 0 where masked
    int Hv, Wv, tiles_x, n_tiles;
    const unsigned *amax;  // [0] max |R| bits, [1] max |g| bits
    double *partials;      // per CTA: np doubles (dK at 1 .. m*m, the rest 0)
    int np;
    int *status;           // set to 1 if a wait ran out
};

__global__ void __launch_bounds__(kGThreads, 1) tc_grad_kernel(const GradArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    GradSmem &S = *reinterpret_cast<GradSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m;
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(su32(&S.tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&S.mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int i = tid; i < kGDiagWarps * kGMaxM * kGMaxM; i += kGThreads) {
        (&S.s32[0][0][0])[i] = 0.f;
        (&S.s64[0][0][0])[i] = 0.0;
    }
    const float sR = pow2_scale(__uint_as_float(a.amax[0]));
    const float sG = pow2_scale(__uint_as_float(a.amax[1]));
    const float unscale = 1.f / (sR * sG);   // an exact power of two
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = S.tslot;
    const int never = 0;
    bool fail = false;
    uint32_t phase = 0;   // parity of the next round's completion
    const int n_rounds = (m + kGB - 1) / kGB;

    for (int tile = blockIdx.x; tile < a.n_tiles && !fail; tile += gridDim.x) {
        const int y0 = (tile / a.tiles_x) * kGI, x0 = (tile % a.tiles_x) * kGJ;
        if (tid < kGProd) {
            // window: chunk (yc, x) = 8 rows of column x, scaled and split
            for (int c = tid; c < kGYC * kGXT; c += kGProd) {
                const int yc = c / kGXT, x = c % kGXT;
                const int gx = x0 + x;
                __align__(16) __half hi[8], lo[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int gy = y0 + 8 * yc + e;
                    const float v = (gy < a.H && gx < a.W) ? __ldg(a.R + (size_t)gy * a.ld + gx) : 0.f;
                    split_f16(v * sR, hi[e], lo[e]);
                }
                *reinterpret_cast<uint4 *>(&S.t[0][yc][x][0]) = *reinterpret_cast<const uint4 *>(hi);
                *reinterpret_cast<uint4 *>(&S.t[1][yc][x][0]) = *reinterpret_cast<const uint4 *>(lo);
            }
            // g tile: chunk (i, jb) = 8 consecutive columns of row i
            for (int c = tid; c < kGI * (kGJ / 8); c += kGProd) {
                const int i = c / (kGJ / 8), jb = c % (kGJ / 8);
                const int yv = y0 + i;
                __align__(16) __half hi[8], lo[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int xv = x0 + 8 * jb + e;
                    const float v = (yv < a.Hv && xv < a.Wv) ? __ldg(a.G + (size_t)yv * a.Wv + xv) : 0.f;
                    split_f16(v * sG, hi[e], lo[e]);
                }
                *reinterpret_cast<uint4 *>(&S.g[0][i / 8][jb][i % 8][0]) = *reinterpret_cast<const uint4 *>(hi);
                *reinterpret_cast<uint4 *>(&S.g[1][i / 8][jb][i % 8][0]) = *reinterpret_cast<const uint4 *>(lo);
            }
            asm volatile("fence.proxy.async.shared::cta;");
        }
        __syncthreads();   // operands staged; the previous tile's sums are flushed

        for (int r = 0; r < n_rounds; ++r) {
            const int b0 = r * kGB, nb = min(kGB, m - b0);
            if (warp == 4) {
                if (lane == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    // A_b: window [split][.][x][.], MN-major: K step (8 columns) = 128 B,
                    // M step (8 rows) = kGXT * 16 B; B: g tile K-major: K step 128 B,
                    // N step (8 rows) = (kGJ / 8) * 128 B
                    const uint32_t idesc = tc_idesc(128, kGI, 1, 0, 1);
                    constexpr uint32_t kTs = sizeof(S.t[0]), kGs = sizeof(S.g[0]);
                    const uint32_t t0a = su32(&S.t[0][0][0][0]), g0a = su32(&S.g[0][0][0][0][0]);
                    for (int bb = 0; bb < nb; ++bb) {
                        const int b = b0 + bb;
                        const uint32_t acc = tmem + (uint32_t)(bb * kGI);
                        for (int ks = 0; ks < kGJ / 16; ++ks) {
                            const uint32_t ta = t0a + (uint32_t)(b * 16 + ks * 256);
                            const uint32_t ga = g0a + (uint32_t)(ks * 256);
                            const uint64_t ahi = tc_desc(ta, 128, kGXT * 16);
                            const uint64_t alo = tc_desc(ta + kTs, 128, kGXT * 16);
                            const uint64_t bhi = tc_desc(ga, 128, (kGJ / 8) * 128);
                            const uint64_t blo = tc_desc(ga + kGs, 128, (kGJ / 8) * 128);
                            tc_mma(acc, ahi, bhi, idesc, ks > 0 ? 1 : 0);
                            tc_mma(acc, ahi, blo, idesc, 1);
                            tc_mma(acc, alo, bhi, idesc, 1);
                        }
                    }
                    tc_commit(&S.mb);
                }
                __syncwarp();
            }
            // every thread waits for the round's products (the MMA warp too, so
            // that no MMA is in flight when the tile's operands are replaced);
            // the outcome is made the same for every thread before anyone acts
            const bool ok = tc_wait(&S.mb, phase, &never);
            fail = __syncthreads_or(!ok) != 0;
            if (fail) break;   // the MMAs of this round are drained below
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (warp < kGDiagWarps) {
                // lane y of this warp: P_b[y][i] for the round's kernel columns b
                const int y = 32 * warp + lane;
                for (int bb = 0; bb < nb; ++bb) {
                    const int b = b0 + bb;
                    float* const sw = &S.s32[warp][b][0];
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        uint32_t v[32];
                        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) +
                                            (uint32_t)(bb * kGI + 32 * half);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
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
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const int dia_a = y - (32 * half + q);   // the diagonal a = y - i
                            if (dia_a >= 0 && dia_a < m)
                                atomicAdd(sw + dia_a, __uint_as_float(v[q]) * unscale);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();   // tensor memory and the sums are free for the next round
        }
        // this tile's float32 diagonal sums into the float64 totals (each warp
        // its own set, so the order of additions is fixed)
        if (warp < kGDiagWarps) {
            float *s32 = &S.s32[warp][0][0];
            double *s64 = &S.s64[warp][0][0];
            for (int k = lane; k < kGMaxM * kGMaxM; k += 32) {
                s64[k] += (double)s32[k];
                s32[k] = 0.f;
            }
        }
        // the next tile's staging waits at its first barrier
    }
    if (fail) {
        // a round did not complete within the limit: wait once more (default
        // limit) so that no MMA still writes tensor memory when it is released
        tc_wait(&S.mb, phase, &never);
        if (tid == 0) atomicExch(a.status, 1);
    }
    __syncthreads();
    double *out = a.partials + (size_t)blockIdx.x * a.np;
    for (int k = tid; k < a.np; k += kGThreads) {
        double t = 0.0;
        if (k >= 1 && k <= m * m) {
            const int aa = (k - 1) / m, b = (k - 1) % m;
            for (int w = 0; w < kGDiagWarps; ++w) t += S.s64[w][b][aa];
        }
        out[k] = t;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// Largest magnitude of R over the image and of the g map (non-negative floats
// order like their bit patterns).
__global__ void absmax_kernel(const float *R, int H, int W, int ld, unsigned *out) {
    float mx = 0.f;
    const long long n = (long long)H * W;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / W), x = (int)(k % W);
        mx = fmaxf(mx, fabsf(__ldg(R + (size_t)y * ld + x)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(out, __float_as_uint(mx));
}

// g = dl/dM over the valid region from the difference image D = I - M of the
// tensor-core forward pass (M = I - D; the residual is D itself), 0 where
// masked; per-CTA partials of the loss, dL/dB0, pixel count and the two
// curvature sums (float32 per thread, float64 across the block); the largest
// |g| into amax[1].
constexpr int kGmThreads = 256;
__global__ void __launch_bounds__(kGmThreads) gmap_kernel(const EvalArgs a, const float *D, float *G,
                                                          double *partials, int np, int nk,
                                                          unsigned *amax) {
    const int h = (a.H - a.Hv) / 2;
    float l = 0.f, gs = 0.f, cnt = 0.f, kr = 0.f, ks = 0.f, gmx = 0.f;
    const long long n = (long long)a.Hv * a.Wv;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / a.Wv), x = (int)(k % a.Wv);
        const size_t off = (size_t)(y + h) * a.ld + (x + h);
        float gv = 0.f;
        if (a.mask == nullptr || a.mask[off] != 0) {
            const float Iv = __ldg(a.I + off);
            const float M = Iv - D[k];
            const float vm = a.var ? __ldg(a.var + off) : a.lp.var_scalar;
            const float F = a.flat ? __ldg(a.flat + off) : 1.0f;
            float g, z, kap;
            const float ell = pixel_loss(a.lp, Iv, M, vm, F, g, z, kap);
            const float rc = __ldg(a.R + off);
            l += ell;
            gs += g;
            cnt += 1.f;
            kr = fmaf(kap * rc, rc, kr);
            ks += kap;
            gv = g;
            gmx = fmaxf(gmx, fabsf(g));
        }
        G[k] = gv;
    }
    __shared__ double red[5][kGmThreads / 32];
    const float vals[5] = {l, gs, cnt, kr, ks};
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double v = (double)vals[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][w] = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gmx = fmaxf(gmx, __shfl_xor_sync(0xffffffffu, gmx, o));
    if (lane == 0 && gmx > 0.f) atomicMax(amax + 1, __float_as_uint(gmx));
    __syncthreads();
    double *out = partials + (size_t)blockIdx.x * np;
    for (int k = threadIdx.x; k < np; k += kGmThreads) {
        int q = -1;
        if (k == 0) q = 0;
        else if (k == nk + 1) q = 1;
        else if (k == red_count(nk)) q = 2;
        else if (k == red_count(nk) + 1) q = 3;
        else if (k == red_count(nk) + 2) q = 4;
        double t = 0.0;
        if (q >= 0)
            for (int ww = 0; ww < kGmThreads / 32; ++ww) t += red[q][ww];
        out[k] = t;
    }
}

}  // namespace

int tc_grad_smem_bytes() { return (int)sizeof(GradSmem); }

cudaError_t launch_tc_grad_eval(const EvalArgs &ea, int m, const float *D, float *G,
                                unsigned *amax, double *partials, int np, int sms,
                                int *status, cudaStream_t s) {
    if (m < 1 || m > kGMaxM || (m & 1) == 0) return cudaErrorInvalidValue;
    const int gm_grid = sms, gr_grid = sms;   // partial rows [0, sms) and [sms, 2 sms)
    absmax_kernel<<<sms * 4, 256, 0, s>>>(ea.R, ea.H, ea.W, ea.ld, amax);
    gmap_kernel<<<gm_grid, kGmThreads, 0, s>>>(ea, D, G, partials, np, m * m, amax);
    GradArgs a;
    a.R = ea.R;
    a.H = ea.H;
    a.W = ea.W;
    a.ld = ea.ld;
    a.m = m;
    a.G = G;
    a.Hv = ea.Hv;
    a.Wv = ea.Wv;
    a.tiles_x = (ea.Wv + kGJ - 1) / kGJ;
    a.n_tiles = a.tiles_x * ((ea.Hv + kGI - 1) / kGI);
    a.amax = amax;
    a.partials = partials + (size_t)gm_grid * np;
    a.np = np;
    a.status = status;
    const int smem = tc_grad_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(tc_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int grid = a.n_tiles < gr_grid ? a.n_tiles : gr_grid;
    tc_grad_kernel<<<grid, kGThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the grid may be smaller than its partial rows: clear the rest
    if (grid < gr_grid)
        e = cudaMemsetAsync(a.partials + (size_t)grid * np, 0, (size_t)(gr_grid - grid) * np * 8, s);
    return e;
}

}  // namespace dia

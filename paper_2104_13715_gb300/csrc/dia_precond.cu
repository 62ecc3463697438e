// Block-Toeplitz preconditioner of L-BFGS, built once per fit, and its
// application P v inside every optimiser step.
//
// For kernel pixels u = (a, b), v = (a', b') the Gauss-Newton Hessian of the
// loss, sum_p w_p R[p+u] R[p+v], is, up to the image border and the variation
// of w, the weighted autocorrelation of R at lag v - u.  Built from the
// zero-padded autocorrelation of Rt = sqrt(w) R over a window it is exactly
// the Gram matrix of the shifted copies of Rt (and of a constant, for B0),
// hence positive semidefinite; the preconditioned Hessian is well
// conditioned (condition number about 4 on a 128 x 128, m = 11 pair, against
// 2e5 with a diagonal preconditioner).
//
// Build, every launch over all pairs of a batch (blockIdx.y, or blockIdx.x
// for one-CTA-per-pair kernels):
//   rtilde      Rt over the window;
//   autocorr    one CTA per row lag dr: sum over row pairs (y, y + dr) held
//               in shared memory, every column lag at once;
//   fill        T (np x np, float64, padded with the identity), scaled by
//               the window's pixel count (the optimiser's loss is per pixel);
//   per block column K of 32: chol_diag (factor the diagonal block, invert
//               it), chol_panel (L_IK = A_IK L_KK^-T), chol_update
//               (A_IJ -= L_IK L_JK^T);
//   per block diagonal d: trtri (X_IJ = -X_II sum_T L_IT X_TJ), X = L^-1;
//   gram        P = X^T X = T^-1 (float32, symmetric).
// pc_ok is cleared when a pivot is not positive (the diagonal preconditioner
// is used instead).
#include <cmath>

#include "dia_eval.cuh"
#include "dia_ops.cuh"

namespace dia {

namespace {

constexpr int kB = kPcB;

__device__ __forceinline__ double block_sum256(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

// Weight of image pixel q (offset in the pitched image): mask / variance at M = I.
__device__ __forceinline__ float pc_weight(const PrecondArgs &a, size_t q) {
    float v;
    if (a.lp.var_model == 0) {
        v = a.var ? a.var[q] : a.lp.var_scalar;
    } else {
        const float F = a.flat ? a.flat[q] : 1.f, Iv = fmaxf(a.I[q], 0.f);
        v = a.lp.var_model == 1 ? a.lp.s0sq / (F * F) + Iv * a.lp.inv_gain / F
                                : a.lp.excess * Iv * a.lp.inv_gain / F;
        v = fmaxf(v, a.lp.var_floor);
    }
    return (a.mask && a.mask[q] == 0) ? 0.f : 1.0f / v;
}

__global__ void rtilde_kernel(const PrecondArgs *pas, int npairs) {
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int h = a.m / 2, wx = a.x1 - a.x0;
        const long long total = (long long)(a.y1 - a.y0) * wx;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
             i += (long long)gridDim.x * blockDim.x) {
            const int py = a.y0 + (int)(i / wx), px = a.x0 + (int)(i % wx);
            const size_t q = (size_t)(py + h) * a.ld + (px + h);   // pixel p + c of the image
            a.Rt[i] = sqrtf(pc_weight(a, q)) * a.R[q];
        }
    }
}

// Block dr < m: C[dr][dc + m - 1] for every dc in [-(m-1), m-1].  Thread t
// takes column lag t % L over the t / L-th chunk of the columns; row pairs are
// staged in shared memory; float32 per row, float64 across rows.
// Block dr == m: sum of Rt and sum of w over the window.
constexpr int kAcThreads = 256;
constexpr int kAcMaxW = 1024;

__global__ void __launch_bounds__(kAcThreads) autocorr_kernel(const PrecondArgs *pas, int npairs) {
    __shared__ float ra[kAcMaxW], rb[kAcMaxW];
    __shared__ double part[kAcThreads];
    __shared__ double sh[kAcThreads / 32];
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int m = a.m, h = m / 2, L = 2 * m - 1, nl = m * L;
        const int wy = a.y1 - a.y0, wx = a.x1 - a.x0;
        const int dr = blockIdx.x;
        if (dr > m) continue;
        if (dr == m) {
            double tot = 0.0, tot_w = 0.0;
            for (int y = 0; y < wy; ++y) {
                float acc = 0.f, acc_w = 0.f;
                for (int x = threadIdx.x; x < wx; x += blockDim.x) {
                    acc += a.Rt[(size_t)y * wx + x];
                    acc_w += pc_weight(a, (size_t)(a.y0 + y + h) * a.ld + (a.x0 + x + h));
                }
                tot += acc;
                tot_w += acc_w;
            }
            tot = block_sum256(tot, sh);
            tot_w = block_sum256(tot_w, sh);
            if (threadIdx.x == 0) {
                a.C[nl] = tot;
                a.C[nl + 1] = tot_w;
            }
            __syncthreads();
            continue;
        }
        const int nch = kAcThreads / L;
        const int t = threadIdx.x, li = t % L, ch = t / L;
        const int dc = li - (m - 1);
        const int xa = dc < 0 ? -dc : 0, nx = wx - (dc < 0 ? -dc : dc);
        const int per = nx > 0 ? (nx + nch - 1) / nch : 0;
        const int xb = xa + ch * per, xe = min(xa + nx, xb + per);
        double acc = 0.0;
        for (int y = 0; y + dr < wy; ++y) {
            __syncthreads();
            for (int x = t; x < wx; x += kAcThreads) {
                ra[x] = a.Rt[(size_t)y * wx + x];
                rb[x] = a.Rt[(size_t)(y + dr) * wx + x];
            }
            __syncthreads();
            if (ch < nch) {
                float s = 0.f;
                for (int x = xb; x < xe; ++x) s = fmaf(ra[x], rb[x + dc], s);
                acc += s;
            }
        }
        part[t] = (ch < nch) ? acc : 0.0;
        __syncthreads();
        if (t < L) {
            double c = 0.0;
            for (int k = 0; k < nch; ++k) c += part[k * L + t];
            a.C[dr * L + t] = c;
        }
        __syncthreads();
    }
}

// T (padded to np with the identity) into A64, X64 zeroed, pc_ok set.
__global__ void fill_kernel(const PrecondArgs *pas, int npairs) {
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int m = a.m, n = m * m + 1, np = pc_np(n), L = 2 * m - 1, nl = m * L;
        const int wy = a.y1 - a.y0, wx = a.x1 - a.x0;
        const double npx = (double)wy * wx;
        const double wbar = a.C[nl + 1] / npx;   // mean weight over the window
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)np * np;
             e += (long long)gridDim.x * blockDim.x) {
            const int u = (int)(e / np), v = (int)(e % np);
            double t;
            if (u >= n || v >= n) {
                t = (u == v) ? 1.0 : 0.0;
            } else {
                if (u == n - 1 && v == n - 1) {
                    // the constant sqrt(wbar) over the window dilated by m - 1
                    t = wbar * (double)(wy + m - 1) * (double)(wx + m - 1);
                } else if (u == n - 1 || v == n - 1) {
                    t = sqrt(wbar) * a.C[nl];
                } else {
                    int dr = v / m - u / m, dc = v % m - u % m;
                    if (dr < 0 || (dr == 0 && dc < 0)) {
                        dr = -dr;
                        dc = -dc;
                    }
                    t = a.C[dr * L + dc + (m - 1)];
                }
                if (u == v) t *= (1.0 + a.eps);
                t /= npx;
            }
            a.A64[e] = t;
            a.X64[e] = 0.0;
        }
        // P, including the pitch padding that P v reads (times zero)
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * a.ldp;
             e += (long long)gridDim.x * blockDim.x)
            a.P[e] = 0.f;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.st->pc_ok = 1;
    }
}

// 32 x 32 tile (I, J) of an np x np row-major matrix into shared memory.
__device__ __forceinline__ void load_tile(const double *M, int np, int I, int J, double (*t)[kB + 1]) {
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    t[ty][tx] = M[(size_t)(I * kB + ty) * np + J * kB + tx];
}

// Diagonal block K: Cholesky in shared memory, L_KK into A64, L_KK^-1 into X64.
__global__ void __launch_bounds__(1024) chol_diag_kernel(const PrecondArgs *pas, int npairs, int K) {
    __shared__ double Ls[kB][kB + 1], Xs[kB][kB + 1];
    __shared__ int bad;
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
        const PrecondArgs &a = pas[p];
        const int np = pc_np(a.m * a.m + 1);
        if (K >= np / kB) continue;
        __syncthreads();
        if (threadIdx.x == 0) bad = 0;
        load_tile(a.A64, np, K, K, Ls);
        for (int k = 0; k < kB; ++k) {
            __syncthreads();
            if (threadIdx.x == 0) {
                const double d = Ls[k][k];
                if (!(d > 0.0)) bad = 1;
                Ls[k][k] = d > 0.0 ? sqrt(d) : 1.0;
            }
            __syncthreads();
            if (tx == k && ty > k) Ls[ty][k] /= Ls[k][k];
            __syncthreads();
            if (ty > k && tx > k && tx <= ty) Ls[ty][tx] -= Ls[ty][k] * Ls[tx][k];
        }
        __syncthreads();
        if (tx > ty) Ls[ty][tx] = 0.0;
        __syncthreads();
        if (threadIdx.x < kB) {   // column j of L^-1 by forward substitution
            const int j = threadIdx.x;
            for (int i = 0; i < kB; ++i) {
                if (i < j) {
                    Xs[i][j] = 0.0;
                    continue;
                }
                double s = (i == j) ? 1.0 : 0.0;
                for (int k = j; k < i; ++k) s -= Ls[i][k] * Xs[k][j];
                Xs[i][j] = s / Ls[i][i];
            }
        }
        __syncthreads();
        a.A64[(size_t)(K * kB + ty) * np + K * kB + tx] = Ls[ty][tx];
        a.X64[(size_t)(K * kB + ty) * np + K * kB + tx] = Xs[ty][tx];
        if (threadIdx.x == 0 && bad) a.st->pc_ok = 0;
    }
}

// Panel: L_IK = A_IK L_KK^-T for the block rows I > K (blockIdx.x = I - K - 1).
__global__ void __launch_bounds__(1024) chol_panel_kernel(const PrecondArgs *pas, int npairs, int K) {
    __shared__ double As[kB][kB + 1], Xs[kB][kB + 1];
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    const int I = K + 1 + blockIdx.x;
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int np = pc_np(a.m * a.m + 1);
        if (I >= np / kB) continue;
        __syncthreads();
        load_tile(a.A64, np, I, K, As);
        load_tile(a.X64, np, K, K, Xs);
        __syncthreads();
        double s = 0.0;
        for (int t = 0; t <= tx; ++t) s += As[ty][t] * Xs[tx][t];
        a.A64[(size_t)(I * kB + ty) * np + K * kB + tx] = s;
    }
}

// Trailing update: A_IJ -= L_IK L_JK^T for K < J <= I (blockIdx.x enumerates
// the (nb - K - 1)^2 pairs; the upper ones return).
__global__ void __launch_bounds__(1024) chol_update_kernel(const PrecondArgs *pas, int npairs, int K) {
    __shared__ double Li[kB][kB + 1], Lj[kB][kB + 1];
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int np = pc_np(a.m * a.m + 1), nb = np / kB, r = nb - K - 1;
        if (r <= 0 || (int)blockIdx.x >= r * r) continue;
        const int I = K + 1 + blockIdx.x / r, J = K + 1 + blockIdx.x % r;
        if (J > I) continue;
        __syncthreads();
        load_tile(a.A64, np, I, K, Li);
        load_tile(a.A64, np, J, K, Lj);
        __syncthreads();
        double s = 0.0;
#pragma unroll 8
        for (int t = 0; t < kB; ++t) s += Li[ty][t] * Lj[tx][t];
        a.A64[(size_t)(I * kB + ty) * np + J * kB + tx] -= s;
    }
}

// Block diagonal d of X = L^-1: X_IJ = -X_II sum_{T=J}^{I-1} L_IT X_TJ,
// I = J + d (blockIdx.x = J).
__global__ void __launch_bounds__(1024) trtri_kernel(const PrecondArgs *pas, int npairs, int d) {
    __shared__ double Ls[kB][kB + 1], Xs[kB][kB + 1];
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    const int J = blockIdx.x, I = J + d;
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int np = pc_np(a.m * a.m + 1);
        if (I >= np / kB) continue;
        double y = 0.0;
        for (int T = J; T < I; ++T) {
            __syncthreads();
            load_tile(a.A64, np, I, T, Ls);
            load_tile(a.X64, np, T, J, Xs);
            __syncthreads();
#pragma unroll 8
            for (int t = 0; t < kB; ++t) y += Ls[ty][t] * Xs[t][tx];
        }
        __syncthreads();
        Ls[ty][tx] = y;   // Y = sum_T L_IT X_TJ
        load_tile(a.X64, np, I, I, Xs);
        __syncthreads();
        double s = 0.0;
        for (int t = 0; t <= ty; ++t) s += Xs[ty][t] * Ls[t][tx];
        a.X64[(size_t)(I * kB + ty) * np + J * kB + tx] = -s;
    }
}

// P = X^T X: block (I, J), J <= I, sums X_TI^T X_TJ over T >= I; written to
// both triangles of the n x n float32 matrix.
__global__ void __launch_bounds__(1024) gram_kernel(const PrecondArgs *pas, int npairs) {
    __shared__ double Xa[kB][kB + 1], Xb[kB][kB + 1];
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int n = a.m * a.m + 1, np = pc_np(n), nb = np / kB;
        if ((int)blockIdx.x >= nb * nb) continue;
        const int I = blockIdx.x / nb, J = blockIdx.x % nb;
        if (J > I) continue;
        double s = 0.0;
        for (int T = I; T < nb; ++T) {
            __syncthreads();
            load_tile(a.X64, np, T, I, Xa);
            load_tile(a.X64, np, T, J, Xb);
            __syncthreads();
#pragma unroll 8
            for (int t = 0; t < kB; ++t) s += Xa[t][ty] * Xb[t][tx];
        }
        const int r = I * kB + ty, c = J * kB + tx;
        if (r < n && c < n) {
            a.P[(size_t)r * a.ldp + c] = (float)s;
            a.P[(size_t)c * a.ldp + r] = (float)s;
        }
    }
}

// ---------------------------------------------------------------- P v
// For a fit with a direction pending: pg = P g, and PY[slot] = P y_new when
// need_pc == 2.  P is applied as a dense float32 matrix (warp per row, rows
// over the CTAs), or, without the factorisation, as the diagonal pdiag.
constexpr int kPaThreads = 256;
constexpr int kPaRowsPerCta = kPaThreads / 32;
constexpr int kPaW = (kPcMaxN + 7) & ~3;   // staged vector length (16-byte multiple)

__device__ void pc_apply_body(const StepArgs &a, int blk, int nblk, float *ws) {
    const FitState *st = a.st;
    if (*((volatile const int *)&st->done) != 0) return;
    const int need = *((volatile const int *)&st->need_pc);
    if (need == 0) return;
    const OptBuffers &b = a.b;
    const int n = a.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int slot = st->pc_slot;
    const double *yv = need == 2 ? b.Y + (size_t)slot * n : nullptr;
    double *pyv = need == 2 ? b.PY + (size_t)slot * n : nullptr;
    if (!(st->pc_ok && b.P)) {
        for (int k = blk * kPaThreads + tid; k < n; k += nblk * kPaThreads) {
            b.pg[k] = b.pdiag[k] * b.grad[k];
            if (yv) pyv[k] = b.pdiag[k] * yv[k];
        }
        return;
    }
    const int ldp = b.ldp;
    float *g = ws, *y = ws + kPaW;
    for (int k = tid; k < ldp; k += kPaThreads) {
        g[k] = k < n ? (float)b.grad[k] : 0.f;
        y[k] = (yv && k < n) ? (float)yv[k] : 0.f;
    }
    __syncthreads();
    for (int r = blk * kPaRowsPerCta + warp; r < n; r += nblk * kPaRowsPerCta) {
        const float4 *row = reinterpret_cast<const float4 *>(b.P + (size_t)r * ldp);
        const float4 *g4 = reinterpret_cast<const float4 *>(g);
        const float4 *y4 = reinterpret_cast<const float4 *>(y);
        float s0 = 0.f, s1 = 0.f;
        for (int k = lane; k < ldp / 4; k += 32) {
            const float4 pv = row[k], gv = g4[k];
            s0 = fmaf(pv.x, gv.x, fmaf(pv.y, gv.y, fmaf(pv.z, gv.z, fmaf(pv.w, gv.w, s0))));
            if (yv) {
                const float4 yw = y4[k];
                s1 = fmaf(pv.x, yw.x, fmaf(pv.y, yw.y, fmaf(pv.z, yw.z, fmaf(pv.w, yw.w, s1))));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (lane == 0) {
            b.pg[r] = (double)s0;
            if (yv) pyv[r] = (double)s1;
        }
    }
}

__global__ void __launch_bounds__(kPaThreads) pc_apply_kernel(const StepArgs a) {
    __shared__ __align__(16) float ws[2 * kPaW];
    pc_apply_body(a, blockIdx.x, gridDim.x, ws);
}

__global__ void __launch_bounds__(kPaThreads) pc_apply_batch_kernel(const StepArgs *args,
                                                                    int npairs) {
    __shared__ __align__(16) float ws[2 * kPaW];
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        __syncthreads();
        const StepArgs a = args[p];
        if ((int)blockIdx.x * kPaRowsPerCta >= a.n) continue;
        pc_apply_body(a, blockIdx.x, gridDim.x, ws);
    }
}

}  // namespace

cudaError_t launch_precond(const PrecondArgs *d_pas, const PrecondArgs *h_pas, int npairs,
                           cudaStream_t s) {
    if (npairs < 1) return cudaErrorInvalidValue;
    int max_m = 1;
    for (int i = 0; i < npairs; ++i) {
        const PrecondArgs &a = h_pas[i];
        if (a.m * a.m + 1 > kPcMaxN || a.x1 - a.x0 > kAcMaxW || a.x1 <= a.x0 || a.y1 <= a.y0 ||
            a.ldp < a.m * a.m + 1 || (a.ldp & 3) != 0)
            return cudaErrorInvalidValue;
        max_m = max(max_m, a.m);
    }
    const int max_n = max_m * max_m + 1, nb = pc_np(max_n) / kB;
    const unsigned gy = (unsigned)min(npairs, 65535);
    rtilde_kernel<<<dim3(npairs == 1 ? 256 : 16, gy), 256, 0, s>>>(d_pas, npairs);
    autocorr_kernel<<<dim3(max_m + 1, gy), kAcThreads, 0, s>>>(d_pas, npairs);
    fill_kernel<<<dim3(npairs == 1 ? 64 : 8, gy), 256, 0, s>>>(d_pas, npairs);
    for (int K = 0; K < nb; ++K) {
        chol_diag_kernel<<<min(npairs, 65535), 1024, 0, s>>>(d_pas, npairs, K);
        const int r = nb - K - 1;
        if (r > 0) {
            chol_panel_kernel<<<dim3(r, gy), 1024, 0, s>>>(d_pas, npairs, K);
            chol_update_kernel<<<dim3(r * r, gy), 1024, 0, s>>>(d_pas, npairs, K);
        }
    }
    for (int d = 1; d < nb; ++d) trtri_kernel<<<dim3(nb - d, gy), 1024, 0, s>>>(d_pas, npairs, d);
    gram_kernel<<<dim3(nb * nb, gy), 1024, 0, s>>>(d_pas, npairs);
    return cudaGetLastError();
}

int precond_launches(int max_m) {
    const int nb = pc_np(max_m * max_m + 1) / kB;
    return 3 + nb + 2 * (nb - 1) + (nb - 1) + 1;
}

cudaError_t launch_pc_apply(const StepArgs &a, cudaStream_t s) {
    const int grid = (a.n + kPaRowsPerCta - 1) / kPaRowsPerCta;
    pc_apply_kernel<<<grid, kPaThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pc_apply_batch(const StepArgs *args, int npairs, int max_n, cudaStream_t s) {
    const int grid = (max_n + kPaRowsPerCta - 1) / kPaRowsPerCta;
    pc_apply_batch_kernel<<<dim3(grid, (unsigned)min(npairs, 65535)), kPaThreads, 0, s>>>(args,
                                                                                         npairs);
    return cudaGetLastError();
}

}  // namespace dia

// Preconditioner of L-BFGS, built once per fit, and its application P v
// inside every optimiser step.
//
// P is the inverse of the Gauss-Newton Hessian of the per-pixel loss over a
// window of valid pixels, H = sum_p w_p phi_p phi_p^T / N_window, with
// phi_p = [R window of p (Eq. 2), background basis at p (Eq. 18; 1 for B0)]
// and w_p = mask / (variance at M = I):
// for the fixed-variance chi^2 this is the exact Hessian (on the window), for
// the other losses its Gauss-Newton part.  As a Gram matrix it is positive
// semidefinite; the window keeps its cost to a few ms (pc_window_side).
//
// Build, every launch over all pairs of a batch (blockIdx.y, or blockIdx.x
// for one-CTA-per-pair kernels):
//   gn          64 x 64 blocks of the upper triangle of H, one pixel chunk per
//               CTA: phi of 32 pixels gathered into shared memory, a 4 x 4
//               register block per thread, float32 sums flushed to float64
//               every 512 pixels;
//   fill        chunks summed in a fixed order, scaled, the lower triangle
//               mirrored, the padding set to the identity (np = n rounded up
//               to 64);
//   per block column K of 32: chol_diag (factor the diagonal block, invert
//               it), chol_panel (L_IK = A_IK L_KK^-T), chol_update
//               (A_IJ -= L_IK L_JK^T);
//   per block diagonal d: trtri (X_IJ = -X_II sum_T L_IT X_TJ), X = L^-1;
//   gram        P = X^T X = H^-1 (float32, symmetric).
// pc_ok is cleared when a pivot is not positive (the diagonal preconditioner
// is used instead).
#include <cmath>

#include "dia_eval.cuh"
#include "dia_ops.cuh"

namespace dia {

namespace {

constexpr int kB = kPcB;

constexpr int kGnThreads = 256;
constexpr int kGnKB = 32;          // pixels per shared-memory batch
constexpr int kPadCol = -1000;     // column code of the zero padding beyond n

__host__ __device__ inline long long window_px(const PrecondArgs &a) {
    return (long long)(a.y1 - a.y0) * (a.x1 - a.x0);
}

// Block b of the upper triangle (row-major over U <= V) of nt x nt tiles.
__device__ __forceinline__ void gn_block(int b, int nt, int &U, int &V) {
    U = 0;
    while (b >= nt - U) {
        b -= nt - U;
        ++U;
    }
    V = U + b;
}

// Entry (u, v) of the Laplacian of the kernel-pixel graph (Eq. 21): the number
// of edge neighbours on the diagonal, -1 for pixels sharing an edge.
__device__ __forceinline__ int lap_entry(int u, int v, int mk) {
    const int ru = u / mk, cu = u - ru * mk;
    if (u == v) return (ru > 0) + (ru < mk - 1) + (cu > 0) + (cu < mk - 1);
    const int rv = v / mk, cv = v - rv * mk;
    return (abs(ru - rv) + abs(cu - cv) == 1) ? -1 : 0;
}

// 2 lambda (L^T L)_uv, the Hessian of the regulariser of Eq. 20 in the
// optimiser's 1/N_data scale; (L^T L)_uv = sum over k in {u} and the
// neighbours of u of L_uk L_kv (L symmetric).  Zero for B0.
__device__ __forceinline__ double reg_hess(const PrecondArgs &a, int u, int v) {
    const int mk = a.m, nk = mk * mk;
    if (a.reg2 == 0.0 || u >= nk || v >= nk) return 0.0;
    const int r = u / mk, c = u - r * mk;
    int s = lap_entry(u, u, mk) * lap_entry(u, v, mk);
    if (r > 0) s -= lap_entry(u - mk, v, mk);
    if (r < mk - 1) s -= lap_entry(u + mk, v, mk);
    if (c > 0) s -= lap_entry(u - 1, v, mk);
    if (c < mk - 1) s -= lap_entry(u + 1, v, mk);
    return a.reg2 * s;
}

// Per-pixel data of one batch: the pixel's offset in R, its weight and the
// Eq. 18 / Eq. 19 bases.  The global loads (weight inputs) are issued one
// batch early and the values formed after the FMA loop of the current batch.
struct GnPixLoads {
    float var, I, flat, wm;
    int mask;
};

__device__ __forceinline__ void gn_pix_load(const PrecondArgs &a, long long k, long long k1, int wx,
                                            int h, int ld, GnPixLoads &L) {
    L.var = 0.f;
    L.I = 0.f;
    L.flat = 1.f;
    L.wm = 0.f;
    L.mask = 1;
    if (k >= k1) return;
    const int py = a.y0 + (int)(k / wx), px = a.x0 + (int)(k % wx);
    if (a.wmap) {
        L.wm = a.wmap[(size_t)py * a.wmap_ld + px];
        return;
    }
    const size_t q = (size_t)(py + h) * ld + (px + h);
    if (a.lp.var_model == 0) {
        if (a.var) L.var = a.var[q];
    } else {
        L.I = a.I[q];
        if (a.flat) L.flat = a.flat[q];
    }
    if (a.mask) L.mask = a.mask[q];
}

// Weight of a target pixel from its loaded values: mask / variance at M = I
// (or the given per-pixel weight).
__device__ __forceinline__ float gn_pix_weight(const PrecondArgs &a, const GnPixLoads &L) {
    if (a.wmap) return L.wm;
    float v;
    if (a.lp.var_model == 0) {
        v = a.var ? L.var : a.lp.var_scalar;
    } else {
        const float F = a.flat ? L.flat : 1.f, Iv = fmaxf(L.I, 0.f);
        v = a.lp.var_model == 1 ? a.lp.s0sq / (F * F) + Iv * a.lp.inv_gain / F
                                : a.lp.excess * Iv * a.lp.inv_gain / F;
        v = fmaxf(v, a.lp.var_floor);
    }
    return (a.mask && L.mask == 0) ? 0.f : 1.0f / v;
}

// Sum of w_p phi_p phi_p^T over one 64 x 64 block (U, V) of the upper triangle
// and one chunk of window pixels; 16 x 16 threads of 4 x 4 entries each.
// Software-pipelined over batches of kGnKB pixels with one barrier per batch:
// while the FMA loop runs on batch i, every thread's phi loads of batch i+1
// and the per-pixel loads of batch i+2 are in flight; the products and their
// order (and the float64 flushes every a.flush batches) are those of a plain
// batch-by-batch loop.
__global__ void __launch_bounds__(kGnThreads, 2) gn_kernel(const PrecondArgs *pas, int npairs) {
    __shared__ __align__(16) float sA[2][kGnKB][kGnT], sB[2][kGnKB][kGnT];
    __shared__ int offU[kGnT], offV[kGnT];
    __shared__ long long sBase[2][kGnKB];
    __shared__ float sW[2][kGnKB];
    __shared__ float sBg[2][kGnKB][kBgMax];   // background basis eta^i xi^j of each pixel
    __shared__ float sKb[2][kGnKB][6];        // basis of a spatially varying kernel (degree <= 2)
    __shared__ unsigned char cU[kGnT], cV[kGnT];   // coefficient kernel of column u, v
    constexpr int kRows = kGnThreads / kGnT;        // batch rows one pass of the threads covers
    constexpr int kPer = kGnKB / kRows;             // phi values per thread and operand
    static_assert(kGnThreads % kGnT == 0 && kGnKB % kRows == 0, "gather layout");
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int ul = tid & (kGnT - 1), kr = tid / kGnT;   // this thread's column and first row
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int m = a.m, nk1 = m * m, nk = n_background(a.kdeg) * nk1, n = pc_n(a), h = m / 2,
                  ld = a.ld, nt = gn_tiles(n);
        const int deg = bg_degree_of(a.nbg), kdeg = a.kdeg;
        const int wx = a.x1 - a.x0;
        const long long npx = window_px(a);
        const int nch = a.gn_chunks, nblk = gn_blocks(n);
        if ((int)blockIdx.x >= nblk * nch) continue;
        const int b = blockIdx.x / nch, chunk = blockIdx.x % nch;
        int U, V;
        gn_block(b, nt, U, V);
        __syncthreads();   // shared memory of the previous pair
        // offset of phi_u in R relative to the window pixel's R[py][px];
        // -1 - c: background basis function c, kPadCol: padding (zero)
        if (tid < 2 * kGnT) {
            const int u = (tid < kGnT ? U : V) * kGnT + (tid & (kGnT - 1));
            const int uk = u % nk1;   // kernel pixel of a kernel column
            const int o = u < nk ? (uk / m) * ld + uk % m : (u < n ? -1 - (u - nk) : kPadCol);
            const unsigned char cc = (unsigned char)(u < nk ? u / nk1 : 0);
            if (tid < kGnT) {
                offU[tid] = o;
                cU[tid] = cc;
            } else {
                offV[tid - kGnT] = o;
                cV[tid - kGnT] = cc;
            }
        }
        float acc[4][4];
        double acc64[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[i][j] = 0.f;
                acc64[i][j] = 0.0;
            }
        const long long k0 = (long long)chunk * ((npx + nch - 1) / nch);
        const long long k1 = min(npx, k0 + (npx + nch - 1) / nch);
        const int nbat = k1 > k0 ? (int)((k1 - k0 + kGnKB - 1) / kGnKB) : 0;

        // per-pixel data of batch j into buffer j & 1 (threads < kGnKB)
        auto pix_store = [&](int j, const GnPixLoads &L) {
            const int sb = j & 1;
            const long long k = k0 + (long long)j * kGnKB + tid;
            if (k < k1) {
                const int py = a.y0 + (int)(k / wx), px = a.x0 + (int)(k % wx);
                sBase[sb][tid] = (long long)py * ld + px;
                sW[sb][tid] = gn_pix_weight(a, L);
                // basis of Eq. 18 in the coefficient order (power of xi fastest)
                const float eta = fmaf((float)px, a.eta_s, a.eta0);
                const float xi = fmaf((float)py, a.xi_s, a.xi0);
                int c = 0;
                float ep = 1.f;
                for (int i = 0; i <= deg; ++i) {
                    float t = ep;
                    for (int jj = 0; jj <= deg - i; ++jj) {
                        sBg[sb][tid][c++] = t;
                        t *= xi;
                    }
                    ep *= eta;
                }
                // the same basis for the coefficient kernels (degree kdeg)
                c = 0;
                ep = 1.f;
                for (int i = 0; i <= kdeg; ++i) {
                    float t = ep;
                    for (int jj = 0; jj <= kdeg - i; ++jj) {
                        sKb[sb][tid][c++] = t;
                        t *= xi;
                    }
                    ep *= eta;
                }
            } else {
                sBase[sb][tid] = -1;
                sW[sb][tid] = 0.f;
            }
        };
        // phi_u, phi_v of this thread's column for the rows of batch buffer sb
        auto gather = [&](int sb, float (&va)[kPer], float (&vb)[kPer]) {
            const int ou = offU[ul], ov = offV[ul];
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const int kk = kr + r * kRows;
                const long long base = sBase[sb][kk];
                float x = 0.f, y = 0.f;
                if (base >= 0) {
                    x = ou >= 0 ? a.R[base + ou] : (ou > kPadCol ? sBg[sb][kk][-1 - ou] : 0.f);
                    y = ov >= 0 ? a.R[base + ov] : (ov > kPadCol ? sBg[sb][kk][-1 - ov] : 0.f);
                    if (kdeg > 0) {   // column of coefficient kernel c: eta^p xi^q R
                        if (ou >= 0) x *= sKb[sb][kk][cU[ul]];
                        if (ov >= 0) y *= sKb[sb][kk][cV[ul]];
                    }
                }
                va[r] = x;
                vb[r] = y;
            }
        };
        auto put = [&](int sb, const float (&va)[kPer], const float (&vb)[kPer]) {
#pragma unroll
            for (int r = 0; r < kPer; ++r) {
                const int kk = kr + r * kRows;
                sA[sb][kk][ul] = sW[sb][kk] * va[r];
                sB[sb][kk][ul] = vb[r];
            }
        };

        // prologue: per-pixel data of batches 0 and 1, phi of batch 0
        GnPixLoads L;
        if (tid < kGnKB) {
            gn_pix_load(a, k0 + tid, k1, wx, h, ld, L);
            pix_store(0, L);
            gn_pix_load(a, k0 + kGnKB + tid, k1, wx, h, ld, L);
            pix_store(1, L);
        }
        __syncthreads();
        float va[kPer], vb[kPer];
        if (nbat > 0) {
            gather(0, va, vb);
            put(0, va, vb);
        }
        __syncthreads();
        int nb = 0;
        for (int i = 0; i < nbat; ++i) {
            const int cur = i & 1, nxt = cur ^ 1;
            const bool more = i + 1 < nbat;
            if (more) gather(nxt, va, vb);   // phi of batch i + 1 (in flight)
            if (tid < kGnKB) gn_pix_load(a, k0 + (long long)(i + 2) * kGnKB + tid, k1, wx, h, ld, L);
#pragma unroll 8
            for (int kk = 0; kk < kGnKB; ++kk) {
                const float4 av = *reinterpret_cast<const float4 *>(&sA[cur][kk][ty * 4]);
                const float4 bv = *reinterpret_cast<const float4 *>(&sB[cur][kk][tx * 4]);
                const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = fmaf(ar[ii], br[jj], acc[ii][jj]);
            }
            if (++nb == a.flush) {
                nb = 0;
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        acc64[ii][jj] += acc[ii][jj];
                        acc[ii][jj] = 0.f;
                    }
            }
            if (more) put(nxt, va, vb);
            // per-pixel data of batch i + 2 replaces that of batch i (read by the
            // phi of batch i, before the last barrier)
            if (tid < kGnKB) pix_store(i + 2, L);
            __syncthreads();
        }
        const double inv = a.scale;
        const int np = pc_np(n);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const double v = acc64[i][j] + acc[i][j];
                const int il = ty * 4 + i, jl = tx * 4 + j;
                if (nch > 1) {
                    a.part[((size_t)chunk * nblk + b) * (kGnT * kGnT) + il * kGnT + jl] = v;
                } else {   // final values of the upper blocks, in place
                    const int u = U * kGnT + il, w = V * kGnT + jl;
                    double t;
                    if (u >= n || w >= n)
                        t = (u == w) ? 1.0 : 0.0;
                    else
                        t = v * inv * ((u == w) ? 1.0 + a.eps : 1.0) + reg_hess(a, u, w);
                    a.A64[(size_t)u * np + w] = t;
                }
            }
    }
}

// H from the chunk partials (fixed order) or, with one chunk, the lower
// blocks mirrored from the upper ones; X64 and P zeroed; pc_ok set.
__global__ void fill_kernel(const PrecondArgs *pas, int npairs) {
    for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
        const PrecondArgs &a = pas[p];
        const int n = pc_n(a), np = pc_np(n), nt = gn_tiles(n), nblk = gn_blocks(n);
        const int nch = a.gn_chunks;
        const double inv = a.scale;
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)np * np;
             e += (long long)gridDim.x * blockDim.x) {
            const int u = (int)(e / np), w = (int)(e % np);
            // every entry from the upper one (a, b), a <= b, so that H is exactly
            // symmetric (the two triangles of a diagonal block are rounded differently)
            const int ea = min(u, w), eb = max(u, w);
            a.X64[e] = 0.0;
            if (nch == 1) {
                const double t = a.A64[(size_t)ea * np + eb];
                if (u > w) a.A64[e] = t;
                if (a.F_out && u < n && w < n) a.F_out[(size_t)u * n + w] = t;
                continue;
            }
            const int U = ea / kGnT, V = eb / kGnT;
            const int il = ea - U * kGnT, jl = eb - V * kGnT;
            const int b = U * nt - U * (U - 1) / 2 + (V - U);
            double t;
            if (u >= n || w >= n) {
                t = (u == w) ? 1.0 : 0.0;
            } else {
                double s = 0.0;
                for (int c = 0; c < nch; ++c)
                    s += a.part[((size_t)c * nblk + b) * (kGnT * kGnT) + il * kGnT + jl];
                t = s * inv * ((u == w) ? 1.0 + a.eps : 1.0) + reg_hess(a, u, w);
                if (a.F_out) a.F_out[(size_t)u * n + w] = t;
            }
            a.A64[e] = t;
        }
        // P, including the pitch padding that P v reads (times zero)
        if (a.P)
            for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
                 e < (long long)n * a.ldp; e += (long long)gridDim.x * blockDim.x)
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
        const int np = pc_np(pc_n(a));
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
        const int np = pc_np(pc_n(a));
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
        const int np = pc_np(pc_n(a)), nb = np / kB, r = nb - K - 1;
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
        const int np = pc_np(pc_n(a));
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
        const int n = pc_n(a), np = pc_np(n), nb = np / kB;
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
            if (a.cov_out) {
                a.cov_out[(size_t)r * n + c] = s;
                a.cov_out[(size_t)c * n + r] = s;
            } else if (a.P) {
                a.P[(size_t)r * a.ldp + c] = (float)s;
                a.P[(size_t)c * a.ldp + r] = (float)s;
            }
        }
    }
}

// ---------------------------------------------------------------- P v
// For a fit with a direction pending: pg = P g, and PY[slot] = P y_new when
// need_pc == 2.  P is applied as a dense float32 matrix (warp per row, rows
// over the CTAs), or, without the factorisation, as the diagonal pdiag.
__global__ void __launch_bounds__(kPaThreads) pc_apply_kernel(const StepArgs a) {
    __shared__ __align__(16) float ws[2 * kPaW];
    pc_apply_body(a, blockIdx.x, gridDim.x, ws);
}

}  // namespace

cudaError_t launch_precond(const PrecondArgs *d_pas, const PrecondArgs *h_pas, int npairs,
                           cudaStream_t s) {
    if (npairs < 1) return cudaErrorInvalidValue;
    int max_n = 1, gn_grid = 1;
    for (int i = 0; i < npairs; ++i) {
        const PrecondArgs &a = h_pas[i];
        const int n = pc_n(a);
        if (a.nbg < 1 || a.nbg > kBgMax || n > kPcMaxN || a.x1 <= a.x0 || a.y1 <= a.y0 || a.ldp < n || (a.ldp & 3) != 0 ||
            a.gn_chunks < 1 || (a.gn_chunks > 1 && !a.part) || a.flush < 1 ||
            (long long)a.gn_chunks > window_px(a))
            return cudaErrorInvalidValue;
        max_n = max(max_n, n);
        gn_grid = max(gn_grid, gn_blocks(n) * a.gn_chunks);
    }
    const int nb = pc_np(max_n) / kB;
    const unsigned gy = (unsigned)min(npairs, 65535);
    gn_kernel<<<dim3(gn_grid, gy), kGnThreads, 0, s>>>(d_pas, npairs);
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

int precond_launches(int max_n) {
    const int nb = pc_np(max_n) / kB;
    return 2 + nb + 2 * (nb - 1) + (nb - 1) + 1;
}

// Window (centred, side pc_window_side) and chunk count of a pair's
// Hessian sum; chunks > 1 only for a single pair (a batch has parallelism
// across its pairs).
void precond_window(int H, int W, int m, bool single, int side_opt, int *y0, int *y1, int *x0,
                    int *x1, int *chunks) {
    const int h = m / 2, Hv = H - 2 * h, Wv = W - 2 * h;
    const int side = side_opt > 0 ? side_opt : pc_window_side(m * m + 1);
    const int sy = min(Hv, side), sx = min(Wv, side);
    *y0 = (Hv - sy) / 2;
    *y1 = *y0 + sy;
    *x0 = (Wv - sx) / 2;
    *x1 = *x0 + sx;
    const long long px = (long long)sy * sx;
    *chunks = single ? (int)min(64LL, (px + kGnChunk - 1) / kGnChunk) : 1;
}

cudaError_t launch_pc_apply(const StepArgs &a, cudaStream_t s) {
    const int grid = (a.n + kPaRowsPerCta - 1) / kPaRowsPerCta;
    pc_apply_kernel<<<grid, kPaThreads, 0, s>>>(a);
    return cudaGetLastError();
}


}  // namespace dia

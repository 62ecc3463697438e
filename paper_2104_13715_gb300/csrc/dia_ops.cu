// Reduction, optimiser, initialisation and median kernels (see dia_ops.cuh).
#include <cmath>
#include <cstring>

#include "dia_eval.cuh"
#include "dia_ops.cuh"

namespace dia {

// ----------------------------------------------------------------------------
// Float64 sum of the per-CTA partials in a fixed order (bitwise repeatable).
// Block b handles entries [32b, 32b+32); its 8 warps take every 8th CTA row.
// acc32: the same sums in float32 (the comparison form of the precision study).
__global__ void __launch_bounds__(256) reduce_kernel(const double *__restrict__ partials, int G,
                                                     int NP, double *__restrict__ out,
                                                     const int *done, int acc32) {
    if (done != nullptr && *((volatile const int *)done) != 0) return;
    __shared__ double sh[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    double s = 0.0;
    float s32 = 0.f;
    if (e < NP)
        for (int g = warp; g < G; g += 8) {
            const double v = partials[(size_t)g * NP + e];
            s += v;
            s32 += (float)v;
        }
    sh[warp][lane] = acc32 ? (double)s32 : s;
    __syncthreads();
    if (warp == 0 && e < NP) {
        double t = 0.0;
        float t32 = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            t += sh[w][lane];
            t32 += (float)sh[w][lane];
        }
        out[e] = acc32 ? (double)t32 : t;
    }
}

cudaError_t launch_reduce(const double *partials, int G, int NP, double *out, const int *done,
                          cudaStream_t s, int acc32) {
    reduce_kernel<<<(NP + 31) / 32, 256, 0, s>>>(partials, G, NP, out, done, acc32);
    return cudaGetLastError();
}

// float32 copy of theta for the fused kernels: nc blocks (one per kernel
// coefficient of a spatially varying kernel, nc = 1 otherwise) of m rows of kp
// floats (zero padded), then the nb background coefficients and zeros up to
// kBgMax + 1.
__device__ __forceinline__ void write_kpad(const double *th, int mk, int kp, int nb, float *Kpad,
                                           int tid, int nt, int nc = 1) {
    const int blk = mk * kp;
    for (int i = tid; i < nc * blk; i += nt) {
        const int c = i / blk, r = i - c * blk;
        const int a = r / kp, b = r - a * kp;
        Kpad[i] = (b < mk) ? (float)th[(c * mk + a) * mk + b] : 0.f;
    }
    for (int i = tid; i < kBgMax + 1; i += nt)
        Kpad[nc * blk + i] = (i < nb) ? (float)th[nc * mk * mk + i] : 0.f;
}

// kernel coefficient sets of a fit (a spatially varying kernel has several)
__host__ __device__ inline int n_coef(const StepArgs &a) { return a.nc > 1 ? a.nc : 1; }
__host__ __device__ inline int n_kpar(const StepArgs &a) { return n_coef(a) * a.mk * a.mk; }

__global__ void prep_kpad_kernel(const double *theta, int mk, int kp, int nb, float *Kpad, int nc) {
    write_kpad(theta, mk, kp, nb, Kpad, threadIdx.x, blockDim.x, nc);
}

cudaError_t launch_prep_kpad(const double *theta, int mk, int kp, int nb, float *Kpad,
                             cudaStream_t s, int nc) {
    prep_kpad_kernel<<<1, 256, 0, s>>>(theta, mk, kp, nb, Kpad, nc);
    return cudaGetLastError();
}

__global__ void emit_kernel(const double *red, int nk, int nb, double *loss, double *grad) {
    const int n = nk + nb;
    for (int k = threadIdx.x; k < n; k += blockDim.x) grad[k] = red[1 + k];
    if (threadIdx.x == 0) *loss = red[0];
}

cudaError_t launch_emit_loss_grad(const double *red, int mk, int nb, double *loss, double *grad,
                                  cudaStream_t s, int nc) {
    emit_kernel<<<1, 256, 0, s>>>(red, nc * mk * mk, nb, loss, grad);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// One-CTA float64 helpers
constexpr int kStepThreads = 256;

__device__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kStepThreads / 32; ++w) t += sh[w];
    return t;
}

__device__ double block_max(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = sh[0];
#pragma unroll
    for (int w = 1; w < kStepThreads / 32; ++w) t = fmax(t, sh[w]);
    return t;
}

__device__ double dot(const double *x, const double *y, int n, double *sh) {
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += kStepThreads) s += x[k] * y[k];
    return block_sum(s, sh);
}

enum { kActContinue = 0, kActAcceptTrial = 1, kActAcceptLo = 2, kActFail = 3 };

struct StepShared {
    double red[kStepThreads / 32];
    double gt[1024];          // scaled gradient at the trial point
    double lt[1024];          // L theta of the regulariser (kernel pixels)
    double v[4][kHistMax];    // compact-form vectors over the history
    int act, finish_status, copy_glo;
    double new_alpha;
};

// x . y over n entries by one warp (every lane gets the sum).
__device__ __forceinline__ double warp_dot(const double *x, const double *y, int n) {
    double s = 0.0;
    for (int k = threadIdx.x & 31; k < n; k += 32) s = fma(x[k], y[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// History slot of chronological entry c (0 = oldest) of hl entries ending before head.
__device__ __forceinline__ int hist_slot(int c, int hl, int head, int H) {
    return (head - hl + c + 2 * H) % H;
}

__device__ void set_trial(const StepArgs &a, double alpha) {
    const OptBuffers &b = a.b;
    for (int k = threadIdx.x; k < a.n; k += kStepThreads) b.trial[k] = b.theta[k] + alpha * b.dir[k];
    __syncthreads();
    write_kpad(b.trial, a.mk, a.kp, a.n - n_kpar(a), a.Kpad, threadIdx.x, kStepThreads, n_coef(a));
}

constexpr double kNoProgress = 1e-2;   // see finish()

// Finish the pass: theta is the answer; the next evaluation (if any) sees it.
__device__ void finish(const StepArgs &a, int status, int reason) {
    FitState *st = a.st;
    for (int k = threadIdx.x; k < a.n; k += kStepThreads) a.b.trial[k] = a.b.theta[k];
    __syncthreads();
    write_kpad(a.b.theta, a.mk, a.kp, a.n - n_kpar(a), a.Kpad, threadIdx.x, kStepThreads,
               n_coef(a));
    if (threadIdx.x == 0) {
        // a pass that stops for lack of progress is at the limit of numerical
        // precision only if max|g| came down by orders of magnitude from the
        // fit's start (measured floors are ~1e-6 of it); otherwise it failed
        if (status == 0 && (reason == kStopStall || reason == kStopLineSearch) &&
            !st->from_theta0 && st->ginf_first > 0.0 && st->ginf_best > kNoProgress * st->ginf_first)
            status = 5; /* DIA_ERR_LINESEARCH */
        st->status = status;
        st->reason = reason;
        // the float32 floor of max|g| found by this pass serves the refits
        if (status == 0 && (reason == kStopStall || reason == kStopLineSearch))
            st->ginf_floor = st->ginf_best;
        st->phase = kPhaseDone;
        st->L_sum = st->L * st->ndata;
        __threadfence();
        st->done = 1;
        if (a.n_done) atomicAdd(a.n_done, 1);
    }
}

// Graph Laplacian of the kernel surface (Eq. 21) applied to x at kernel pixel
// k = r * mk + c: sum over its edge neighbours j of (x_k - x_j).
__device__ __forceinline__ double lap_apply(const double *x, int k, int mk) {
    const int r = k / mk, c = k - r * mk;
    const double t = x[k];
    double v = 0.0;
    if (r > 0) v += t - x[k - mk];
    if (r < mk - 1) v += t - x[k + mk];
    if (c > 0) v += t - x[k - 1];
    if (c < mk - 1) v += t - x[k + 1];
    return v;
}

// Regulariser of Eq. 20 at the evaluated point (trial), in the optimiser's
// 1/N_data scale: returns lambda |L theta|^2 and adds 2 lambda L^T L theta
// (L symmetric) to the scaled gradient sm.gt.  B0 is not penalised.
__device__ double add_penalty(const StepArgs &a, StepShared &sm) {
    const int mk = a.mk, nk = mk * mk;
    const double lam = a.p.reg_lambda;
    double s = 0.0;
    for (int k = threadIdx.x; k < nk; k += kStepThreads) {
        const double v = lap_apply(a.b.trial, k, mk);
        sm.lt[k] = v;
        s += v * v;
    }
    const double pen = block_sum(s, sm.red);   // also orders the sm.lt writes
    for (int k = threadIdx.x; k < nk; k += kStepThreads) sm.gt[k] += 2.0 * lam * lap_apply(sm.lt, k, mk);
    __syncthreads();
    return lam * pen;
}

// Diagonal preconditioner from the curvature sums of the last evaluation:
// kernel pixels ~ 1/sum(kappa R^2), B0 ~ 1/sum(kappa) (Gauss-Newton diagonal
// with the kernel-pixel entries approximated by the centre pixel); background
// coefficient b_ij ~ 1/(sum(kappa) E[eta^2i] E[xi^2j]) with eta, xi taken as
// uniform on [-1/2, 1/2] (E[eta^2i] = 4^-i / (2i + 1)).
__device__ void update_precond(const StepArgs &a) {
    const int mk = a.mk, nk = n_kpar(a), deg = bg_degree_of(a.n - nk);
    const int kdeg = bg_degree_of(n_coef(a));   // degree of a spatially varying kernel
    const double dk = a.red[red_count(nk) + 1], db = a.red[red_count(nk) + 2];
    const double pk = (dk > 0.0 && isfinite(dk)) ? 1.0 / dk : 1.0;
    const double pb = (db > 0.0 && isfinite(db)) ? 1.0 / db : 1.0;
    const double N = a.red[red_count(nk)];
    for (int k = threadIdx.x; k < a.n; k += kStepThreads) {
        double p = N * ((k >= nk) ? pb : pk);   // the loss is scaled by 1/N
        if (k < nk && k >= mk * mk) {
            // coefficient kernel c of a spatially varying kernel: its pixels are
            // scaled like the background coefficient of the same (i, j)
            int c = k / (mk * mk), i = 0;
            while (c > kdeg - i) {
                c -= kdeg - i + 1;
                ++i;
            }
            const int j = c;
            p *= (double)(2 * i + 1) * (double)(1 << (2 * i)) * (double)(2 * j + 1) *
                 (double)(1 << (2 * j));
        }
        if (k > nk) {
            int c = k - nk, i = 0;
            while (c > deg - i) {   // (i, j) of coefficient c
                c -= deg - i + 1;
                ++i;
            }
            const int j = c;
            p *= (double)(2 * i + 1) * (double)(1 << (2 * i)) * (double)(2 * j + 1) *
                 (double)(1 << (2 * j));
        }
        if (a.p.reg_lambda > 0.0 && k < nk) {
            // plus the regulariser's diagonal 2 lambda (L^T L)_kk = 2 lambda d (d + 1),
            // d the number of edge neighbours of kernel pixel k
            const int r = k / mk, c = k - r * mk;
            const int d = (r > 0) + (r < mk - 1) + (c > 0) + (c < mk - 1);
            p = 1.0 / (1.0 / p + 2.0 * a.p.reg_lambda * d * (d + 1));
        }
        a.b.pdiag[k] = p;
    }
}

// A new L-BFGS direction is needed at the accepted point: P g (and P y_new
// when a curvature pair was just stored in slot `slot`) are computed by the
// multi-CTA preconditioner kernel, then direction_body finishes the step.
__device__ void request_direction(const StepArgs &a, int slot) {
    if (threadIdx.x == 0) {
        a.st->need_pc = slot >= 0 ? 2 : 1;
        a.st->pc_slot = slot;
    }
}

// The direction half of the step (one CTA): new row of y'Py, the compact
// representation of the L-BFGS inverse Hessian (Byrd, Nocedal & Schnabel
// 1994, Theorem 2.2) with H0 = tau P, tau = s'y / y'Py of the newest pair,
//   H g = tau P g + S p1 + tau (PY) p2,  u = R^-1 S'g,  p2 = -u,
//   p1 = R^-T ((D + tau Y'PY) u - tau (PY)'g),
// R the upper triangle of S'Y and D its diagonal (chronological order); then
// the start of the line search at alpha = 1 (Sec. 2.9).
__device__ void direction_body(const StepArgs &a, StepShared &sm) {
    FitState *st = a.st;
    if (*((volatile int *)&st->done) != 0) return;
    const int need = st->need_pc;
    if (need == 0) return;
    const OptBuffers &b = a.b;
    const int n = a.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, H = a.p.history;
    constexpr int NWS = kStepThreads / 32;
    int hl = st->hist_len;
    const int head = st->hist_head;
    if (need == 2) {   // row and column of y_new' P y_j
        const int sn = st->pc_slot;
        const double *py = b.PY + (size_t)sn * n;
        for (int c = warp; c < hl; c += NWS) {
            const int j = hist_slot(c, hl, head, H);
            const double v = warp_dot(py, b.Y + (size_t)j * n, n);
            if (lane == 0) {
                b.YPY[(size_t)sn * H + j] = v;
                b.YPY[(size_t)j * H + sn] = v;
            }
        }
        __syncthreads();
    }
    double tau = 1.0;
    if (hl > 0) {
        const int nw = hist_slot(hl - 1, hl, head, H);
        tau = b.SY[(size_t)nw * H + nw] / b.YPY[(size_t)nw * H + nw];
        if (!(tau > 0.0) || !isfinite(tau)) tau = 1.0;
    }
    // a_c = s_c . g, b_c = tau (P y_c) . g
    for (int t = warp; t < 2 * hl; t += NWS) {
        const int c = t < hl ? t : t - hl;
        const int j = hist_slot(c, hl, head, H);
        const double v = warp_dot(t < hl ? b.S + (size_t)j * n : b.PY + (size_t)j * n, b.grad, n);
        if (lane == 0) sm.v[t < hl ? 0 : 1][c] = t < hl ? v : tau * v;
    }
    __syncthreads();
    if (warp == 0 && hl > 0) {
        double *A = sm.v[0], *B = sm.v[1], *U = sm.v[2], *T = sm.v[3];
        auto R = [&](int c1, int c2) {   // s_c1 . y_c2 (chronological indices)
            return b.SY[(size_t)hist_slot(c1, hl, head, H) * H + hist_slot(c2, hl, head, H)];
        };
        // U = R^-1 A (back substitution, column sweep; A is the accumulator)
        for (int c = hl - 1; c >= 0; --c) {
            const double uc = A[c] / R(c, c);
            __syncwarp();
            if (lane == 0) U[c] = uc;
            for (int r = lane; r < c; r += 32) A[r] -= R(r, c) * uc;
            __syncwarp();
        }
        // T = D U + tau Y'PY U
        for (int r = lane; r < hl; r += 32) {
            const int jr = hist_slot(r, hl, head, H);
            double t = R(r, r) * U[r];
            for (int c = 0; c < hl; ++c)
                t += tau * b.YPY[(size_t)jr * H + hist_slot(c, hl, head, H)] * U[c];
            T[r] = t;
        }
        __syncwarp();
        // T <- R^-T T, B <- R^-T B (forward substitution, column sweep, in place)
        for (int c = 0; c < hl; ++c) {
            const double d = R(c, c);
            const double tc = T[c] / d, bc = B[c] / d;
            __syncwarp();
            if (lane == 0) {
                T[c] = tc;
                B[c] = bc;
            }
            for (int r = c + 1 + lane; r < hl; r += 32) {
                const double rc = R(c, r);
                T[r] -= rc * tc;
                B[r] -= rc * bc;
            }
            __syncwarp();
        }
        // p1 = T - B (in T), p2 = -U (in U)
        for (int r = lane; r < hl; r += 32) {
            T[r] -= B[r];
            U[r] = -U[r];
        }
    }
    __syncthreads();
    for (int k = tid; k < n; k += kStepThreads) {
        double hg = tau * b.pg[k];
        for (int c = 0; c < hl; ++c) {
            const int j = hist_slot(c, hl, head, H);
            hg += sm.v[3][c] * b.S[(size_t)j * n + k] + tau * sm.v[2][c] * b.PY[(size_t)j * n + k];
        }
        b.dir[k] = -hg;
    }
    __syncthreads();
    double gd0 = dot(b.grad, b.dir, n, sm.red);
    if (!(gd0 < 0.0) || !isfinite(gd0)) {          // not a descent direction: preconditioned SD
        for (int k = tid; k < n; k += kStepThreads) b.dir[k] = -b.pg[k];
        __syncthreads();
        gd0 = dot(b.grad, b.dir, n, sm.red);
        if (tid == 0) st->hist_len = 0;
    }
    for (int k = tid; k < n; k += kStepThreads) b.glo[k] = b.grad[k];
    // L-BFGS learning rate 1 (Sec. 2.9).  Without curvature pairs the step is
    // the preconditioner's Gauss-Newton step, whose model can be far off where
    // the variance depends on M and the residuals are large: the first trial
    // is then capped so that its predicted decrease is at most 4 |L| (the
    // loss), and scaled down further after a failed search (alpha0)
    double a_init = 1.0;
    if (st->hist_len == 0) {
        const double L = st->L;
        if (L > 0.0 && -gd0 > 4.0 * L) a_init = 4.0 * L / -gd0;
        a_init *= st->alpha0 > 0.0 ? st->alpha0 : 1.0;
    }
    if (tid == 0) {
        st->gd0 = gd0;
        st->alpha = a_init;
        st->lo = 0.0;
        st->L_lo = st->L;
        st->gd_lo = gd0;
        st->hi = -1.0;
        st->ls_evals = 0;
        st->need_pc = 0;
    }
    __syncthreads();
    set_trial(a, a_init);
}

// A refit (sigma-clip pass) is at the limit of numerical precision once max|g|
// is within kFloorFactor of the floor an earlier pass of the same fit reached
// (same images, same float32 arithmetic, nearly the same theta), so it need
// not spend stall_iters evaluations finding that floor again.
constexpr double kFloorFactor = 3.0;
__device__ __forceinline__ bool at_floor(const FitState *st, double ginf) {
    return st->ginf_floor > 0.0 && ginf <= kFloorFactor * st->ginf_floor;
}

// Evaluations without a halving of max|g| that end the pass: the block-
// Newton preconditioned iteration reaches its float32 floor within tens of
// evaluations, the diagonally preconditioned one needs far more.
__device__ __forceinline__ int stall_limit(const StepArgs &a) {
    const FitState *st = a.st;
    int lim = (st->pc_ok && a.b.P) ? a.p.stall_iters : a.p.stall_iters_diag;
    // far above any float32 floor (max|g| not yet down to kNoProgress of the
    // fit's first gradient, e.g. a redescending loss started far from the
    // optimum) a stall is slow progress, not the precision limit
    if (!st->from_theta0 && st->ginf_first > 0.0 && st->ginf_best > kNoProgress * st->ginf_first)
        lim = max(lim, a.p.stall_iters_diag);
    return lim;
}

// Line-search decision for the trial alpha (thread 0).  Wolfe conditions, or
// the approximate Wolfe conditions of Hager & Zhang (2005), which rely on the
// float64 directional derivative when loss differences fall below the
// float32 pixel-rounding level; brackets are updated on the sign of phi'.
__device__ int line_search_decide(FitState *st, double Lt, double gdt, int max_ls, double &na,
                                  int &copy_glo) {
    const double al = st->alpha, L0 = st->L, gd0 = st->gd0;
    const double delta = 0.1, sigma = 0.9, eps_f = 1e-6 * fabs(L0);
    copy_glo = 0;
    const bool wolfe = (Lt <= L0 + delta * al * gd0) && (gdt >= sigma * gd0);
    const bool approx = (Lt <= L0 + eps_f) && ((2.0 * delta - 1.0) * gd0 >= gdt) && (gdt >= sigma * gd0);
    if (isfinite(Lt) && (wolfe || approx)) return kActAcceptTrial;
    if (gdt >= 0.0 || !isfinite(Lt)) {
        st->hi = al; st->L_hi = Lt; st->gd_hi = isfinite(gdt) ? gdt : 1.0;
    } else if (Lt <= L0 + eps_f) {
        st->lo = al; st->L_lo = Lt; st->gd_lo = gdt;
        copy_glo = 1;
    } else {
        st->hi = al; st->L_hi = Lt; st->gd_hi = gdt;   // too high with a negative slope
    }
    if (st->hi < 0.0) {
        na = 5.0 * al;                                  // no bracket yet: expand
    } else {
        const double a0 = st->lo, a1 = st->hi, w = a1 - a0;
        na = 0.5 * (a0 + a1);
        if (st->gd_hi >= 0.0 && st->gd_hi > st->gd_lo) {   // secant on phi'
            const double c = (a0 * st->gd_hi - a1 * st->gd_lo) / (st->gd_hi - st->gd_lo);
            if (isfinite(c) && c > a0 + 0.01 * w && c < a1 - 0.01 * w) na = c;
        }
    }
    st->ls_evals += 1;
    const bool collapsed = st->hi >= 0.0 && (st->hi - st->lo) <= 1e-13 * fmax(1.0, st->lo);
    if (st->ls_evals >= max_ls || collapsed || na > 1e10) {
        return (st->lo > 0.0) ? kActAcceptLo : kActFail;
    }
    return kActContinue;
}

// One optimiser step of one fit (the whole CTA): reads the reduced sums of
// the last evaluation, updates the FP64 state and writes the next trial K.
__device__ void step_body(const StepArgs &a, StepShared &sm) {
    FitState *st = a.st;
    if (*((volatile int *)&st->done) != 0) return;
    const OptBuffers &b = a.b;
    const OptParams &p = a.p;
    const int n = a.n, tid = threadIdx.x;

    const double N = a.red[red_count(n_kpar(a))];
    if (!(N > 0.0)) {
        finish(a, 6 /* DIA_ERR_DEGENERATE */, kStopDegenerate);
        return;
    }
    const double invN = 1.0 / N;
    double Lt = a.red[0] * invN;
    const bool first_eval = *((volatile int *)&st->evals) == 0;   // read before the update below
    for (int k = tid; k < n; k += kStepThreads) sm.gt[k] = a.red[1 + k] * invN;
    if (p.reg_lambda > 0.0) {
        __syncthreads();
        Lt += add_penalty(a, sm);
    }
    bool bad = !isfinite(Lt);
    for (int k = tid; k < n; k += kStepThreads) bad |= !isfinite(sm.gt[k]);
    const int nbad = __syncthreads_or(bad);
    if (tid == 0) {
        st->evals += 1;
        st->ndata = N;
    }
    if (nbad) {
        finish(a, 3 /* DIA_ERR_NONFINITE */, kStopNonfinite);
        return;
    }
    if (first_eval) {   // the scale against which progress is measured (finish())
        double mx = 0.0;
        for (int k = tid; k < n; k += kStepThreads) mx = fmax(mx, fabs(sm.gt[k]));
        const double g0 = block_max(mx, sm.red);
        if (tid == 0) st->ginf_first = g0;
    }

    int phase = st->phase;
    if (phase == kPhaseAdam) {
        const bool sw = (st->it_adam > 0 && fabs(Lt - st->L_prev) <= p.switch_tol * fabs(st->L_prev)) ||
                        st->it_adam >= p.max_adam;
        if (!sw) {
            // Adam step (Kingma & Ba), per-parameter learning rates (Sec. 2.9)
            const double b1t = st->b1t * p.beta1, b2t = st->b2t * p.beta2;
            const double bc1 = 1.0 - b1t, bc2 = 1.0 - b2t;
            for (int k = tid; k < n; k += kStepThreads) {
                const double g = sm.gt[k];
                const double m1 = p.beta1 * b.m1[k] + (1.0 - p.beta1) * g;
                const double m2 = p.beta2 * b.m2[k] + (1.0 - p.beta2) * g * g;
                b.m1[k] = m1;
                b.m2[k] = m2;
                const double lr = (k >= n_kpar(a)) ? p.lr_b0 : p.lr_kernel;
                const double th = b.theta[k] - lr * (m1 / bc1) / (sqrt(m2 / bc2) + p.adam_eps);
                b.theta[k] = th;
                b.trial[k] = th;
            }
            __syncthreads();
            write_kpad(b.trial, a.mk, a.kp, n - n_kpar(a), a.Kpad, tid, kStepThreads, n_coef(a));
            if (tid == 0) {
                st->b1t = b1t;
                st->b2t = b2t;
                st->L_prev = Lt;
                st->L = Lt;
                st->it_adam += 1;
                sm.finish_status = (st->evals >= p.max_evals) ? 4 /* DIA_ERR_MAXITER */ : -1;
            }
            __syncthreads();
            if (sm.finish_status >= 0) finish(a, sm.finish_status, kStopMaxEvals);
            return;
        }
        phase = kPhaseLbfgsStart;  // hand over to L-BFGS at the point just evaluated
    }

    if (phase == kPhaseLbfgsStart) {
        update_precond(a);
        double mx = 0.0;
        for (int k = tid; k < n; k += kStepThreads) {
            b.grad[k] = sm.gt[k];
            mx = fmax(mx, fabs(sm.gt[k]));
        }
        const double ginf = block_max(mx, sm.red);
        if (tid == 0) {
            st->L = Lt;
            st->L_sum = Lt * N;
            st->grad_inf = ginf;
            st->hist_len = 0;
            st->hist_head = 0;
            st->ls_restarts = 0;
            st->ginf_best = ginf;
            st->ev_best = st->evals;
            st->stall = 0;
            st->phase = kPhaseLbfgs;
        }
        __syncthreads();
        if (ginf < p.grad_tol) {
            finish(a, 0, kStopGradTol);
            return;
        }
        if (at_floor(st, ginf)) {
            finish(a, 0, kStopFloor);
            return;
        }
        request_direction(a, -1);
        return;
    }

    // ---- L-BFGS line search: trial = theta + alpha * dir was evaluated
    const double gdt = dot(sm.gt, b.dir, n, sm.red);
    if (tid == 0) {
        double na = st->alpha;
        int copy_glo = 0;
        int act = line_search_decide(st, Lt, gdt, p.max_ls, na, copy_glo);
        if (act == kActContinue && st->evals >= p.max_evals) act = (st->lo > 0.0) ? kActAcceptLo : kActFail;
        sm.act = act;
        sm.copy_glo = copy_glo;
        sm.new_alpha = na;
    }
    __syncthreads();
    const int act = sm.act;
    if (sm.copy_glo)
        for (int k = tid; k < n; k += kStepThreads) b.glo[k] = sm.gt[k];
    __syncthreads();

    if (act == kActContinue) {
        if (tid == 0) st->alpha = sm.new_alpha;
        set_trial(a, sm.new_alpha);
        return;
    }
    if (act == kActFail) {
        // restart from preconditioned steepest descent (at most twice in a
        // row), else stop: no decrease is found at this precision
        if (tid == 0) {
            sm.finish_status = -1;
            sm.act = kStopLineSearch;
            st->stall = st->evals - st->ev_best;
            if (st->evals >= p.max_evals) {
                sm.finish_status = 4; /* DIA_ERR_MAXITER */
                sm.act = kStopMaxEvals;
            } else if (st->stall >= stall_limit(a) && st->it_lbfgs > 0) {
                sm.finish_status = 0;
                sm.act = kStopStall;
            } else if (st->ls_restarts < 2) {
                // restart from preconditioned steepest descent; a search that
                // already had no history retries with a 100x shorter first step
                if (st->hist_len == 0) st->alpha0 = (st->alpha0 > 0.0 ? st->alpha0 : 1.0) * 0.01;
                st->hist_len = 0;
                st->ls_restarts += 1;
            } else {
                sm.finish_status = st->it_lbfgs > 0 ? 0 : 5 /* DIA_ERR_LINESEARCH */;
            }
        }
        __syncthreads();
        if (sm.finish_status < 0)
            request_direction(a, -1);
        else
            finish(a, sm.finish_status, sm.act);
        return;
    }

    // ---- accept: the trial point, or the best point of the search
    const bool use_trial = (act == kActAcceptTrial);
    const double aacc = use_trial ? st->alpha : st->lo;
    const double Lacc = use_trial ? Lt : st->L_lo;
    const double *gacc = use_trial ? sm.gt : b.glo;
    const int H = p.history, head = st->hist_head, hl0 = st->hist_len;
    double *Sn = b.S + (size_t)head * n, *Yn = b.Y + (size_t)head * n;
    for (int k = tid; k < n; k += kStepThreads) {
        Sn[k] = aacc * b.dir[k];
        Yn[k] = gacc[k] - b.grad[k];
    }
    __syncthreads();
    const double sy = dot(Sn, Yn, n, sm.red);
    const double yy = dot(Yn, Yn, n, sm.red);
    double mx = 0.0;
    for (int k = tid; k < n; k += kStepThreads) {
        b.theta[k] += Sn[k];
        b.grad[k] = gacc[k];
        mx = fmax(mx, fabs(gacc[k]));
    }
    const double ginf = block_max(mx, sm.red);
    if (use_trial) update_precond(a);
    const bool keep = sy > 1e-12 * yy && sy > 0.0;   // curvature pair kept only if y's > 0
    const int hl = keep ? min(hl0 + 1, H) : hl0, hd = keep ? (head + 1) % H : head;
    if (tid == 0) {
        const double Lold = st->L;
        st->hist_head = hd;
        st->hist_len = hl;
        st->L = Lacc;
        st->L_sum = Lacc * N;
        st->grad_inf = ginf;
        st->it_lbfgs += 1;
        st->ls_restarts = 0;
        st->alpha0 = 1.0;
        if (ginf < 0.5 * st->ginf_best) {
            st->ginf_best = ginf;
            st->ev_best = st->evals;
        }
        st->stall = st->evals - st->ev_best;
        // Convergence (Sec. 2.9): every |dL/dtheta| below grad_tol, or the
        // limit of numerical precision: max|g| has not halved over the last
        // stall_iters evaluations (float32 pixel rounding sets a floor on the
        // gradient; once there, line searches fail and spend many
        // evaluations per step), or, if enabled, a relative loss change
        // below rel_tol.
        sm.finish_status = -1;
        sm.act = kStopNone;
        if (ginf < p.grad_tol) {
            sm.finish_status = 0; sm.act = kStopGradTol;
        } else if (at_floor(st, ginf)) {
            sm.finish_status = 0; sm.act = kStopFloor;
        } else if (p.rel_tol > 0.0 && fabs(Lold - Lacc) < p.rel_tol * fabs(Lacc)) {
            sm.finish_status = 0; sm.act = kStopRelTol;
        } else if (st->stall >= stall_limit(a)) {
            sm.finish_status = 0; sm.act = kStopStall;
        } else if (st->it_lbfgs >= p.max_lbfgs) {
            sm.finish_status = 4; sm.act = kStopMaxIter; /* DIA_ERR_MAXITER */
        } else if (st->evals >= p.max_evals) {
            sm.finish_status = 4; sm.act = kStopMaxEvals;
        }
    }
    __syncthreads();
    if (sm.finish_status >= 0) {
        finish(a, sm.finish_status, sm.act);
        return;
    }
    if (keep) {   // s_new . y_j and s_j . y_new over the history, the new pair included
        const int warp = tid >> 5, lane = tid & 31;
        constexpr int NWS = kStepThreads / 32;
        for (int t = warp; t < 2 * hl; t += NWS) {
            const int c = t < hl ? t : t - hl;
            const int j = hist_slot(c, hl, hd, H);
            const double v = t < hl ? warp_dot(Sn, b.Y + (size_t)j * n, n)
                                    : warp_dot(b.S + (size_t)j * n, Yn, n);
            if (lane == 0) {
                if (t < hl)
                    b.SY[(size_t)head * H + j] = v;
                else
                    b.SY[(size_t)j * H + head] = v;
            }
        }
        __syncthreads();
    }
    request_direction(a, keep ? head : -1);
}

__global__ void __launch_bounds__(kStepThreads) step_kernel(const StepArgs a) {
    __shared__ StepShared sm;
    step_body(a, sm);
}

__global__ void __launch_bounds__(kStepThreads) direction_kernel(const StepArgs a) {
    __shared__ StepShared sm;
    direction_body(a, sm);
}

// Batched step: CTA p reduces pair p's chunk partials (fixed order) and runs
// its optimiser step.  CTA 0 first resets the evaluation work queues.
__global__ void __launch_bounds__(kStepThreads)
    step_batch_kernel(const StepArgs *args, const BatchRed *red, const double *partials,
                      int *queue_counters, int n_counters) {
    if (blockIdx.x == 0 && threadIdx.x < n_counters) queue_counters[threadIdx.x] = 0;
    const StepArgs a = args[blockIdx.x];
    if (*((volatile int *)&a.st->done) != 0) return;
    const BatchRed r = red[blockIdx.x];
    for (int k = threadIdx.x; k < r.np; k += kStepThreads) {
        double t = 0.0;
        for (int c = 0; c < r.n_chunks; ++c) t += partials[r.part_off + (long long)c * r.np + k];
        r.red[k] = t;
    }
    __syncthreads();
    __shared__ StepShared sm;
    step_body(a, sm);
}

// Batched direction: the CTA of pair p applies P itself (one CTA holds a
// pair's P v easily; a grid of row blocks x pairs would mostly find nothing
// to do), then finishes the step.
__global__ void __launch_bounds__(kStepThreads) direction_batch_kernel(const StepArgs *args) {
    __shared__ StepShared sm;
    __shared__ __align__(16) float ws[2 * kPaW];
    const StepArgs a = args[blockIdx.x];
    pc_apply_body(a, 0, 1, ws);
    __syncthreads();
    direction_body(a, sm);
}

cudaError_t launch_step_batch(const StepArgs *args, const BatchRed *red, const double *partials,
                              int npairs, int *queue_counters, int n_counters, cudaStream_t s) {
    step_batch_kernel<<<npairs, kStepThreads, 0, s>>>(args, red, partials, queue_counters,
                                                      n_counters);
    direction_batch_kernel<<<npairs, kStepThreads, 0, s>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_step(const StepArgs &a, cudaStream_t s) {
    step_kernel<<<1, kStepThreads, 0, s>>>(a);
    cudaError_t e = launch_pc_apply(a, s);
    if (e != cudaSuccess) return e;
    direction_kernel<<<1, kStepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Initialisation: K box-car (1/m^2) or a normalised Gaussian (Sec. 2.9, Sec. 5.1),
// B0 = median of the unmasked valid target pixels; or theta already in place.
__device__ void init_body(FitState *st, OptBuffers b, float *Kpad, int mk, int kp, int nb,
                          int mode, double sigma, double median, int degenerate,
                          int start_phase, double *sh, int nc = 1) {
    // the constant part K_00 starts as the box-car / Gaussian kernel, the
    // other coefficient kernels of a spatially varying kernel at zero
    const int nk = mk * mk, nkt = nc * nk, n = nkt + nb, tid = threadIdx.x, h = mk / 2;
    if (mode == 0 || mode == 1) {
        double w = 0.0;
        for (int k = tid; k < nk; k += kStepThreads) {
            double v = 1.0;
            if (mode == 1) {
                const int a = k / mk - h, c = k % mk - h;
                v = exp(-(double)(a * a + c * c) / (2.0 * sigma * sigma));
            }
            b.theta[k] = v;
            w += v;
        }
        w = block_sum(w, sh);
        for (int k = tid; k < nk; k += kStepThreads) b.theta[k] /= w;
        for (int k = nk + tid; k < nkt; k += kStepThreads) b.theta[k] = 0.0;
        // B0 = median (Sec. 2.9); a polynomial background starts flat
        for (int k = nkt + tid; k < n; k += kStepThreads) b.theta[k] = (k == nkt) ? median : 0.0;
    }
    __syncthreads();
    for (int k = tid; k < n; k += kStepThreads) {
        b.trial[k] = b.theta[k];
        b.m1[k] = 0.0;
        b.m2[k] = 0.0;
    }
    __syncthreads();
    write_kpad(b.theta, mk, kp, nb, Kpad, tid, kStepThreads, nc);
    if (tid == 0) {
        FitState z;
        memset(&z, 0, sizeof(z));
        z.b1t = 1.0;
        z.b2t = 1.0;
        z.phase = start_phase;
        z.median = median;
        z.from_theta0 = (mode == 2) ? 1 : 0;
        z.alpha0 = 1.0;
        if (degenerate) {
            z.status = 6; /* DIA_ERR_DEGENERATE */
            z.reason = kStopDegenerate;
            z.phase = kPhaseDone;
            z.done = 1;
        }
        *st = z;
    }
}

__global__ void init_kernel(FitState *st, OptBuffers b, float *Kpad, int mk, int kp, int nb,
                            int mode, double sigma, const SelectState *sel, int start_phase,
                            int nc) {
    __shared__ double sh[kStepThreads / 32];
    init_body(st, b, Kpad, mk, kp, nb, mode, sigma, sel ? sel->median : 0.0,
              sel ? sel->degenerate : 0, start_phase, sh, nc);
}

cudaError_t launch_init(FitState *st, OptBuffers b, float *Kpad, int mk, int kp, int nb,
                        int init_mode, double init_sigma, const SelectState *sel,
                        int start_phase, cudaStream_t s, int nc) {
    init_kernel<<<1, kStepThreads, 0, s>>>(st, b, Kpad, mk, kp, nb, init_mode, init_sigma, sel,
                                           start_phase, nc);
    return cudaGetLastError();
}

// Restart the optimiser from the accepted theta (refit after clipping): the
// next evaluation at theta starts L-BFGS afresh.
__global__ void restart_kernel(FitState *st, float *Kpad, OptBuffers b, int mk, int kp, int nb,
                               int nc) {
    const int n = nc * mk * mk + nb;
    for (int k = threadIdx.x; k < n; k += blockDim.x) b.trial[k] = b.theta[k];
    __syncthreads();
    write_kpad(b.theta, mk, kp, nb, Kpad, threadIdx.x, blockDim.x, nc);
    if (threadIdx.x == 0) {
        st->done = 0;
        st->phase = kPhaseLbfgsStart;
        st->status = 0;
        st->hist_len = 0;
        st->hist_head = 0;
        st->ls_restarts = 0;
        st->need_pc = 0;
    }
}

cudaError_t launch_restart(FitState *st, float *Kpad, OptBuffers b, int mk, int kp, int nb,
                           cudaStream_t s, int nc) {
    restart_kernel<<<1, 256, 0, s>>>(st, Kpad, b, mk, kp, nb, nc);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Exact median by radix select over the order-preserving keys of the unmasked
// valid target pixels: three histogram passes (11, 11, 10 bits) per rank, for
// the two middle ranks (N-1)/2 and N/2; the median is their mean.
constexpr int kBins = 2048;

__global__ void hist_kernel(const float *__restrict__ I, const uint8_t *__restrict__ mask, int H,
                            int W, int ld, int h, uint32_t *__restrict__ hist,
                            const SelectState *sel, int slot, int pass) {
    __shared__ uint32_t sh[kBins];
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int Hv = H - 2 * h, Wv = W - 2 * h;
    const long long total = (long long)Hv * Wv;
    const uint32_t pre = (pass == 0) ? 0u : sel->prefix[slot];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / Wv), x = (int)(i - (long long)y * Wv);
        const size_t off = (size_t)(y + h) * ld + (x + h);
        if (mask && mask[off] == 0) continue;
        const uint32_t k = float_key(I[off]);
        uint32_t bin;
        if (pass == 0) {
            bin = k >> 21;
        } else if (pass == 1) {
            if ((k >> 21) != (pre >> 21)) continue;
            bin = (k >> 10) & 0x7ffu;
        } else {
            if ((k >> 10) != (pre >> 10)) continue;
            bin = k & 0x3ffu;
        }
        atomicAdd(&sh[bin], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__global__ void select_kernel(uint32_t *hist, SelectState *sel, int slot, int pass) {
    // one thread walks the bins (at most 2048)
    if (threadIdx.x == 0) {
        if (pass == 0 && slot == 0) {
            unsigned long long tot = 0;
            for (int i = 0; i < kBins; ++i) tot += hist[i];
            sel->count = tot;
            sel->degenerate = (tot == 0);
            sel->rank[0] = tot ? (uint32_t)((tot - 1) / 2) : 0u;
            sel->rank[1] = tot ? (uint32_t)(tot / 2) : 0u;
        }
        const int shift = (pass == 0) ? 21 : (pass == 1 ? 10 : 0);
        const int nb = (pass == 2) ? 1024 : 2048;
        uint32_t k = sel->rank[slot];
        unsigned long long cum = 0;
        int bin = nb - 1;
        for (int i = 0; i < nb; ++i) {
            if (cum + hist[i] > k) {
                bin = i;
                break;
            }
            cum += hist[i];
        }
        sel->rank[slot] = (uint32_t)(k - cum);
        sel->prefix[slot] = (pass == 0 ? 0u : sel->prefix[slot]) | ((uint32_t)bin << shift);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[i] = 0;
}

__device__ inline float key_float(uint32_t k) {
    const uint32_t u = (k & 0x80000000u) ? (k ^ 0x80000000u) : ~k;
    return __uint_as_float(u);
}

__global__ void median_finish_kernel(SelectState *sel) {
    if (threadIdx.x == 0)
        sel->median = sel->degenerate ? 0.0
                                      : 0.5 * ((double)key_float(sel->prefix[0]) +
                                               (double)key_float(sel->prefix[1]));
}

__global__ void zero_u32(uint32_t *p, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

cudaError_t launch_median(const float *I, const uint8_t *mask, int H, int W, int ld, int mk,
                          uint32_t *hist, SelectState *sel, int grid, cudaStream_t s) {
    const int h = mk / 2;
    zero_u32<<<1, 1024, 0, s>>>(hist, kBins);
    for (int slot = 0; slot < 2; ++slot)
        for (int pass = 0; pass < 3; ++pass) {
            hist_kernel<<<grid, 512, 0, s>>>(I, mask, H, W, ld, h, hist, sel, slot, pass);
            select_kernel<<<1, 1024, 0, s>>>(hist, sel, slot, pass);
        }
    median_finish_kernel<<<1, 32, 0, s>>>(sel);
    return cudaGetLastError();
}

// Median of the unmasked valid target pixels of one pair by one CTA: the
// same three-pass radix select over order-preserving keys, with the
// histogram in shared memory, for the two middle ranks.
__device__ void cta_median(const EvalArgs &ea, int h, unsigned *hist, double *out_median,
                           int *out_degenerate) {
    __shared__ unsigned long long s_count;
    __shared__ uint32_t s_rank[2], s_prefix[2];
    const int Hv = ea.H - 2 * h, Wv = ea.W - 2 * h;
    const long long total = (long long)Hv * Wv;
    for (int slot = 0; slot < 2; ++slot) {
        for (int pass = 0; pass < 3; ++pass) {
            for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            const uint32_t pre = (pass == 0) ? 0u : s_prefix[slot];
            for (long long i = threadIdx.x; i < total; i += blockDim.x) {
                const int y = (int)(i / Wv), x = (int)(i - (long long)y * Wv);
                const size_t off = (size_t)(y + h) * ea.ld + (x + h);
                if (ea.mask && ea.mask[off] == 0) continue;
                const uint32_t k = float_key(ea.I[off]);
                uint32_t bin;
                if (pass == 0) {
                    bin = k >> 21;
                } else if (pass == 1) {
                    if ((k >> 21) != (pre >> 21)) continue;
                    bin = (k >> 10) & 0x7ffu;
                } else {
                    if ((k >> 10) != (pre >> 10)) continue;
                    bin = k & 0x3ffu;
                }
                atomicAdd(&hist[bin], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                if (pass == 0 && slot == 0) {
                    unsigned long long tot = 0;
                    for (int i = 0; i < kBins; ++i) tot += hist[i];
                    s_count = tot;
                    s_rank[0] = tot ? (uint32_t)((tot - 1) / 2) : 0u;
                    s_rank[1] = tot ? (uint32_t)(tot / 2) : 0u;
                }
                const int shift = (pass == 0) ? 21 : (pass == 1 ? 10 : 0);
                const int nb = (pass == 2) ? 1024 : 2048;
                const uint32_t k = s_rank[slot];
                unsigned long long cum = 0;
                int bin = nb - 1;
                for (int i = 0; i < nb; ++i) {
                    if (cum + hist[i] > k) {
                        bin = i;
                        break;
                    }
                    cum += hist[i];
                }
                s_rank[slot] = (uint32_t)(k - cum);
                s_prefix[slot] = (pass == 0 ? 0u : s_prefix[slot]) | ((uint32_t)bin << shift);
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        *out_degenerate = (s_count == 0);
        *out_median = s_count ? 0.5 * ((double)key_float(s_prefix[0]) + (double)key_float(s_prefix[1]))
                              : 0.0;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kStepThreads)
    init_batch_kernel(const StepArgs *args, const EvalArgs *eas, int mode, double sigma,
                      int start_phase) {
    __shared__ unsigned hist[kBins];
    __shared__ double sh[kStepThreads / 32];
    __shared__ double s_med;
    __shared__ int s_deg;
    const StepArgs a = args[blockIdx.x];
    const EvalArgs ea = eas[blockIdx.x];
    if (mode != 2) {
        cta_median(ea, a.mk / 2, hist, &s_med, &s_deg);
    } else if (threadIdx.x == 0) {
        s_med = 0.0;
        s_deg = 0;
    }
    __syncthreads();
    init_body(a.st, a.b, a.Kpad, a.mk, a.kp, a.n - a.mk * a.mk, mode, sigma, s_med, s_deg,
              start_phase, sh);
    if (threadIdx.x == 0 && s_deg && a.n_done) atomicAdd(a.n_done, 1);   // finished at once
}

cudaError_t launch_init_batch(const StepArgs *args, const EvalArgs *eas, int npairs, int init_mode,
                              double init_sigma, int start_phase, cudaStream_t s) {
    init_batch_kernel<<<npairs, kStepThreads, 0, s>>>(args, eas, init_mode, init_sigma,
                                                      start_phase);
    return cudaGetLastError();
}

__global__ void pack_batch_kernel(const StepArgs *args, const long long *theta_off,
                                  double *theta_out) {
    const StepArgs a = args[blockIdx.x];
    for (int k = threadIdx.x; k < a.n; k += blockDim.x)
        theta_out[theta_off[blockIdx.x] + k] = a.b.theta[k];
}

cudaError_t launch_pack_batch(const StepArgs *args, const long long *theta_off, double *theta_out,
                              int npairs, cudaStream_t s) {
    pack_batch_kernel<<<npairs, 256, 0, s>>>(args, theta_off, theta_out);
    return cudaGetLastError();
}

// K_out: the constant kernel (K_00, the kernel at the image centre, for a
// spatially varying one); b0_out: b_00
__global__ void pack_kernel(const double *theta, int mk, int nb, double *theta_out, float *K_out,
                            float *b0_out, int nc) {
    const int nk = mk * mk, nkt = nc * nk, n = nkt + nb;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        if (theta_out) theta_out[k] = theta[k];
        if (K_out && k < nk) K_out[k] = (float)theta[k];
    }
    if (threadIdx.x == 0 && b0_out) *b0_out = (float)theta[nkt];
}

cudaError_t launch_pack_outputs(const double *theta, int mk, int nb, double *theta_out,
                                float *K_out, float *b0_out, cudaStream_t s, int nc) {
    pack_kernel<<<1, 256, 0, s>>>(theta, mk, nb, theta_out, K_out, b0_out, nc);
    return cudaGetLastError();
}

}  // namespace dia

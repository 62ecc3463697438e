// Small kernels around the fused evaluation: the float64 cross-CTA reduction,
// the on-device optimiser (Adam, then L-BFGS with a Wolfe / approximate-Wolfe
// line search and a Gauss-Newton preconditioner, Sec. 2.3 and Sec. 2.9),
// initialisation (box-car or Gaussian kernel, B0 =
// median of the target, Sec. 2.9) and output packing.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dia_eval.cuh"

namespace dia {

constexpr int kHistMax = 128;  // largest L-BFGS memory
// largest theta of a fit: m <= 31 with the largest background (976), and a
// spatially varying kernel whose nc m^2 + background coefficients fit
constexpr int kMaxN = 1024;
constexpr int kPcMaxN = kMaxN;

enum Phase { kPhaseAdam = 0, kPhaseLbfgs = 1, kPhaseLbfgsStart = 2, kPhaseDone = 3 };

// Why a fit pass stopped (FitState::reason, dia_fit_info::reason).
enum StopReason {
    kStopNone = 0, kStopGradTol = 1, kStopRelTol = 2, kStopStall = 3, kStopLineSearch = 4,
    kStopMaxIter = 5, kStopMaxEvals = 6, kStopNonfinite = 7, kStopDegenerate = 8,
    kStopFloor = 9
};

// Optimiser state, float64, resident in the caller's workspace.  The first
// fields are read back by the host after every graph launch.
struct FitState {
    int done;        // 1 once the fit pass has finished (evaluation kernels exit early)
    int phase;       // Phase
    int status;      // dia_status of the pass
    int it_adam, it_lbfgs, evals;
    int ls_evals, hist_len, hist_head, ls_restarts, stall, reason;
    int pc_ok;       // 1: the Gauss-Newton preconditioner is factored and used
    int ev_best;     // evals when max|g| last halved (stall detection)
    int need_pc;     // new L-BFGS direction pending: 1 needs P g, 2 also P y_new
    int pc_slot;     // history slot of y_new (need_pc == 2)
    int from_theta0; // 1: the fit started from the caller's theta (no progress test)
    double ndata;    // unmasked valid pixels of the last evaluation
    double L;        // scaled loss (L_sum / N) at the accepted theta
    double L_sum;    // unscaled loss at the accepted theta
    double grad_inf; // max |g| of the scaled loss at the accepted theta
    double ginf_best; // smallest grad_inf so far (stall detection)
    double L_prev;   // previous Adam loss
    double gd0;      // phi'(0) of the current line search
    double alpha;    // step being evaluated
    double lo, L_lo, gd_lo, hi, L_hi, gd_hi;  // line-search bracket (hi < 0: none yet)
    double b1t, b2t; // Adam beta powers
    double median;   // B0 initialisation
    double ginf_floor; // best max|g| of the last pass that ended at the precision limit (0: none)
    double ginf_first; // max|g| of the fit's first evaluation
    double alpha0;     // scale of the first trial step of a search without history (restarts)
};

struct OptParams {
    double lr_kernel, lr_b0, beta1, beta2, adam_eps, switch_tol;
    double rel_tol, grad_tol;
    double reg_lambda;   // kernel regulariser of Eq. 20 (0 = off)
    int max_adam, history, max_lbfgs, max_evals, stall_iters, stall_iters_diag, max_ls;
};

// Float64 vectors of the optimiser (n = m*m + 1 each).  L-BFGS history in
// slots of a ring of `history` entries: S, Y and PY = P y are history x n;
// SY[i][j] = s_i.y_j and YPY[i][j] = y_i.P y_j are history x history (the
// compact representation of Byrd, Nocedal & Schnabel 1994).  pg = P g for the
// current gradient; pdiag is the diagonal preconditioner, an approximate
// inverse Hessian diagonal.
struct OptBuffers {
    double *theta, *trial, *grad, *glo, *m1, *m2, *dir, *pg, *pdiag;
    double *S, *Y, *PY, *SY, *YPY;
    // Gauss-Newton preconditioner (nullable): P = H^-1, n x n float32, row
    // pitch ldp (a multiple of 4); used when FitState::pc_ok is set
    const float *P;
    int ldp;
};

struct StepArgs {
    FitState *st;
    OptBuffers b;
    const double *red;   // reduced partials: loss, dK[m*m], dB0, count, sum kR^2, sum k
    float *Kpad;         // float32 copy of the trial theta for the next evaluation
    int n, mk, kp;
    OptParams p;
    int *n_done;         // nullable: incremented once when the fit finishes (batched fits)
    int nc;              // kernel coefficient sets (a spatially varying kernel; 0 or 1: one)
};

// Order-preserving map float -> uint32 (for the radix-select median).
__host__ __device__ inline uint32_t float_key(float f) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

struct SelectState {
    uint32_t prefix[2];
    uint32_t rank[2];
    unsigned long long count;
    int degenerate;
    double median;
};

// Batched fits: the partial sums of pair p's work items (chunks of its
// tiles) sit at part_off + c * np for c < n_chunks; the step kernel of pair p
// sums them in chunk order into red.
struct BatchRed {
    long long part_off;
    int n_chunks, np;
    double *red;
};

// Preconditioner of L-BFGS: the Gauss-Newton Hessian of the per-pixel loss
// over a window of valid pixels p (valid-region coordinates [y0, y1) x
// [x0, x1)), H = sum_p w_p phi_p phi_p^T / N_window with phi_p = [R window of
// p, 1] and w_p = mask / (pixel variance at M = I); then P = H^-1.
struct PrecondArgs {
    const float *R, *I;
    const uint8_t *mask;
    const float *var, *flat;
    int H, W, ld, m;
    int y0, y1, x0, x1;   // window of valid-region coordinates
    LossParams lp;
    double *part;         // gn_chunks x gn_blocks(n) x 64 x 64 partial sums (gn_chunks > 1)
    int gn_chunks;        // pixel chunks the Hessian sum is split into
    double *A64;          // np x np (np = n rounded up to 64): H, then its Cholesky factor
    double *X64;          // np x np: the inverse of the factor
    float *P;             // n x ldp: H^-1, the preconditioner
    int ldp;
    FitState *st;         // receives pc_ok
    double eps;           // relative diagonal regularisation of H
    double reg2;          // 2 lambda: H += 2 lambda L^T L, the regulariser of Eq. 20 (0 = off)
    int nbg;              // background coefficients (1: the constant B0)
    int kdeg;             // degree of a spatially varying kernel (0: one kernel); its
                          // design columns are eta^p xi^q R windows (Eq. 19 coordinates)
    float eta0, eta_s, xi0, xi_s;   // Eq. 19 coordinates of valid-region pixels (EvalArgs)
    double scale;         // H is scaled by this (1 / window pixels for the preconditioner)
    int flush;            // shared-memory batches of 32 px per float64 flush
    int wmap_ld;
    const float *wmap;    // nullable: per-pixel weights (valid-region coordinates, pitch
                          // wmap_ld) instead of mask / variance
    double *F_out;        // nullable: n x n float64 copy of H (before factorisation)
    double *cov_out;      // nullable: n x n float64 H^-1 (then P is not written)
};

constexpr int kPcB = 32;    // block size of the factorisation
constexpr int kGnT = 64;    // block size of the Hessian sum
constexpr int kGnChunk = 16384;   // pixels per chunk of the Hessian sum
constexpr int kGnFlushPc = 16;    // 32-px batches per float64 flush for the preconditioner
__host__ __device__ inline int pc_np(int n) { return (n + kGnT - 1) / kGnT * kGnT; }
__host__ __device__ inline int pc_n(const PrecondArgs &a) {
    return n_background(a.kdeg) * a.m * a.m + a.nbg;
}
__host__ __device__ inline int pc_ldp(int n) { return (n + 3) & ~3; }
__host__ __device__ inline int gn_tiles(int n) { return (n + kGnT - 1) / kGnT; }
__host__ __device__ inline int gn_blocks(int n) { return gn_tiles(n) * (gn_tiles(n) + 1) / 2; }
// Window side for a kernel of n parameters: about 1.2e11 / n^2 pixels (a few
// ms of FP32 work), between 256^2 and 1024^2.
inline int pc_window_side(int n) {
    double s = 0.0;
    const double t = 1.2e11 / ((double)n * n);
    while ((s + 32.0) * (s + 32.0) <= t) s += 32.0;
    return s < 256.0 ? 256 : (s > 1024.0 ? 1024 : (int)s);
}

// ---------------------------------------------------------------- P v
// For a fit with a direction pending: pg = P g, and PY[slot] = P y_new when
// need_pc == 2.  P is applied as a dense float32 matrix (warp per row; rows
// strided over CTAs blk of nblk), or, without the factorisation, as the
// diagonal pdiag.  Block size kPaThreads.
constexpr int kPaThreads = 256;
constexpr int kPaRowsPerCta = kPaThreads / 32;
constexpr int kPaW = (kPcMaxN + 7) & ~3;   // staged vector length (16-byte multiple)

__device__ __forceinline__ void pc_apply_body(const StepArgs &a, int blk, int nblk, float *ws) {
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


// host launchers (dia_ops.cu)
cudaError_t launch_reduce(const double *partials, int G, int NP, double *out, const int *done,
                          cudaStream_t s, int acc32 = 0);
// nb: background coefficients of the pair (1 for the constant B0)
// nc: kernel coefficient sets (spatially varying kernel), 1 otherwise
cudaError_t launch_prep_kpad(const double *theta, int mk, int kp, int nb, float *Kpad,
                             cudaStream_t s, int nc = 1);
cudaError_t launch_emit_loss_grad(const double *red, int mk, int nb, double *loss, double *grad,
                                  cudaStream_t s, int nc = 1);
// One optimiser step: the line-search / history half (one CTA), P g and
// P y_new (many CTAs), the direction half (one CTA).
constexpr int kStepLaunches = 3;
cudaError_t launch_step(const StepArgs &a, cudaStream_t s);
// d_pas: device array of npairs descriptors; h_pas: the same on the host
cudaError_t launch_precond(const PrecondArgs *d_pas, const PrecondArgs *h_pas, int npairs,
                           cudaStream_t s);
int precond_launches(int max_n);   // kernels one launch_precond call enqueues (largest n)
// Observed Fisher information (dia_fisher.cu): w[p] <- d2l/dM2 at M = I - D for
// the valid pixels (D = the difference image held in w on entry; 0 where masked)
cudaError_t launch_fisher_weights(const EvalArgs &ea, float *w, unsigned long long *count,
                                  cudaStream_t s);
// res[0] = log det H, res[1] = smallest pivot of its Cholesky factor (squared)
cudaError_t launch_fisher_finish(const double *A64, int n, int np, double *res, cudaStream_t s);
void precond_window(int H, int W, int m, bool single, int side, int *y0, int *y1, int *x0,
                    int *x1, int *chunks);
// Tensor-core forward pass (dia_tc.cu): D = I - M over the valid region with the
// correlation on tcgen05 (split bf16, float32 accumulators in tensor memory);
// constant background B0 = Kpad[m * kp].  *status is set to 1 if a bounded wait
// ran out.
// wait_cycles: limit of each pipeline wait (0: about one second)
cudaError_t launch_tc_forward(const float *R, const float *I, int H, int W, int ld, int m,
                              const float *Kpad, int kp, float *diff_out, int *status,
                              cudaStream_t s, long long wait_cycles = 0);
// The same pass in loss mode: instead of D, g = dl/dM into gmap (gmap_rows
// rows of pitch gld, at least the tiles' padded height and width; rows of the
// tiles past the valid region get 0),
// partial rows [0, rows) of loss, dL/dB0, pixel count and curvature sums
// (np = red_size(m*m) doubles each, 0 in the other slots), and max |R|,
// max |g| (float bits) into amax[0..1] (zeroed by the caller)
cudaError_t launch_tc_forward_gmap(const EvalArgs &ea, int m, const float *Kpad, int kp,
                                   float *gmap, int gld, int gmap_rows, double *partials, int np,
                                   int rows, unsigned *amax, int *status, cudaStream_t s,
                                   long long wait_cycles = 0, const int *done = nullptr);
// sets the tensor-core forward kernels' shared-memory attribute (D mode and
// the loss mode of (rho, var_model)) so that later launches, also inside a
// graph capture, need no attribute call
cudaError_t tc_forward_prepare(int rho, int var_model);
// P g (and P y_new) for every fit with a direction pending (dia_precond.cu)
cudaError_t launch_pc_apply(const StepArgs &a, cudaStream_t s);
cudaError_t launch_init(FitState *st, OptBuffers b, float *Kpad, int mk, int kp, int nb,
                        int init_mode, double init_sigma, const SelectState *sel,
                        int start_phase, cudaStream_t s, int nc = 1);
cudaError_t launch_restart(FitState *st, float *Kpad, OptBuffers b, int mk, int kp, int nb,
                           cudaStream_t s, int nc = 1);
constexpr int kMedianLaunches = 14;   // kernels launch_median enqueues
cudaError_t launch_median(const float *I, const uint8_t *mask, int H, int W, int ld, int mk,
                          uint32_t *hist, SelectState *sel, int grid, cudaStream_t s);
cudaError_t launch_pack_outputs(const double *theta, int mk, int nb, double *theta_out,
                                float *K_out, float *b0_out, cudaStream_t s, int nc = 1);
// batched: one CTA per pair for the two optimiser halves, P v inside the
// second (kStepLaunchesBatch kernels)
constexpr int kStepLaunchesBatch = 2;
cudaError_t launch_step_batch(const StepArgs *args, const BatchRed *red, const double *partials,
                              int npairs, int *queue_counters, int n_counters, cudaStream_t s);
cudaError_t launch_init_batch(const StepArgs *args, const EvalArgs *eas, int npairs,
                              int init_mode, double init_sigma, int start_phase, cudaStream_t s);
cudaError_t launch_pack_batch(const StepArgs *args, const long long *theta_off, double *theta_out,
                              int npairs, cudaStream_t s);

}  // namespace dia

/*
 * dia.h -- C ABI of the GB300 (sm_103a) DIA kernel-fit library.
 *
 * The library fits the model image of Bramich (2008) as used by PyTorchDIA
 * (arXiv 2104.13715):
 *
 *     M_ij = sum_{l,m} K_lm R_(i+l)(j+m) + B_ij               (Sec. 2.1, Eq. 2)
 *
 * with a constant background B_ij = B0 or the polynomial of Sec. 2.6 (Eq. 18)
 *
 * to a target image I by minimising a per-pixel negative log-likelihood
 * (Sec. 2.3, Eq. 8; Sec. 2.4, Eq. 13) with Adam followed by L-BFGS
 * (Sec. 2.3, Sec. 2.9).  Every step of the fit runs in this library's own
 * CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Images: float32, row-major, H rows by W columns, row pitch `ld` elements
 *   (ld >= W).  The reference R, target I and the optional per-pixel maps
 *   (mask, fixed variance, flat field) share H, W and ld; the mask is one
 *   byte per pixel with the same pitch in elements (= bytes).
 * Kernel: odd side m = 2h+1, 1 <= m <= min(H, W), m <= DIA_MAX_M.
 *   K[a][b] (a, b in [0, m)) multiplies R[i-h+a][j-h+b] for the target pixel
 *   (i, j): centred offsets l = a-h, m = b-h as in Eq. 2.  A target moved by
 *   +1 pixel in x and y is fitted by a delta at a = b = h-1 (Sec. 3.4 iii).
 * Valid region: only pixels with i in [h, H-h) and j in [h, W-h) enter the
 *   loss (Sec. 2.1: the convolution is undefined within half a kernel width
 *   of the edge); the difference image covers exactly that region,
 *   (H-2h) x (W-2h), row-major, dense, its (0,0) at pixel (h, h).
 * Background: a pair's bg_degree d (0 <= d <= DIA_MAX_BG_DEGREE) selects
 *   B = sum_{p=0..d} sum_{q=0..d-p} b_pq eta^p xi^q (Eq. 18) with the
 *   normalised coordinates of Eq. 19, eta = (x - x_c)/N_x, xi = (y - y_c)/N_y:
 *   x = column j and y = row i of the full image, x_c = (W-1)/2,
 *   y_c = (H-1)/2, N_x = W, N_y = H.  d = 0 is the constant B0 = b_00.
 * theta: float64 vector of n = m*m + (d+1)(d+2)/2 entries: K row-major, then
 *   b_00, b_01, ..., b_0d, b_10, ..., b_d0 (power of xi fastest, the order of
 *   the double sum of Eq. 18); n = m*m + 1 (K, then B0) for d = 0.  b_00 is the
 *   background at the image centre.
 * Spatially varying kernel: a pair's kernel_degree dk (0 <= dk <=
 *   DIA_MAX_KERNEL_DEGREE) makes every kernel pixel a polynomial of degree dk
 *   in the same coordinates, K_ab(x, y) = sum_{p+q<=dk} K_pq[a][b] eta^p xi^q,
 *   evaluated at the output pixel (the extension Sec. 1 cites, in the Bramich
 *   et al. 2013 form); theta then holds nc = (dk+1)(dk+2)/2 kernels of m*m
 *   (K_00, K_01, ..., K_dk0, the order of Eq. 18) before the background
 *   coefficients: n = nc*m*m + (d+1)(d+2)/2.  K_00 is the kernel at the image
 *   centre.  dk = 0 is the constant kernel.
 * Mask: nonzero = use the pixel, 0 = masked.  The mask refers to target
 *   pixels; a bad reference pixel must be masked (dilated by h) by the caller.
 * Memory: unless a pair says DIA_MEM_HOST, every pointer is a DEVICE pointer
 *   owned by the caller.  The library never frees or keeps caller memory and
 *   allocates no device memory inside these calls: all scratch lives in the
 *   caller's `workspace` (size from dia_workspace_size()).  It does create
 *   and cache, per host thread, one internal stream and CUDA graphs.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *   work is ordered on it; dia_fit and dia_fit_batch return after the fit
 *   (they wait on the stream to poll the convergence flag); dia_loss_grad
 *   and dia_diff_image are asynchronous.
 * Errors: every entry returns a dia_status and never aborts or throws.
 *   Arguments are validated before any launch (DIA_ERR_ARG).  A CUDA error
 *   is reported as DIA_ERR_CUDA; dia_last_cuda_error() gives its code.
 */
#ifndef DIA_H
#define DIA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DIA_MAX_M 31           /* largest odd kernel side of the fused kernels */
#define DIA_MAX_BG_DEGREE 4    /* largest degree of the polynomial background */
#define DIA_MAX_KERNEL_DEGREE 2 /* largest degree of a spatially varying kernel */
#define DIA_ABI_VERSION 4

typedef enum {
    DIA_OK = 0,
    DIA_ERR_ARG = 1,           /* invalid argument (checked before any launch) */
    DIA_ERR_CUDA = 2,          /* a CUDA call failed */
    DIA_ERR_NONFINITE = 3,     /* loss or gradient became NaN/Inf */
    DIA_ERR_MAXITER = 4,       /* iteration cap reached; outputs hold the last theta */
    DIA_ERR_LINESEARCH = 5,    /* L-BFGS line search found no decrease */
    DIA_ERR_DEGENERATE = 6,    /* no usable pixel (all masked) */
    DIA_ERR_TIMEOUT = 7,       /* host wall-clock limit while polling */
    DIA_ERR_WORKSPACE = 8,     /* workspace too small or misaligned */
    DIA_ERR_UNSUPPORTED = 9    /* e.g. m > DIA_MAX_M */
} dia_status;

/* Loss shape rho(z) of the pixel residual z = (I - M)/sigma. */
typedef enum {
    DIA_RHO_GAUSS = 0,         /* z^2/2                        (Eq. 8)  */
    DIA_RHO_HUBER = 1,         /* Huber with threshold c       (Eq. 12) */
    DIA_RHO_CAUCHY = 2         /* ln(1 + z^2), the Student-t nu=1 drop-in (Sec. 2.4) */
} dia_rho;

/* Pixel variance sigma^2. */
typedef enum {
    DIA_VAR_FIXED = 0,         /* var map, else var_scalar; ln sigma dropped (constant) */
    DIA_VAR_CCD = 1,           /* sigma0^2/F^2 + M/(G F)       (Eq. 6) */
    DIA_VAR_EMCCD = 2          /* E M/(G F), G = G_total       (Eq. 7) */
} dia_var_model;

typedef struct {
    int32_t rho;               /* dia_rho */
    int32_t var_model;         /* dia_var_model */
    float sigma0;              /* read noise (image units), CCD */
    float gain;                /* G (CCD) or G_total (EMCCD), > 0 */
    float excess;              /* EMCCD excess noise factor E (paper: 2) */
    float huber_c;             /* Huber threshold c (paper: 1.345) */
    float var_scalar;          /* fixed variance when the pair has no var map (> 0) */
    float var_floor;           /* model-dependent variance clamp (> 0); where
                                  clamped, dsigma^2/dM is taken as 0 */
} dia_loss_spec;

typedef enum { DIA_MEM_DEVICE = 0, DIA_MEM_HOST = 1 } dia_mem;

/* One reference/target pair. */
typedef struct {
    const float *ref;          /* R, H x W pitch ld (background-subtracted, Sec. 2.9) */
    const float *img;          /* I, H x W pitch ld */
    const uint8_t *mask;       /* nullable: every pixel used */
    const float *var;          /* nullable: fixed variance map (DIA_VAR_FIXED) */
    const float *flat;         /* nullable: flat field F (CCD/EMCCD), else 1 */
    int32_t H, W, ld;
    int32_t m;                 /* odd kernel side */
    int32_t mem;               /* dia_mem: where the pointers above AND the
                                  outputs of the call live */
    int32_t bg_degree;         /* degree d of the background polynomial (Eq. 18);
                                  0 = constant B0 */
    int32_t kernel_degree;     /* degree dk of a spatially varying kernel (0 = one
                                  kernel for the whole image); dia_loss_grad,
                                  dia_diff_image, dia_fit and dia_fisher take dk > 0
                                  (with reg_lambda = 0); the other entries return
                                  DIA_ERR_UNSUPPORTED */
} dia_pair;

/* Optimiser settings (Sec. 2.9).  dia_opts_default() fills the paper's
 * values; a NULL dia_opts* means those defaults. */
typedef struct {
    double lr_kernel;          /* Adam learning rate of the kernel pixels (1e-3) */
    double lr_b0;              /* Adam learning rate of B0 and of the other background
                                  coefficients (10; the paper uses 1, 10 or 100) */
    double beta1, beta2;       /* Adam moment decays (0.9, 0.999) */
    double adam_eps;           /* Adam epsilon (1e-8) */
    double switch_tol;         /* |dL/L| between Adam steps that hands over to L-BFGS (1e-6) */
    int32_t max_adam_iters;    /* Adam step cap (5000) */
    int32_t history;           /* L-BFGS memory (20, at most 128) */
    double rel_tol;            /* if > 0: stop when |dL/L| between L-BFGS steps < rel_tol
                                  (0 = off: the loss is flat along ill-conditioned kernel
                                  directions, so this test can stop far from the optimum) */
    double grad_tol;           /* stop when every |dL/dtheta_k| / N_data < grad_tol (1e-7) */
    int32_t max_lbfgs_iters;   /* L-BFGS iteration cap (3000) */
    int32_t max_evals;         /* cap on loss+gradient evaluations per fit, all passes (20000) */
    int32_t clip_passes;       /* sigma-clip-and-refit passes after the first fit (0) */
    float clip_kappa;          /* clip |z| > kappa (5, Sec. 4.2) */
    int32_t init;              /* 0: box-car K = 1/m^2, 1: Gaussian of init_sigma,
                                  2: theta0; B0 = median of the unmasked valid I
                                  for 0 and 1 (Sec. 2.9), the other background
                                  coefficients 0 */
    double init_sigma;         /* Gaussian init width phi_K (px) */
    const double *theta0;      /* HOST pointer, n entries, used when init == 2 */
    int32_t graph_iters;       /* optimiser iterations per CUDA-graph launch (16) */
    double timeout_s;          /* host polling limit per fit (600 s) */
    int32_t stall_iters;       /* limit of numerical precision: stop when max|dL/dtheta| has
                                  not halved over this many loss+gradient evaluations of
                                  the L-BFGS phase (30) */
    int32_t use_graph;         /* 1: replay optimiser iterations from a CUDA graph (default);
                                  0: launch them one by one (the plain form) */
    int32_t precond;           /* L-BFGS initial inverse Hessian: 1 = the inverse of the
                                  Gauss-Newton Hessian over a window of target pixels
                                  (default), 0 = diagonal */
    int32_t stall_iters_diag;  /* stall_iters when L-BFGS runs with the diagonal
                                  preconditioner (precond = 0, or the Gauss-Newton
                                  factorisation failed), which converges far more slowly
                                  (1000) */
    int32_t max_ls_evals;      /* evaluations one line search may take before it gives up
                                  (restart from preconditioned steepest descent, twice at
                                  most, then stop) (12) */
    int32_t precond_window;    /* side of the centred window of target pixels whose
                                  Gauss-Newton Hessian is the preconditioner; 0 = automatic
                                  (about sqrt(1.2e11) / n, between 256 and 1024; 544 at
                                  m = 25) (0) */
    double reg_lambda;         /* lambda of the kernel regulariser of Sec. 2.7 (Eq. 20):
                                  minimise L0 + lambda N_data theta^T L^T L theta, L the
                                  Laplacian of the kernel-pixel graph (Eq. 21, kernel
                                  pixels sharing an edge are adjacent; B0 is not
                                  penalised); 0 = off (0) */
} dia_opts;

typedef struct {
    int32_t status;            /* dia_status of the fit */
    int32_t adam_iters, lbfgs_iters, evals;
    int32_t clip_passes_done;
    int64_t ndata;             /* unmasked valid pixels at the end (N_data) */
    double loss;               /* final objective, sum over pixels (float64; with
                                  reg_lambda > 0 the regulariser of Eq. 20 included) */
    double grad_inf;           /* max |dL/dtheta| / N_data at the end */
    double scale;              /* photometric scale P = sum K (Eq. 3) */
    double b0;                 /* fitted B0 (b_00: the background at the image centre) */
    int32_t reason;            /* why the last pass stopped: 1 grad_tol, 2 rel_tol, 3 stall
                                  (precision limit), 4 line search, 5 max iterations,
                                  6 max evaluations, 7 non-finite, 8 degenerate, 9 a
                                  refit reached (within 3x) the max|dL/dtheta| floor of
                                  an earlier pass of the same fit */
    int64_t kernel_launches;   /* CUDA kernels this call launched (graph nodes included) */
    int32_t precond_used;      /* 1: L-BFGS ran with the Gauss-Newton preconditioner
                                  (asked for and factored), 0: with the diagonal one */
} dia_fit_info;

/* Human-readable status name (static string). */
const char *dia_status_str(int32_t status);

/* Version of this ABI (DIA_ABI_VERSION). */
int32_t dia_abi_version(void);

/* CUDA error code of the last DIA_ERR_CUDA on this host thread (0 if none).
 * A tensor-core kernel's own bounds check reports -2 (forward pass) or -3
 * (weight gradient) here: an index outside its buffers was skipped. */
int32_t dia_last_cuda_error(void);

/* Where the library caught that error: the source line of its C-ABI file
 * (0 if none), for bug reports. */
int32_t dia_last_cuda_error_site(void);

/* Fill `opts` with the paper's defaults (values in the field comments). */
dia_status dia_opts_default(dia_opts *opts);

/* Tile variants of the fused kernel (shape choices of the same computation:
 * warps per CTA, output rows per warp; the autotuner picks one per kernel
 * side and image size).  dia_kernel_variants(m) is their number (0 if m is
 * unsupported); dia_select_kernel_variant(m, v) makes variant v the one every
 * later call with kernel side m uses (process-wide, default 0; not safe to
 * change while another host thread is launching work of the same m);
 * dia_kernel_variant_desc(m, v, ...) describes variant v (v < 0: the
 * selected one); output pointers are nullable host pointers.  Results of all
 * variants agree up to the order of float32 tile sums. */
int32_t dia_kernel_variants(int32_t m);

/* Accumulation of the per-pixel loss and gradient terms (the precision
 * study of the high-dynamic-range workload compares the two forms):
 *   DIA_ACCUM_FP64 (default) -- float32 per-lane runs of at most 4096 pixels,
 *     Kahan-compensated float32 per tile run for dL/dK, float64 across tiles,
 *     warps and CTAs;
 *   DIA_ACCUM_FP32 -- float32 everywhere without compensation, a comparison
 *     form for the precision study, not for production.
 * Process-wide; applies to dia_loss_grad and dia_fit from the next call on
 * (not to dia_fit_batch or dia_loss_grad_noalloc); the optimiser's own
 * arithmetic stays float64.  Not safe to change while another host thread
 * launches work. */
#define DIA_ACCUM_FP64 0
#define DIA_ACCUM_FP32 1
dia_status dia_set_accumulation(int32_t mode);
int32_t dia_get_accumulation(void);

/* Form of the gradient-mode evaluations (loss and dL/dtheta, Eq. 8 / Eq. 13)
 * of dia_loss_grad, dia_fit and dia_time_eval:
 *   DIA_EVAL_FP32 (default) -- the fused float32 CUDA-core kernels;
 *   DIA_EVAL_TC -- both contractions on the tensor cores, the kernels of
 *     dia_loss_grad_tc (split-precision products, float64 across tiles),
 *     wherever they apply: m <= 31, constant background, one kernel
 *     (bg_degree = kernel_degree = 0); elsewhere the float32 form runs;
 *   DIA_EVAL_AUTO -- the tensor-core form where it applies and was measured
 *     faster than the float32 form (19 <= m <= 31: 1.27x at m = 19, 1.38x at
 *     m = 25, 1.9x at m = 31 for a 4096^2 pair; slower below m = 15), the
 *     float32 form elsewhere.
 * While DIA_EVAL_TC is set, dia_workspace_size and dia_pair_workspace_size
 * include its g map (the valid region padded to multiples of 128), two
 * partial rows per SM and a status word: size the workspace after choosing
 * the form.  dia_loss_grad then waits on its stream to read the status word;
 * a bounded wait of a tensor-core kernel that ran out is reported as
 * DIA_ERR_TIMEOUT (by dia_fit at its end).  The optimiser, the
 * preconditioner, sigma clipping and the outputs are the same in both forms.
 * Process-wide; not safe to change while another host thread launches work.
 * Returns DIA_ERR_ARG for any other value. */
#define DIA_EVAL_FP32 0
#define DIA_EVAL_TC 1
#define DIA_EVAL_AUTO 2
dia_status dia_set_eval_form(int32_t form);
int32_t dia_get_eval_form(void);
/* Streaming form of the fused evaluation for small kernels (m = 1, 3, 5: the
 * memory-bound end of the kernel-size sweep of Sec. 5.3, where each pixel
 * costs 2 m^2 FMAs against 8-17 bytes of input).  Enabled (1, default), the
 * gradient-mode evaluations of dia_loss_grad and dia_fit use it whenever it
 * applies: m <= 5, constant background, DIA_ACCUM_FP64, 16-byte aligned
 * images with a row pitch that is a multiple of 4 floats (of 16 bytes when a
 * mask is given; dia_fit's clipping mask has the pair's pitch); otherwise,
 * and with 0, the tiled kernel runs.  Each warp streams a strip of rows
 * through a private shared-memory ring (cp.async) and keeps the R window in
 * registers; per-lane float32 sums over one strip (at most 4096 pixels),
 * float64 across lanes, warps and CTAs.  Process-wide; not safe to change
 * while another host thread launches work.  Returns DIA_ERR_ARG unless
 * enable is 0 or 1. */
dia_status dia_set_small_kernel(int32_t enable);
int32_t dia_get_small_kernel(void);
dia_status dia_select_kernel_variant(int32_t m, int32_t variant);
dia_status dia_kernel_variant_desc(int32_t m, int32_t variant, int32_t *warps,
                                   int32_t *rows_per_warp, int32_t *tile_rows,
                                   int32_t *smem_bytes);

/* Workspace bytes needed by dia_loss_grad / dia_fit / dia_diff_image for an
 * H x W image of row pitch ld, kernel side m, with `clip` != 0 if dia_fit
 * will clip (clip_passes > 0) or return a mask, and `mem` = DIA_MEM_HOST if
 * the pair's buffers are on the host (the images are then staged through the
 * workspace).  Returns 0 for invalid sizes.  The workspace must be 256-byte
 * aligned device memory; its contents need no initialisation.  The size
 * covers every tile variant of m. */
size_t dia_workspace_size(int32_t H, int32_t W, int32_t ld, int32_t m, int32_t clip, int32_t mem);

/* The same for a whole pair description (its H, W, ld, m, mem and
 * kernel_degree); the only size query for pairs with kernel_degree > 0.
 * Returns 0 for an invalid pair. */
size_t dia_pair_workspace_size(const dia_pair *pair, int32_t clip);

/* One loss + gradient evaluation at theta (Sec. 2.3, Eq. 8 / Eq. 13).
 *   theta     device float64[n]  (read; the kernel works in float32 pixels)
 *   loss_out  device float64[1]  L = sum over unmasked valid pixels
 *   grad_out  device float64[n]  dL/dtheta, same layout as theta
 * The fused kernel computes M, the per-pixel loss and dL/dM and the
 * correlation of dL/dM with R in one pass, never storing M; per-CTA sums are
 * float32 over one tile and float64 across tiles and CTAs, reduced in a
 * fixed order (bitwise repeatable).  The pair must be DIA_MEM_DEVICE.
 * Asynchronous on `stream`. */
dia_status dia_loss_grad(const dia_pair *pair, const dia_loss_spec *loss,
                         const double *theta, double *loss_out, double *grad_out,
                         void *workspace, size_t workspace_bytes, void *stream);

/* Device time of the fused evaluation kernel alone (the gradient-mode
 * launch dia_loss_grad makes: the streaming small-kernel form or the tiled
 * kernel, as dia_set_small_kernel and the pair decide), for roofline figures
 * and the tile autotuner.  The float32 copy of theta is prepared once, then:
 * if flush_bytes > 0, `reps` launches are each bracketed by CUDA events on
 * `stream`, and flush_buf (device, 16-byte aligned, flush_bytes; make it
 * larger than the L2 cache; its contents are only read) is read through L2
 * before every launch, so each launch reads its inputs from HBM and finds no
 * dirty lines to write back; if flush_bytes == 0, the `reps` launches run back
 * to back between one pair of events (no launch gaps in the figure; inputs
 * larger than the L2 cache stand in for the flush).  *ms_out (HOST) receives
 * the mean milliseconds per launch.  The
 * partial sums are left in the workspace (no reduction runs).  Synchronous.
 * Errors: DIA_ERR_ARG (reps outside 1..100000, flush_bytes without a buffer,
 * bad pair or loss), DIA_ERR_WORKSPACE, DIA_ERR_CUDA. */
dia_status dia_time_eval(const dia_pair *pair, const dia_loss_spec *loss, const double *theta,
                         int32_t reps, void *flush_buf, size_t flush_bytes, float *ms_out,
                         void *workspace, size_t workspace_bytes, void *stream);

/* Difference image D = I - M over the valid region (Sec. 1) for theta
 * (device float64[n]); diff_out is (H-2h) x (W-2h) float32.  Asynchronous. */
dia_status dia_diff_image(const dia_pair *pair, const double *theta, float *diff_out,
                          void *workspace, size_t workspace_bytes, void *stream);

/* The same difference image with the correlation on the tensor cores
 * (tcgen05.mma, sm_103a): per output tile of 32 rows x 128 columns and per
 * kernel column b, a 128 x 32 x 64 product of the tile's R window (shifted by
 * b columns) with a Hankel matrix of kernel column b accumulates M - B0 in
 * tensor memory; R and K are split into bf16 high and low parts and the three
 * products hi*hi, hi*lo, lo*hi are summed in float32 (each term of M within
 * 3 x 2^-16 of its magnitude, against 2^-24 for the float32 CUDA-core form).
 * Constant background only (bg_degree 0, else DIA_ERR_UNSUPPORTED); m <= 31.
 * Synchronous: waits on `stream` and returns DIA_ERR_TIMEOUT if a kernel wait
 * ran out (the kernel bounds every wait). */
dia_status dia_diff_image_tc(const dia_pair *pair, const double *theta, float *diff_out,
                             void *workspace, size_t workspace_bytes, void *stream);

/* One loss + gradient evaluation with both contractions on the tensor cores
 * (tcgen05.mma, sm_103a).  The forward pass of dia_diff_image_tc (split bf16)
 * forms, in its epilogue, the loss terms and g = dl/dM (float32, the same
 * pixel terms as dia_loss_grad; 0 where masked) into a g map padded to whole
 * tiles, with max |R| and max |g|; the weight gradient
 * dL/dK[a][b] = sum_i P_b[i][i + a], P_b[i][y] = sum_j g[i][j] W[y][j + b],
 * over 128 x 64 tiles of g and their 160 x 96 R windows W, is one GEMM per
 * kernel column b (M = 128 tile rows, N = 160 window rows) with g and R
 * scaled by powers of two and split into float16 hi + lo (three products,
 * float32 accumulation in tensor memory), then sums along the diagonals
 * (float32 per tile and column, float64 across tiles).  Same arguments and
 * outputs as dia_loss_grad; constant background, one kernel (bg_degree =
 * kernel_degree = 0) and m <= 31, else DIA_ERR_UNSUPPORTED.  The workspace
 * is dia_tc_workspace_size(H, W, ld, m) bytes (the evaluation workspace plus
 * the g map and two partial rows per SM).  Synchronous: waits on `stream` and
 * returns DIA_ERR_TIMEOUT if a bounded wait of a tensor-core kernel ran out,
 * DIA_ERR_CUDA with dia_last_cuda_error() = -2 / -3 if a kernel's own bounds
 * check failed.  dia_set_eval_form(DIA_EVAL_TC) makes dia_loss_grad and
 * dia_fit use the same kernels. */
size_t dia_tc_workspace_size(int32_t H, int32_t W, int32_t ld, int32_t m);
dia_status dia_loss_grad_tc(const dia_pair *pair, const dia_loss_spec *loss, const double *theta,
                            double *loss_out, double *grad_out, void *workspace,
                            size_t workspace_bytes, void *stream);

/* Limit, in SM clock cycles, of each pipeline wait of dia_diff_image_tc's
 * kernel (an mbarrier wait of a producer or MMA role); 0 restores the default
 * (2e9 cycles, about one second).  A wait that runs out aborts every role of
 * the CTA: in-flight copies and MMAs are drained (with the default limit),
 * tensor memory is released and the call returns DIA_ERR_TIMEOUT; the next
 * call runs normally.  For exercising that failure path (a short limit makes
 * a wait run out on a healthy GPU); process-wide.  DIA_ERR_ARG if cycles < 0. */
dia_status dia_set_tc_wait_cycles(int64_t cycles);

/* Fit theta = [K, background] (Sec. 2.10 algorithm): initialise, Adam until the
 * relative loss change drops below switch_tol, then L-BFGS (preconditioned
 * by the inverse Gauss-Newton Hessian of a window of the pair, Wolfe /
 * approximate-Wolfe line search) until grad_tol, rel_tol or the limit of
 * numerical precision (stall_iters); optionally clip |z| > kappa and refit
 * clip_passes times.  Each optimiser iteration is one fused evaluation, a
 * float64 reduction and the float64 optimiser step (a line-search kernel, a
 * multi-CTA P v and a direction kernel), replayed graph_iters at a time from
 * a CUDA graph.
 * Outputs (all nullable; device pointers, or host pointers if the pair is
 * DIA_MEM_HOST):
 *   theta_out  float64[n]; K_out float32[m*m]; b0_out float32[1] (b_00);
 *   diff_out   float32 (H-2h) x (W-2h) difference image at the final theta;
 *   mask_out   uint8 H x W final mask (input mask with clipped pixels zeroed).
 * info (HOST, nullable) receives counters, final loss, P = sum K, B0.
 * Returns the fit status (also in info->status); on DIA_ERR_MAXITER the
 * outputs hold the last accepted theta. */
dia_status dia_fit(const dia_pair *pair, const dia_loss_spec *loss, const dia_opts *opts,
                   double *theta_out, float *K_out, float *b0_out, float *diff_out,
                   uint8_t *mask_out, dia_fit_info *info,
                   void *workspace, size_t workspace_bytes, void *stream);

/* Batched fits: many stamp pairs of uneven sizes and kernel sides, each
 * optimiser iteration of the whole batch in a few launches.  `pairs` is a
 * HOST array of npairs DIA_MEM_DEVICE pairs (each with its own H, W, ld, m,
 * maps); one loss spec and one dia_opts apply to all (clip_passes must be 0;
 * init 0 or 1).  Every optimiser iteration compacts the work items of the
 * pairs still running (a pair and a run of its tiles, largest first; the run
 * length per kernel-side group is dia_select_batch_variant's), runs one
 * persistent fused evaluation kernel per group of kernel sides (1-7, 9-15,
 * 17-23, 25-31; parallel graph branches) over those items from atomic queues,
 * then two kernels with one CTA per pair (line search and history; P v and
 * the L-BFGS direction) in which converged pairs return at once.
 * graph_iters iterations are replayed from a CUDA graph.
 * Outputs: theta_out (device, nullable) packs the pairs' theta vectors in
 * order, pair i at offset sum_{j<i} n_j with n_j = m_j^2 + (d_j+1)(d_j+2)/2
 * (d_j its bg_degree); diff_out (nullable HOST array of npairs device
 * pointers, entries nullable) receives each pair's
 * difference image; infos (nullable HOST array of npairs) the per-pair
 * counters and status.  Returns DIA_OK, or the first error; per-pair fit
 * statuses are in infos.  The workspace (256-byte aligned device memory) is
 * dia_batch_workspace_size(pairs, npairs, opts) bytes (0 if invalid). */
size_t dia_batch_workspace_size(const dia_pair *pairs, int32_t npairs, const dia_opts *opts);

/* Work-item size of the batched evaluation, per kernel-side group (0: m 1-7,
 * 1: 9-15, 2: 17-23, 3: 25-31): variant v (0..3) makes a work item of a pair
 * with kernel side m cover about c_v * 441 / m^2 tiles of 32 x 128 pixels
 * (c = 2, 1, 4, 8 for v = 0, 1, 2, 3; between 1 and 32 tiles), so items carry
 * about equal work across sides.  dia_batch_chunk_tiles(m, v) gives that
 * count.  The autotuner times the variants on a batch's own pairs and selects
 * one per group (default 0).  Process-wide; the workspace size depends on the
 * selection, so do not change it between dia_batch_workspace_size and
 * dia_fit_batch.  Errors: DIA_ERR_ARG (group or variant out of range). */
dia_status dia_select_batch_variant(int32_t group, int32_t variant);
int32_t dia_get_batch_variant(int32_t group);

/* Kernel-level timing of the batched evaluation (no counterpart in the
 * paper: a measurement hook).  With reps > 0, every later dia_fit_batch call
 * times, after its initialisation and before its first iteration, each
 * kernel-side group's evaluation kernel alone over all of that group's work
 * items at the starting theta.  It does one untimed launch, then reps
 * launches between CUDA events on the call's stream.  These launches write
 * only partial sums that the first iteration rewrites, so the fit's results
 * are unchanged; they add (reps + 1) launches per group.  reps = 0 (the
 * default) turns it off.  Process-wide.  Errors: DIA_ERR_ARG (reps outside
 * [0, 1000]).
 * dia_get_batch_eval_timing: the last timed call's mean milliseconds per
 * launch and algorithmic flop (4 m^2 per valid pixel, masks not subtracted)
 * for groups 0..3 (kernel sides 1-7, 9-15, 17-23, 25-31), into HOST arrays of
 * 4; 0 for a group without pairs.  Errors: DIA_ERR_ARG (NULL output). */
dia_status dia_set_batch_eval_timing(int32_t reps);
dia_status dia_get_batch_eval_timing(float *ms_out, double *flop_out);
int32_t dia_batch_chunk_tiles(int32_t m, int32_t variant);
dia_status dia_fit_batch(const dia_pair *pairs, int32_t npairs, const dia_loss_spec *loss,
                         const dia_opts *opts, double *theta_out, float *const *diff_out,
                         dia_fit_info *infos, void *workspace, size_t workspace_bytes,
                         void *stream);

/* Size of the fixed device scratch array used by dia_loss_grad_noalloc. */
#define DIA_NOALLOC_SCRATCH_BYTES (2u << 20)

/* dia_loss_grad without a caller workspace and without any device
 * allocation.  The paper has no counterpart: this is an interface for
 * callers that cannot call cudaMalloc or hold a workspace of their own --
 * e.g. code embedded in a host application that owns all device memory
 * through its own pool and forbids outside allocations, or a pipeline that
 * must not allocate once running.  Inputs and outputs are the same as for
 * dia_loss_grad (device pointers owned by the caller, DIA_MEM_DEVICE pair).
 *
 * Scratch: one file-scope device array of DIA_NOALLOC_SCRATCH_BYTES bytes
 * (2 MiB), which every GPU that loads the library keeps until the process
 * exits.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the one array and it keeps
 * the last call's contents: calls that overlap on the GPU (different
 * streams, or different host threads) race and must be serialised by the
 * caller.  Nothing in the array needs to start at zero: every call
 * overwrites what it reads.  The number of CTAs is capped so that their
 * partial sums fit the array; a kernel size whose scratch cannot fit is
 * refused with DIA_ERR_WORKSPACE (none with m <= DIA_MAX_M), m > DIA_MAX_M
 * with DIA_ERR_UNSUPPORTED.  Results equal dia_loss_grad's up to the order
 * of the float64 cross-CTA sums.  Asynchronous on `stream`. */
dia_status dia_loss_grad_noalloc(const dia_pair *pair, const dia_loss_spec *loss,
                                 const double *theta, double *loss_out, double *grad_out,
                                 void *stream);

/* ---------------------------------------------------------------------------
 * Observed Fisher information and covariance (Sec. 2.5, Eq. 15 and 16).
 *
 * F = d^2 L / d theta^2 at theta, L the loss of dia_loss_grad (for the
 * Gaussian loss with a fixed or model-dependent variance this is the negative
 * log-likelihood up to constants, so F is the observed Fisher information; for
 * Huber and Cauchy it is the Hessian of that loss).  M is linear in theta, so
 * F = sum_p l''(M_p) phi_p phi_p^T over every unmasked valid pixel, with
 * phi_p = [R window of p, background basis at p]; float32 per-pixel terms,
 * float64 sums (every 32 pixels), n = m*m + (d+1)(d+2)/2.  The covariance estimate is F^-1 at the fitted theta
 * (Eq. 16); its diagonal square roots are the Cramer-Rao bounds (Eq. 17).
 * Sec. 2.5 asks that the covariance be checked: F is tested for positive
 * definiteness by a float64 Cholesky factorisation (for a symmetric matrix
 * this is the same as every eigenvalue > 0, and then the determinant is > 0).
 */
typedef struct {
    int32_t positive_definite; /* 1: F (and so F^-1) is positive definite; 0: the
                                  warning flag of Sec. 2.5 -- cov_out is NaN */
    int32_t n;                 /* m*m + (d+1)(d+2)/2 */
    double log_det;            /* ln det F (valid when positive_definite) */
    double min_pivot;          /* smallest pivot of the Cholesky factorisation */
    int64_t ndata;             /* unmasked valid pixels summed */
} dia_fisher_info;

/* Workspace bytes of dia_fisher for this image and kernel side, any
 * background degree (0 if invalid). */
size_t dia_fisher_workspace_size(int32_t H, int32_t W, int32_t ld, int32_t m);
/* The same for a pair description (any kernel_degree; 0 if invalid). */
size_t dia_pair_fisher_workspace_size(const dia_pair *pair);

/* pair: DIA_MEM_DEVICE images; theta: DEVICE pointer, n doubles (e.g. the
 * theta_out of dia_fit); F_out, cov_out: nullable DEVICE pointers to n x n
 * row-major doubles (at least one of them, or info, should be given); info:
 * nullable HOST pointer, filled after the stream is synchronised (the call is
 * then synchronous).  Errors: DIA_ERR_ARG (bad pair, loss or pointers),
 * DIA_ERR_WORKSPACE, DIA_ERR_UNSUPPORTED (m > DIA_MAX_M), DIA_ERR_CUDA. */
dia_status dia_fisher(const dia_pair *pair, const dia_loss_spec *loss, const double *theta,
                      double *F_out, double *cov_out, dia_fisher_info *info, void *workspace,
                      size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DIA_H */

// Batched fits: many reference/target pairs of uneven sizes and kernel sides
// fitted together.  One optimiser iteration of the whole batch is
//   1. eval_batch_kernel: persistent CTAs take work items (a pair and a
//      contiguous range of its tiles, largest first) from an atomic queue and
//      run the fused forward/loss/backward pass of that pair's kernel side,
//      writing one set of float64 partial sums per item;
//   2. step_batch_kernel: one CTA per pair sums its items' partials in a
//      fixed order and takes that pair's optimiser step.
// Converged pairs are skipped by both kernels.  graph_iters iterations are
// captured in a CUDA graph; the host polls the count of finished pairs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <list>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dia.h"
#include "dia_batch.cuh"
#include "dia_checks.h"
#include "dia_ops.cuh"

namespace dia {
namespace {

thread_local int g_batch_cuda = 0;
// work-item size variant of each kernel-side group (dia_select_batch_variant)
std::atomic<int> g_batch_variant[4] = {{0}, {0}, {0}, {0}};
// kernel-level timing of the batched evaluation (dia_set_batch_eval_timing):
// repetitions per group (0: off), and the last timed call's per-group mean
// milliseconds and algorithmic flop
std::atomic<int> g_batch_time_reps{0};
std::mutex g_bt_mu;
float g_bt_ms[4] = {0.f, 0.f, 0.f, 0.f};
double g_bt_flop[4] = {0.0, 0.0, 0.0, 0.0};

#define DB_CK(expr)                    \
    do {                               \
        cudaError_t _e = (expr);       \
        if (_e != cudaSuccess) {       \
            g_batch_cuda = (int)_e;    \
            return DIA_ERR_CUDA;       \
        }                              \
    } while (0)

size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

struct PairPlan {
    int m, n, np, tiles_x, n_tiles, n_chunks;
    int y0, y1, x0, x1;   // preconditioner window (valid-region coordinates)
    size_t st_off, red_off, vec_off, hist_off, kpad_off;
    size_t pc_a_off, pc_x_off, pc_p_off;   // preconditioner (if enabled)
    long long part_off, theta_off;
};

struct BatchPlan {
    std::vector<PairPlan> pp;
    std::vector<BatchItem> items;
    size_t off_hdr, off_eas, off_mks, off_items, off_act, off_gbeg, off_sa, off_red, off_thoff,
        off_pas, off_pairs, off_parts, total;
    long long total_parts;
    int history;
    int gbeg[5];   // items of kernel-side group g: [gbeg[g], gbeg[g+1])
};

dia_status plan_batch(const dia_pair *pairs, int npairs, int history, int precond, int pc_side,
                      BatchPlan &P) {
    if (!pairs || npairs <= 0) return DIA_ERR_ARG;
    P.pp.resize(npairs);
    P.history = history;
    long long parts = 0, thoff = 0;
    size_t per = 0;
    for (int i = 0; i < npairs; ++i) {
        const dia_pair &p = pairs[i];
        if (p.mem != DIA_MEM_DEVICE) return DIA_ERR_ARG;
        const dia_status rc = check_pair(&p);
        if (rc != DIA_OK) return rc;
        if (p.kernel_degree != 0) return DIA_ERR_UNSUPPORTED;   // one kernel per pair only
        PairPlan &q = P.pp[i];
        q.m = p.m;
        q.n = p.m * p.m + n_background(p.bg_degree);
        q.np = np_of(p.m);
        const int h = p.m / 2, Hv = p.H - 2 * h, Wv = p.W - 2 * h;
        q.tiles_x = (Wv + kTW - 1) / kTW;
        q.n_tiles = q.tiles_x * ((Hv + kBTH - 1) / kBTH);
        const int ct = batch_chunk(p.m, g_batch_variant[batch_group(p.m)].load());
        q.n_chunks = (q.n_tiles + ct - 1) / ct;
        q.part_off = parts;
        parts += (long long)q.n_chunks * q.np;
        q.theta_off = thoff;
        thoff += q.n;
        // per-pair region: FitState, reduced sums, 9 vectors + S/Y/PY history,
        // S'Y and Y'PY, Kpad
        q.st_off = per;
        per = al(per + sizeof(FitState));
        q.red_off = per;
        per = al(per + (size_t)q.np * 8);
        q.vec_off = per;
        per = al(per + (size_t)q.n * 8 * (9 + 3 * (size_t)history) +
                 2 * (size_t)history * history * 8);
        q.kpad_off = per;
        per = al(per + (size_t)(p.m * round4(p.m) + kBgMax + 1) * 4);
        // preconditioner: float64 Gauss-Newton Hessian (factored in place) and
        // inverse factor, padded to 64, and P; one pixel chunk per pair
        int chunks = 1;
        precond_window(p.H, p.W, p.m, false, pc_side, &q.y0, &q.y1, &q.x0, &q.x1, &chunks);
        q.pc_a_off = q.pc_x_off = q.pc_p_off = 0;
        if (precond) {
            const size_t np2 = (size_t)pc_np(q.n) * pc_np(q.n);
            q.pc_a_off = per;
            per = al(per + np2 * 8);
            q.pc_x_off = per;
            per = al(per + np2 * 8);
            q.pc_p_off = per;
            per = al(per + (size_t)q.n * pc_ldp(q.n) * 4);
        }
        q.hist_off = 0;
        for (int c = 0; c < q.n_chunks; ++c) {
            BatchItem it;
            it.pair = i;
            it.t0 = c * ct;
            it.t1 = std::min(q.n_tiles, (c + 1) * ct);
            it.pad = 0;
            it.part_off = q.part_off + (long long)c * q.np;
            P.items.push_back(it);
        }
    }
    // by kernel-side group, then largest work first (tiles x m^2) so that the
    // tail of each evaluation is short
    std::stable_sort(P.items.begin(), P.items.end(), [&](const BatchItem &a, const BatchItem &b) {
        const int ga = batch_group(P.pp[a.pair].m), gb = batch_group(P.pp[b.pair].m);
        if (ga != gb) return ga < gb;
        const long long ca = (long long)(a.t1 - a.t0) * P.pp[a.pair].m * P.pp[a.pair].m;
        const long long cb = (long long)(b.t1 - b.t0) * P.pp[b.pair].m * P.pp[b.pair].m;
        return ca > cb;
    });
    for (int g = 0; g <= 4; ++g) P.gbeg[g] = 0;
    for (const BatchItem &it : P.items) P.gbeg[batch_group(P.pp[it.pair].m) + 1] += 1;
    for (int g = 0; g < 4; ++g) P.gbeg[g + 1] += P.gbeg[g];
    P.total_parts = parts;
    size_t o = 0;
    P.off_hdr = o;
    o = al(o + 256);
    P.off_eas = o;
    o = al(o + sizeof(EvalArgs) * npairs);
    P.off_mks = o;
    o = al(o + sizeof(int) * npairs);
    P.off_items = o;
    o = al(o + sizeof(BatchItem) * P.items.size());
    P.off_act = o;   // compacted items of the running pairs
    o = al(o + sizeof(BatchItem) * P.items.size());
    P.off_gbeg = o;
    o = al(o + sizeof(int) * 5);
    P.off_sa = o;
    o = al(o + sizeof(StepArgs) * npairs);
    P.off_red = o;
    o = al(o + sizeof(BatchRed) * npairs);
    P.off_thoff = o;
    o = al(o + sizeof(long long) * npairs);
    P.off_pas = o;
    o = al(o + (precond ? sizeof(PrecondArgs) * npairs : 0));
    P.off_pairs = o;
    o = al(o + per);
    P.off_parts = o;
    o = al(o + (size_t)parts * 8);
    P.total = o;
    return DIA_OK;
}

struct BatchGraph {
    std::string key;
    cudaGraphExec_t exec;
};
std::mutex g_bmu;
std::list<BatchGraph> g_bgraphs;

cudaStream_t batch_capture_stream() {
    thread_local int dev_of = -1;
    thread_local cudaStream_t cs = nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cs == nullptr || dev_of != dev) {
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        dev_of = dev;
    }
    return cs;
}

}  // namespace
}  // namespace dia

using namespace dia;

extern "C" dia_status dia_select_batch_variant(int32_t group, int32_t variant) {
    if (group < 0 || group > 3 || variant < 0 || variant >= kBatchVariants) return DIA_ERR_ARG;
    g_batch_variant[group].store(variant);
    return DIA_OK;
}

extern "C" int32_t dia_get_batch_variant(int32_t group) {
    return (group < 0 || group > 3) ? -1 : g_batch_variant[group].load();
}

extern "C" dia_status dia_set_batch_eval_timing(int32_t reps) {
    if (reps < 0 || reps > 1000) return DIA_ERR_ARG;
    dia::g_batch_time_reps.store(reps);
    return DIA_OK;
}

extern "C" dia_status dia_get_batch_eval_timing(float *ms_out, double *flop_out) {
    if (!ms_out || !flop_out) return DIA_ERR_ARG;
    std::lock_guard<std::mutex> lk(dia::g_bt_mu);
    for (int g = 0; g < 4; ++g) {
        ms_out[g] = dia::g_bt_ms[g];
        flop_out[g] = dia::g_bt_flop[g];
    }
    return DIA_OK;
}

extern "C" int32_t dia_batch_chunk_tiles(int32_t m, int32_t variant) {
    if (m < 1 || m > DIA_MAX_M || (m & 1) == 0 || variant < 0 || variant >= kBatchVariants)
        return 0;
    return batch_chunk(m, variant);
}

extern "C" size_t dia_batch_workspace_size(const dia_pair *pairs, int32_t npairs,
                                           const dia_opts *opts) {
    dia_opts o;
    if (opts)
        o = *opts;
    else
        dia_opts_default(&o);
    if (o.history < 1 || o.history > kHistMax) return 0;
    BatchPlan P;
    if (plan_batch(pairs, npairs, o.history, o.precond, o.precond_window, P) != DIA_OK) return 0;
    return P.total;
}

extern "C" dia_status dia_fit_batch(const dia_pair *pairs, int32_t npairs,
                                    const dia_loss_spec *loss, const dia_opts *opts_in,
                                    double *theta_out, float *const *diff_out,
                                    dia_fit_info *infos, void *workspace,
                                    size_t workspace_bytes, void *stream) {
    nvtxRangePushA("dia_fit_batch");
    struct PopOnExit {
        ~PopOnExit() { nvtxRangePop(); }
    } pop_on_exit;
    dia_opts opts;
    if (opts_in)
        opts = *opts_in;
    else
        dia_opts_default(&opts);
    if (!loss || !pairs || npairs <= 0) return DIA_ERR_ARG;
    if (check_opts(opts, 1) != DIA_OK) return DIA_ERR_ARG;   // no theta0 for a batch
    if (opts.clip_passes != 0) return DIA_ERR_UNSUPPORTED;
    for (int i = 0; i < npairs; ++i) {
        const dia_status lrc = check_loss(loss, &pairs[i]);
        if (lrc != DIA_OK) return lrc;
    }
    BatchPlan P;
    dia_status rc = plan_batch(pairs, npairs, opts.history, opts.precond, opts.precond_window, P);
    if (rc != DIA_OK) return rc;
    if (!workspace || workspace_bytes < P.total || ((uintptr_t)workspace & 255) != 0)
        return DIA_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    // header ints: [2] pairs finished, [4+g] evaluation queue of group g,
    // [8+g] forward-pass queue of group g, [12+g] items of group g still
    // running (compacted each iteration), [16+g] all items of group g
    int *hdr = (int *)(ws + P.off_hdr);
    EvalArgs *d_eas = (EvalArgs *)(ws + P.off_eas);
    int *d_mks = (int *)(ws + P.off_mks);
    BatchItem *d_items = (BatchItem *)(ws + P.off_items);
    BatchItem *d_act = (BatchItem *)(ws + P.off_act);
    int *d_gbeg = (int *)(ws + P.off_gbeg);
    StepArgs *d_sa = (StepArgs *)(ws + P.off_sa);
    BatchRed *d_red = (BatchRed *)(ws + P.off_red);
    long long *d_thoff = (long long *)(ws + P.off_thoff);
    PrecondArgs *d_pas = (PrecondArgs *)(ws + P.off_pas);
    char *pairs_base = ws + P.off_pairs;
    double *d_parts = (double *)(ws + P.off_parts);

    // host images of the descriptor arrays
    std::vector<EvalArgs> eas(npairs);
    std::vector<int> mks(npairs);
    std::vector<StepArgs> sas(npairs);
    std::vector<BatchRed> reds(npairs);
    std::vector<long long> thoff(npairs);
    std::vector<PrecondArgs> pas(opts.precond ? npairs : 0);
    const LossParams lp = to_params(loss);
    const int H = opts.history;
    int max_n = 1, bg = 0;   // bg: some pair has a polynomial background
    for (int i = 0; i < npairs; ++i) {
        max_n = std::max(max_n, P.pp[i].n);
        bg |= pairs[i].bg_degree > 0;
    }
    for (int i = 0; i < npairs; ++i) {
        const dia_pair &p = pairs[i];
        const PairPlan &q = P.pp[i];
        char *pb = pairs_base;
        FitState *st = (FitState *)(pb + q.st_off);
        double *vec = (double *)(pb + q.vec_off);
        const int n = q.n, h = p.m / 2;
        EvalArgs &a = eas[i];
        memset(&a, 0, sizeof(a));
        a.R = p.ref;
        a.I = p.img;
        a.mask = p.mask;
        a.var = p.var;
        a.flat = p.flat;
        a.H = p.H;
        a.W = p.W;
        a.ld = p.ld;
        a.Hv = p.H - 2 * h;
        a.Wv = p.W - 2 * h;
        a.tiles_x = q.tiles_x;
        a.n_tiles = q.n_tiles;
        a.Kpad = (const float *)(pb + q.kpad_off);
        a.diff_out = diff_out ? diff_out[i] : nullptr;
        a.clip_kappa = opts.clip_kappa;
        a.done_flag = &st->done;
        a.lp = lp;
        set_background(a, p.bg_degree, p.H, p.W, h);
        mks[i] = p.m;
        StepArgs &sa = sas[i];
        memset(&sa, 0, sizeof(sa));
        sa.st = st;
        sa.b.theta = vec;
        sa.b.trial = vec + n;
        sa.b.grad = vec + 2 * n;
        sa.b.glo = vec + 3 * n;
        sa.b.m1 = vec + 4 * n;
        sa.b.m2 = vec + 5 * n;
        sa.b.dir = vec + 6 * n;
        sa.b.pdiag = vec + 7 * n;
        sa.b.pg = vec + 8 * n;
        sa.b.S = vec + 9 * n;
        sa.b.Y = sa.b.S + (size_t)H * n;
        sa.b.PY = sa.b.Y + (size_t)H * n;
        sa.b.SY = sa.b.PY + (size_t)H * n;
        sa.b.YPY = sa.b.SY + (size_t)H * H;
        sa.b.P = nullptr;
        sa.b.ldp = pc_ldp(n);
        if (opts.precond) {
            PrecondArgs &pa = pas[i];
            memset(&pa, 0, sizeof(pa));
            pa.R = p.ref;
            pa.I = p.img;
            pa.mask = p.mask;
            pa.var = p.var;
            pa.flat = p.flat;
            pa.H = p.H;
            pa.W = p.W;
            pa.ld = p.ld;
            pa.m = p.m;
            pa.y0 = q.y0;
            pa.y1 = q.y1;
            pa.x0 = q.x0;
            pa.x1 = q.x1;
            pa.lp = lp;
            pa.part = nullptr;
            pa.gn_chunks = 1;
            pa.A64 = (double *)(pb + q.pc_a_off);
            pa.X64 = (double *)(pb + q.pc_x_off);
            pa.P = (float *)(pb + q.pc_p_off);
            pa.ldp = pc_ldp(n);
            pa.st = st;
            pa.eps = 1e-6;
            pa.reg2 = 2.0 * opts.reg_lambda;
            pa.nbg = n - p.m * p.m;
            pa.eta0 = a.eta0;
            pa.eta_s = a.eta_s;
            pa.xi0 = a.xi0;
            pa.xi_s = a.xi_s;
            pa.scale = 1.0 / ((double)(pa.y1 - pa.y0) * (pa.x1 - pa.x0));
            pa.flush = kGnFlushPc;
            sa.b.P = pa.P;
        }
        sa.red = (const double *)(pb + q.red_off);
        sa.Kpad = (float *)(pb + q.kpad_off);
        sa.n = n;
        sa.mk = p.m;
        sa.kp = round4(p.m);
        sa.p.lr_kernel = opts.lr_kernel;
        sa.p.lr_b0 = opts.lr_b0;
        sa.p.beta1 = opts.beta1;
        sa.p.beta2 = opts.beta2;
        sa.p.adam_eps = opts.adam_eps;
        sa.p.switch_tol = opts.switch_tol;
        sa.p.rel_tol = opts.rel_tol;
        sa.p.grad_tol = opts.grad_tol;
        sa.p.max_adam = opts.max_adam_iters;
        sa.p.history = H;
        sa.p.max_lbfgs = opts.max_lbfgs_iters;
        sa.p.max_evals = opts.max_evals;
        sa.p.stall_iters = opts.stall_iters;
        sa.p.stall_iters_diag = opts.stall_iters_diag;
        sa.p.max_ls = opts.max_ls_evals;
        sa.p.reg_lambda = opts.reg_lambda;
        sa.n_done = hdr + 2;
        BatchRed &r = reds[i];
        r.part_off = q.part_off;
        r.n_chunks = q.n_chunks;
        r.np = q.np;
        r.red = (double *)(pb + q.red_off);
        thoff[i] = q.theta_off;
    }
    DB_CK(cudaMemsetAsync(hdr, 0, 256, s));
    {
        int cnt[4];
        for (int g = 0; g < 4; ++g) cnt[g] = P.gbeg[g + 1] - P.gbeg[g];
        DB_CK(cudaMemcpyAsync(hdr + 16, cnt, sizeof(cnt), cudaMemcpyHostToDevice, s));
        DB_CK(cudaMemcpyAsync(d_gbeg, P.gbeg, sizeof(int) * 5, cudaMemcpyHostToDevice, s));
    }
    DB_CK(cudaMemcpyAsync(d_eas, eas.data(), sizeof(EvalArgs) * npairs, cudaMemcpyHostToDevice, s));
    DB_CK(cudaMemcpyAsync(d_mks, mks.data(), sizeof(int) * npairs, cudaMemcpyHostToDevice, s));
    DB_CK(cudaMemcpyAsync(d_items, P.items.data(), sizeof(BatchItem) * P.items.size(),
                          cudaMemcpyHostToDevice, s));
    DB_CK(cudaMemcpyAsync(d_sa, sas.data(), sizeof(StepArgs) * npairs, cudaMemcpyHostToDevice, s));
    DB_CK(cudaMemcpyAsync(d_red, reds.data(), sizeof(BatchRed) * npairs, cudaMemcpyHostToDevice, s));
    DB_CK(cudaMemcpyAsync(d_thoff, thoff.data(), sizeof(long long) * npairs,
                          cudaMemcpyHostToDevice, s));
    if (opts.precond)
        DB_CK(cudaMemcpyAsync(d_pas, pas.data(), sizeof(PrecondArgs) * npairs,
                              cudaMemcpyHostToDevice, s));

    // kernel configuration: one persistent kernel per kernel-side group present
    int dev = 0, sms = 1;
    DB_CK(cudaGetDevice(&dev));
    DB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int grid[4] = {0, 0, 0, 0}, n_it[4];
    const int gsmem[4] = {batch_group_smem(0), batch_group_smem(1), batch_group_smem(2),
                          batch_group_smem(3)};
    const BatchItem *g_items[4], *g_act[4];
    const int *g_nall[4], *g_nact[4];
    for (int g = 0; g < 4; ++g) {
        n_it[g] = P.gbeg[g + 1] - P.gbeg[g];
        g_items[g] = d_items + P.gbeg[g];
        g_act[g] = d_act + P.gbeg[g];
        g_nall[g] = hdr + 16 + g;
        g_nact[g] = hdr + 12 + g;
        if (n_it[g] == 0) continue;
        for (int mode = 0; mode < 2; ++mode)
            DB_CK(cudaFuncSetAttribute(batch_kernel_ptr(g, mode, bg),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       gsmem[g]));
        int occ = 1;
        DB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel_ptr(g, kModeGrad, bg),
                                                            kBW * 32, gsmem[g]));
        grid[g] = std::min(n_it[g], sms * (occ < 1 ? 1 : occ));
    }
    // mode kModeGrad walks the compacted items of the running pairs, the
    // final forward pass every item
    auto launch_group = [&](int g, int mode, int *counter, cudaStream_t st) -> cudaError_t {
        const BatchItem *its = mode == kModeGrad ? g_act[g] : g_items[g];
        const int *nit = mode == kModeGrad ? g_nact[g] : g_nall[g];
        void *params[] = {(void *)&d_eas, (void *)&d_mks, (void *)&its, (void *)&nit,
                          (void *)&counter, (void *)&d_parts};
        return cudaLaunchKernel(batch_kernel_ptr(g, mode, bg), dim3(grid[g]), dim3(kBW * 32), params,
                                gsmem[g], st);
    };

    // initialisation: per-pair median and theta (Sec. 2.9)
    const int start_phase = opts.max_adam_iters > 0 ? kPhaseAdam : kPhaseLbfgsStart;
    DB_CK(launch_init_batch(d_sa, d_eas, npairs, opts.init, opts.init_sigma, start_phase, s));
    // per-pair Gauss-Newton preconditioners (after init, which clears the state)
    if (opts.precond) DB_CK(launch_precond(d_pas, pas.data(), npairs, s));

    // optional kernel-level timing: each group's evaluation kernel alone over
    // all its work items at the starting theta, between CUDA events on the
    // stream (one untimed launch first).  The launches write only the items'
    // partial sums, which the first iteration rewrites, and the queue
    // counters are cleared again, so the fit is unchanged.
    long long timing_launches = 0;
    if (const int treps = g_batch_time_reps.load(); treps > 0) {
        float ms_g[4] = {0.f, 0.f, 0.f, 0.f};
        double fl_g[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < npairs; ++i) {
            const int mk = pairs[i].m, h = mk / 2;
            fl_g[batch_group(mk)] +=
                4.0 * mk * mk * (double)(pairs[i].H - 2 * h) * (double)(pairs[i].W - 2 * h);
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        auto launch_all = [&](int g) -> cudaError_t {
            int *counter = hdr + 4 + g;
            const BatchItem *its = g_items[g];
            const int *nit = g_nall[g];
            void *params[] = {(void *)&d_eas, (void *)&d_mks, (void *)&its, (void *)&nit,
                              (void *)&counter, (void *)&d_parts};
            return cudaLaunchKernel(batch_kernel_ptr(g, kModeGrad, bg), dim3(grid[g]),
                                    dim3(kBW * 32), params, gsmem[g], s);
        };
        for (int g = 0; g < 4 && e == cudaSuccess; ++g) {
            if (n_it[g] == 0) continue;
            for (int r = -1; r < treps && e == cudaSuccess; ++r) {
                e = cudaMemsetAsync(hdr + 4 + g, 0, sizeof(int), s);
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                if (e == cudaSuccess) e = launch_all(g);
                timing_launches += 1;
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (r >= 0) ms_g[g] += ms / (float)treps;
            }
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(hdr + 4, 0, 4 * sizeof(int), s);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        DB_CK(e);
        std::lock_guard<std::mutex> lk(g_bt_mu);
        for (int g = 0; g < 4; ++g) {
            g_bt_ms[g] = ms_g[g];
            g_bt_flop[g] = n_it[g] > 0 ? fl_g[g] : 0.0;
        }
    }

    // the iteration graph (cached per workspace / batch shape / settings); the
    // group kernels are parallel branches, joined before the optimiser step
    std::string key;
    auto app = [&](const void *p, size_t n) { key.append((const char *)p, n); };
    app(&dev, sizeof dev);
    app(&ws, sizeof ws);
    app(&npairs, sizeof npairs);
    app(n_it, sizeof n_it);
    app(grid, sizeof grid);
    app(&opts.graph_iters, sizeof opts.graph_iters);
    app(&max_n, sizeof max_n);
    app(&bg, sizeof bg);
    // the captured kernels take pointers into the workspace at these offsets
    const size_t offs[] = {P.off_hdr,   P.off_eas,  P.off_mks,   P.off_items, P.off_act,
                           P.off_gbeg,  P.off_sa,   P.off_red,   P.off_thoff, P.off_pas,
                           P.off_pairs, P.off_parts};
    app(offs, sizeof offs);
    app(P.gbeg, sizeof P.gbeg);
    cudaGraphExec_t gx = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_bmu);
        for (auto &e : g_bgraphs)
            if (e.key == key) gx = e.exec;
        if (!gx) {
            cudaStream_t cs = batch_capture_stream();
            thread_local cudaStream_t side[4] = {nullptr, nullptr, nullptr, nullptr};
            thread_local cudaEvent_t evf = nullptr, evj[4] = {nullptr, nullptr, nullptr, nullptr};
            thread_local int side_dev = -1;
            if (side_dev != dev) {
                for (int g = 0; g < 4; ++g) {
                    DB_CK(cudaStreamCreateWithFlags(&side[g], cudaStreamNonBlocking));
                    DB_CK(cudaEventCreateWithFlags(&evj[g], cudaEventDisableTiming));
                }
                DB_CK(cudaEventCreateWithFlags(&evf, cudaEventDisableTiming));
                side_dev = dev;
            }
            DB_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int it = 0; it < opts.graph_iters && e == cudaSuccess; ++it) {
                // items of the pairs still running, then the group evaluations
                e = launch_compact_items(d_items, d_eas, d_gbeg, d_act, hdr + 12, cs);
                if (e == cudaSuccess) e = cudaEventRecord(evf, cs);
                for (int g = 0; g < 4 && e == cudaSuccess; ++g) {
                    if (n_it[g] == 0) continue;
                    e = cudaStreamWaitEvent(side[g], evf, 0);
                    if (e == cudaSuccess) e = launch_group(g, kModeGrad, hdr + 4 + g, side[g]);
                    if (e == cudaSuccess) e = cudaEventRecord(evj[g], side[g]);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, evj[g], 0);
                }
                if (e == cudaSuccess)
                    e = launch_step_batch(d_sa, d_red, d_parts, npairs, hdr + 4, 4, cs);
            }
            cudaGraph_t gr = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                g_batch_cuda = (int)(e != cudaSuccess ? e : e2);
                return DIA_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&gx, gr, 0);
            cudaGraphDestroy(gr);
            DB_CK(e);
            g_bgraphs.push_front({key, gx});
            if (g_bgraphs.size() > 8) {
                cudaGraphExecDestroy(g_bgraphs.back().exec);
                g_bgraphs.pop_back();
            }
        }
    }
    int n_groups = 0;
    for (int g = 0; g < 4; ++g) n_groups += n_it[g] > 0;

    const auto t0 = std::chrono::steady_clock::now();
    int status = DIA_OK;
    int done_host = 0;
    // init (+ preconditioner, + timed evaluations)
    long long launches = 1 + (opts.precond ? precond_launches(max_n) : 0) + timing_launches;
    for (;;) {
        DB_CK(cudaGraphLaunch(gx, s));
        launches += (long long)(1 + n_groups + kStepLaunchesBatch) * opts.graph_iters;
        DB_CK(cudaMemcpyAsync(&done_host, hdr + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
        DB_CK(cudaStreamSynchronize(s));
        if (done_host >= npairs) break;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > opts.timeout_s) {
            status = DIA_ERR_TIMEOUT;
            break;
        }
    }

    // outputs: difference images (forward pass at the accepted theta) and theta
    bool any_diff = false;
    for (int i = 0; diff_out && i < npairs; ++i) any_diff |= diff_out[i] != nullptr;
    if (any_diff) {
        for (int g = 0; g < 4; ++g) {
            if (n_it[g] == 0) continue;
            DB_CK(launch_group(g, kModeForward, hdr + 8 + g, s));
            launches += 1;
        }
    }
    if (theta_out) {
        DB_CK(launch_pack_batch(d_sa, d_thoff, theta_out, npairs, s));
        launches += 1;
    }
    if (infos) {
        std::vector<FitState> hs(npairs);
        for (int i = 0; i < npairs; ++i)
            DB_CK(cudaMemcpyAsync(&hs[i], pairs_base + P.pp[i].st_off, sizeof(FitState),
                                  cudaMemcpyDeviceToHost, s));
        DB_CK(cudaStreamSynchronize(s));
        for (int i = 0; i < npairs; ++i) {
            dia_fit_info &f = infos[i];
            memset(&f, 0, sizeof(f));
            f.status = (status != DIA_OK && !hs[i].done) ? status : hs[i].status;
            f.adam_iters = hs[i].it_adam;
            f.lbfgs_iters = hs[i].it_lbfgs;
            f.evals = hs[i].evals;
            f.ndata = (int64_t)llround(hs[i].ndata);
            f.loss = hs[i].L_sum;
            f.grad_inf = hs[i].grad_inf;
            f.reason = hs[i].reason;
            f.kernel_launches = launches;
            f.precond_used = (opts.precond && hs[i].pc_ok) ? 1 : 0;
        }
    } else {
        DB_CK(cudaStreamSynchronize(s));
    }
    return (dia_status)status;
}

// Argument checks and loss-parameter conversion shared by every entry point.
#include <cmath>

#include "dia_checks.h"
#include "dia_ops.cuh"

namespace dia {

bool dims_ok(int H, int W, int ld, int m) {
    if (H <= 0 || W <= 0 || ld < W) return false;
    if (m < 1 || (m & 1) == 0 || m > H || m > W) return false;
    if ((long long)H * ld > (1LL << 40)) return false;
    return true;
}

dia_status check_pair(const dia_pair *p) {
    if (!p || !p->ref || !p->img) return DIA_ERR_ARG;
    if (p->mem != DIA_MEM_DEVICE && p->mem != DIA_MEM_HOST) return DIA_ERR_ARG;
    if (!dims_ok(p->H, p->W, p->ld, p->m)) return DIA_ERR_ARG;
    if (p->m > DIA_MAX_M) return DIA_ERR_UNSUPPORTED;
    if (p->bg_degree < 0 || p->bg_degree > DIA_MAX_BG_DEGREE) return DIA_ERR_ARG;
    if (p->kernel_degree < 0 || p->kernel_degree > DIA_MAX_KERNEL_DEGREE) return DIA_ERR_ARG;
    return DIA_OK;
}

dia_status check_loss(const dia_loss_spec *l, const dia_pair *p) {
    if (!l) return DIA_ERR_ARG;
    if (l->rho < 0 || l->rho > 2 || l->var_model < 0 || l->var_model > 2) return DIA_ERR_ARG;
    if (l->var_model == DIA_VAR_FIXED) {
        if (!p->var && !(l->var_scalar > 0.f)) return DIA_ERR_ARG;
    } else {
        if (!(l->gain > 0.f) || !(l->var_floor > 0.f)) return DIA_ERR_ARG;
        if (l->var_model == DIA_VAR_EMCCD && !(l->excess > 0.f)) return DIA_ERR_ARG;
    }
    if (l->rho == DIA_RHO_HUBER && !(l->huber_c > 0.f)) return DIA_ERR_ARG;
    return DIA_OK;
}

namespace {
bool pos_finite(double v) { return std::isfinite(v) && v > 0.0; }
bool nonneg_finite(double v) { return std::isfinite(v) && v >= 0.0; }
}  // namespace

dia_status check_opts(const dia_opts &o, int max_init) {
    // Adam (Sec. 2.3): decays in [0, 1) (beta = 1 divides by zero in the bias
    // correction), positive finite rates and epsilon; finite non-negative
    // stopping tolerances; a positive finite clip threshold when clipping
    // (NaN would clip nothing, 0 every pixel)
    const bool adam_ok = o.beta1 >= 0.0 && o.beta1 < 1.0 && o.beta2 >= 0.0 && o.beta2 < 1.0 &&
                         pos_finite(o.lr_kernel) && pos_finite(o.lr_b0) && pos_finite(o.adam_eps);
    const bool tol_ok = nonneg_finite(o.switch_tol) && nonneg_finite(o.rel_tol) &&
                        nonneg_finite(o.grad_tol);
    const bool clip_ok = o.clip_passes == 0 || (std::isfinite(o.clip_kappa) && o.clip_kappa > 0.f);
    if (!adam_ok || !tol_ok || !clip_ok) return DIA_ERR_ARG;
    const bool ok = o.history >= 1 && o.history <= kHistMax && o.graph_iters >= 1 &&
                    o.graph_iters <= 1024 && o.clip_passes >= 0 && o.max_adam_iters >= 0 &&
                    o.max_evals >= 1 && o.max_lbfgs_iters >= 1 && o.stall_iters >= 1 &&
                    o.stall_iters_diag >= 1 && o.max_ls_evals >= 2 && o.precond_window >= 0 &&
                    o.reg_lambda >= 0.0 && std::isfinite(o.reg_lambda) && o.init >= 0 &&
                    o.init <= max_init && !(o.init == 2 && !o.theta0) &&
                    !(o.init == 1 && !(o.init_sigma > 0.0)) && o.timeout_s > 0.0;
    return ok ? DIA_OK : DIA_ERR_ARG;
}

LossParams to_params(const dia_loss_spec *l) {
    LossParams lp;
    lp.rho = l->rho;
    lp.var_model = l->var_model;
    lp.s0sq = l->sigma0 * l->sigma0;
    lp.inv_gain = (l->gain > 0.f) ? 1.0f / l->gain : 1.0f;
    lp.excess = l->excess;
    lp.huber_c = l->huber_c;
    lp.var_scalar = l->var_scalar;
    lp.var_floor = l->var_floor;
    return lp;
}

}  // namespace dia

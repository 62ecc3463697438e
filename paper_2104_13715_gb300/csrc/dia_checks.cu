// Argument checks and loss-parameter conversion shared by every entry point.
#include "dia_checks.h"

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

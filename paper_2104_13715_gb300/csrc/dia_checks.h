// Argument checks and loss-parameter conversion shared by every entry point
// (host code; every check runs before any launch).
#pragma once

#include "../../include/dia.h"
#include "dia_eval.cuh"

namespace dia {

// H x W image with row pitch ld and odd kernel side m that fits in it; the
// pitched image stays below 2^40 elements
bool dims_ok(int H, int W, int ld, int m);
// a pair with images, a memory kind, valid dimensions (DIA_ERR_ARG), m <= DIA_MAX_M
// (else DIA_ERR_UNSUPPORTED) and a background degree in [0, DIA_MAX_BG_DEGREE]
dia_status check_pair(const dia_pair *p);
// a loss of a known kind with the parameters its variance model needs (p: the
// pair it applies to, for the fixed-variance map)
dia_status check_loss(const dia_loss_spec *l, const dia_pair *p);
// optimiser settings within their documented ranges (include/dia.h); init
// modes up to max_init (2 = theta0, which must then be given)
dia_status check_opts(const dia_opts &o, int max_init);
// the float32 parameters the fused kernel reads
LossParams to_params(const dia_loss_spec *l);

}  // namespace dia

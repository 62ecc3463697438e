// Instantiation helper: DIA_EVAL_INST(MK, V, NW, QF, PF, SPLIT, F2) defines
// kernel_info_<MK>_<V>() for the fused kernel of side MK, tile variant V.
#pragma once

#include "dia_dispatch.h"
#include "dia_eval.cuh"

#define DIA_EVAL_INST(MKV, VAR, NWV, QFV, MBV, SPV, F2V)                                               \
    namespace dia {                                                                            \
    bool kernel_info_##MKV##_##VAR(KernelInfo *o) {                                            \
        using S = EvalShape<MKV, NWV, QFV, SPV, F2V>;                                               \
        o->mk = MKV;                                                                           \
        o->variant = VAR;                                                                      \
        o->nw = NWV;                                                                           \
        o->qf = QFV;                                                                           \
        o->minb = MBV;   /* prefetch flag */                                      \
        o->f2 = F2V;     /* packed float2 FMAs */                                                                         \
        o->th = S::TH;                                                                         \
        o->nt = S::NT;                                                                         \
        o->smem = S::SMEM;                                                                     \
        o->np = S::NP;                                                                         \
        o->kp = S::KP;                                                                         \
        o->fn[kModeGrad] = (const void *)&eval_kernel<MKV, NWV, QFV, MBV, SPV, kModeGrad, F2V>;     \
        o->fn[kModeForward] = (const void *)&eval_kernel<MKV, NWV, QFV, MBV, SPV, kModeForward, F2V>; \
        o->fn_bg[kModeGrad] = (const void *)&eval_kernel<MKV, NWV, QFV, MBV, SPV, kModeGrad, F2V, 1>; \
        o->fn_bg[kModeForward] =                                                               \
            (const void *)&eval_kernel<MKV, NWV, QFV, MBV, SPV, kModeForward, F2V, 1>;         \
        return true;                                                                           \
    }                                                                                          \
    }

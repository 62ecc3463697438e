// Instantiation helper: DIA_EVAL_INST(MK, NW, QF) defines kernel_info_<MK>().
#pragma once

#include "dia_dispatch.h"
#include "dia_eval.cuh"

#define DIA_EVAL_INST(MKV, NWV, QFV)                                                   \
    namespace dia {                                                                    \
    bool kernel_info_##MKV(KernelInfo *o) {                                            \
        using S = EvalShape<MKV, NWV, QFV>;                                            \
        o->mk = MKV;                                                                   \
        o->nw = NWV;                                                                   \
        o->qf = QFV;                                                                   \
        o->th = S::TH;                                                                 \
        o->nt = S::NT;                                                                 \
        o->smem = S::SMEM;                                                             \
        o->np = S::NP;                                                                 \
        o->kp = S::KP;                                                                 \
        o->fn[kModeGrad] = (const void *)&eval_kernel<MKV, NWV, QFV, kModeGrad>;       \
        o->fn[kModeForward] = (const void *)&eval_kernel<MKV, NWV, QFV, kModeForward>; \
        return true;                                                                   \
    }                                                                                  \
    }

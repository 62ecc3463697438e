// Fused evaluation kernels for kernel sides: 13 15
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(13, 13, 8)
DIA_EVAL_INST(15, 8, 8)

// Fused evaluation kernels for kernel sides: 21
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(21, 7, 8)

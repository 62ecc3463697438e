// Fused evaluation kernels for kernel sides: 23
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(23, 8, 8)

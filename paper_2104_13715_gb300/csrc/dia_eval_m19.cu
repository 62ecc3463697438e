// Fused evaluation kernels for kernel sides: 19
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(19, 10, 8)

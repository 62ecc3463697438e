// Fused evaluation kernels for kernel sides: 17
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(17, 9, 8)

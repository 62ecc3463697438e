// Fused evaluation kernels for kernel sides: 29
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(29, 10, 8)

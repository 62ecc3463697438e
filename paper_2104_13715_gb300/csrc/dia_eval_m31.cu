// Fused evaluation kernels for kernel sides: 31
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(31, 11, 8)

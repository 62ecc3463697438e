// Fused evaluation kernels for kernel sides: 25
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(25, 9, 8)

// Fused evaluation kernels for kernel sides: 27
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(27, 9, 8)

// Fused evaluation kernels for kernel sides: 9 11
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(9, 9, 8)
DIA_EVAL_INST(11, 11, 8)

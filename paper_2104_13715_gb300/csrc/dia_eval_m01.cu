// Fused evaluation kernels for kernel sides: 1 3 5 7
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(1, 8, 8)
DIA_EVAL_INST(3, 8, 8)
DIA_EVAL_INST(5, 8, 8)
DIA_EVAL_INST(7, 8, 8)

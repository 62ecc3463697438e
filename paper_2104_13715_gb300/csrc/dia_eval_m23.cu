// Fused evaluation kernels for kernel sides [23] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(23, 0, 8, 4, 0, 0, 0)
DIA_EVAL_INST(23, 1, 8, 4, 1, 0, 0)
DIA_EVAL_INST(23, 2, 8, 4, 1, 0, 1)

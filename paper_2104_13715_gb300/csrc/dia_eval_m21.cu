// Fused evaluation kernels for kernel sides [21] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(21, 0, 7, 4, 1, 0)
DIA_EVAL_INST(21, 1, 7, 8, 1, 0)
DIA_EVAL_INST(21, 2, 8, 4, 1, 0)

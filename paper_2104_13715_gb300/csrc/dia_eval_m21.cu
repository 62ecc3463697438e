// Fused evaluation kernels for kernel sides [21] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(21, 0, 8, 4, 0, 0, 1)
DIA_EVAL_INST(21, 1, 8, 4, 0, 0, 0)
DIA_EVAL_INST(21, 2, 8, 4, 1, 0, 0)
DIA_EVAL_INST(21, 3, 7, 4, 0, 0, 0)

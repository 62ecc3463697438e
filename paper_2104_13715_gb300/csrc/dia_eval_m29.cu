// Fused evaluation kernels for kernel sides [29] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(29, 0, 8, 4, 0, 2, 1)
DIA_EVAL_INST(29, 1, 10, 4, 0, 0, 0)
DIA_EVAL_INST(29, 2, 10, 4, 1, 0, 0)

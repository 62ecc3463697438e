// Fused evaluation kernels for kernel sides [27] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(27, 0, 8, 4, 0, 2, 1)
DIA_EVAL_INST(27, 1, 9, 4, 0, 0, 0)
DIA_EVAL_INST(27, 2, 9, 4, 1, 0, 0)

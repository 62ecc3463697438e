// Fused evaluation kernels for kernel sides [1, 3, 5, 7] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(1, 0, 8, 8, 0, 0, 0)
DIA_EVAL_INST(3, 0, 8, 8, 0, 0, 0)
DIA_EVAL_INST(5, 0, 8, 8, 0, 0, 0)
DIA_EVAL_INST(7, 0, 8, 4, 0, 0, 0)
DIA_EVAL_INST(7, 1, 8, 8, 0, 0, 0)
DIA_EVAL_INST(7, 2, 8, 4, 0, 0, 1)

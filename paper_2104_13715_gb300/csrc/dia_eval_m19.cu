// Fused evaluation kernels for kernel sides [19] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(19, 0, 8, 4, 1, 1, 0)
DIA_EVAL_INST(19, 1, 8, 4, 0, 1, 0)
DIA_EVAL_INST(19, 2, 10, 4, 0, 0, 0)
DIA_EVAL_INST(19, 3, 8, 4, 1, 1, 1)
DIA_EVAL_INST(19, 4, 8, 4, 0, 1, 1)

// Fused evaluation kernels for kernel sides [25] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(25, 0, 9, 8, 1)
DIA_EVAL_INST(25, 1, 9, 4, 1)
DIA_EVAL_INST(25, 2, 13, 4, 1)
DIA_EVAL_INST(25, 3, 9, 4, 2)
DIA_EVAL_INST(25, 4, 7, 8, 1)
DIA_EVAL_INST(25, 5, 13, 8, 1)

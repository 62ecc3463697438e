// Fused evaluation kernels for kernel sides [9, 11] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(9, 0, 8, 4, 0, 2, 1)
DIA_EVAL_INST(9, 1, 8, 4, 0, 1, 0)
DIA_EVAL_INST(9, 2, 8, 8, 0, 1, 0)
DIA_EVAL_INST(9, 3, 8, 4, 0, 1, 1)
DIA_EVAL_INST(9, 4, 8, 4, 0, 2, 0)
DIA_EVAL_INST(11, 0, 8, 4, 0, 1, 1)
DIA_EVAL_INST(11, 1, 8, 4, 1, 1, 0)
DIA_EVAL_INST(11, 2, 8, 4, 0, 1, 0)
DIA_EVAL_INST(11, 3, 12, 4, 0, 0, 0)

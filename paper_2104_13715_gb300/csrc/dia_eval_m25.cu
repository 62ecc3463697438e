// Fused evaluation kernels for kernel sides [25] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(25, 0, 12, 4, 1, 1, 1)
DIA_EVAL_INST(25, 1, 12, 4, 0, 1, 0)
DIA_EVAL_INST(25, 2, 12, 4, 1, 1, 0)
DIA_EVAL_INST(25, 3, 13, 4, 0, 0, 0)
DIA_EVAL_INST(25, 4, 12, 2, 0, 1, 0)
DIA_EVAL_INST(25, 5, 12, 4, 0, 1, 1)
DIA_EVAL_INST(25, 6, 13, 4, 0, 0, 1)

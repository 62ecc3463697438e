// Fused evaluation kernels for kernel sides [17] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(17, 0, 8, 4, 0, 1, 0)
DIA_EVAL_INST(17, 1, 8, 4, 1, 1, 0)
DIA_EVAL_INST(17, 2, 8, 4, 1, 1, 1)

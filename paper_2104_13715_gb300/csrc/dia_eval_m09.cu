// Fused evaluation kernels for kernel sides [9, 11] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(9, 0, 9, 8, 1)
DIA_EVAL_INST(11, 0, 11, 8, 1)

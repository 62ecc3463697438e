// Fused evaluation kernels for kernel sides [21] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(21, 0, 7, 8, 1)

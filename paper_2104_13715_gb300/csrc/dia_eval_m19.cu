// Fused evaluation kernels for kernel sides [19] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(19, 0, 10, 8, 1)

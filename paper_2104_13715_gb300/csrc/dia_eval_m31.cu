// Fused evaluation kernels for kernel sides [31] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(31, 0, 11, 8, 1)

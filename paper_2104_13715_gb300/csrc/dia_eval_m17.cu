// Fused evaluation kernels for kernel sides [17] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(17, 0, 9, 8, 1)

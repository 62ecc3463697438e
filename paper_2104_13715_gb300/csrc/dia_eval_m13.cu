// Fused evaluation kernels for kernel sides [13, 15] (generated by gen_instances.py)
#include "dia_eval_inst.cuh"

DIA_EVAL_INST(13, 0, 12, 4, 1, 1, 0)
DIA_EVAL_INST(13, 1, 12, 4, 0, 1, 0)
DIA_EVAL_INST(13, 2, 13, 4, 0, 0, 0)
DIA_EVAL_INST(13, 3, 12, 4, 1, 1, 1)
DIA_EVAL_INST(13, 4, 12, 4, 0, 2, 1)
DIA_EVAL_INST(15, 0, 12, 4, 0, 2, 1)
DIA_EVAL_INST(15, 1, 12, 4, 1, 1, 0)
DIA_EVAL_INST(15, 2, 12, 4, 0, 1, 0)
DIA_EVAL_INST(15, 3, 12, 4, 1, 1, 1)

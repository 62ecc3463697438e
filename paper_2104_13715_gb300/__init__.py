"""GB300-native (sm_103a) DIA kernel fit: M = R (x) K + B0 fitted to I (PyTorchDIA method).

The compute path is the CUDA library ``_dia_cuda.so`` behind the C ABI of
``include/dia.h``; ``paper_2104_13715_gb300.native`` is its ctypes binding
(import it explicitly; the seeded input generator ``.synth`` needs no library).
"""
__version__ = "0.1.0"

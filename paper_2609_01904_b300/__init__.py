"""B300-native (sm_103a) MPS / quantized-tensor-train stepper for the explicit
2D acoustic FDTD scheme (Nemeth & Vattay, Eq. 17).

The compute path is the CUDA library ``libqtt.so`` behind the C ABI in
``include/qtt.h``; :mod:`paper_2609_01904_b300.qtt` is its ctypes binding and
:mod:`paper_2609_01904_b300.build` compiles the library in-tree.
"""

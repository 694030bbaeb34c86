"""GB300-native quasi-Newton / L-BFGS implicit-Euler solver for hyperelastic tets.

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through the ``extern "C"`` entry points declared in ``include/hqn.h``;
``paper_1604_07378_gb300.hqn`` is the thin ctypes binding over them.
"""

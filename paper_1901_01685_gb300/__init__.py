"""GB300-native ILUT-smoothed p-multigrid for Galerkin IgA Poisson problems.

The CUDA path lives in ``csrc/`` and is reached through the C-ABI declared in
``include/pmg.h``; ``pmg`` is the thin ctypes binding.  Import the binding
explicitly (``from paper_1901_01685_gb300 import pmg``); importing the package
itself loads nothing.
"""

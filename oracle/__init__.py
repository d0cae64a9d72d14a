"""FP64 CPU oracle for the VANSE lattice Boltzmann step (test infrastructure).

``oracle.oracle``    — C oracle (literal push form, OpenMP) via ctypes.
``oracle.torch_ref`` — independent pull-form restatement in PyTorch float64 on
                       CPU, used for cross-checks and reference gradients.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
"""

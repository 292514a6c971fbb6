"""GB300-native explicit finite-volume Euler residual + Runge-Kutta library
(the data-parallel hot path of the SENSEI solver, arXiv 2305.18057).

The compute path is the CUDA library ``csrc/`` builds into ``libsensei.so``;
``paper_2305_18057_gb300.sensei`` is its thin ctypes binding (argument
marshalling only).  ``workloads`` makes seeded synthetic inputs.
"""

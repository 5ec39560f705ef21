"""GB300 (sm_103a) implementation of the PTTK hot path of Khan & Saibaba,
"Parametric kernel low-rank approximations using tensor train decomposition".

The compute lives in libpttk.so (C ABI: include/pttk.h); ``pttk`` is its binding and
``workloads`` holds the seeded synthetic inputs.
"""

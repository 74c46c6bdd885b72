"""GB300-native two-timescale multicomponent lattice Boltzmann (D3Q19).

The compute path is the CUDA library built from ``csrc/`` behind the C ABI
of ``include/lbm.h``; ``lbm`` is its ctypes binding and ``workloads`` holds
the seeded synthetic inputs.
"""

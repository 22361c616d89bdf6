"""B300-native sparse-monomial engine and affine-normal directions.

The compute path lives in the C-ABI library ``libpolylab.so`` (CUDA kernels for
sm_103a, sources under ``csrc/``); :mod:`.polylab` is its thin ctypes binding
and :mod:`.workloads` draws seeded synthetic inputs.
"""

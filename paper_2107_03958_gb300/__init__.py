"""GB300-native FFT convolution with weakly singular kernels and the Lippmann-Schwinger solver
of arXiv 2107.03958 (Tiwari, Pandey, Paul, Anand).

The compute path is the CUDA library built from ``csrc/`` (C ABI in ``include/wsconv.h``);
``api`` marshals torch tensors into it.  ``inputs`` generates the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401


def __getattr__(name):
    # the torch-facing API is imported lazily so that `inputs` works without torch/CUDA
    if name in ("ConvPlan", "ls_solve", "measure_peaks", "default_scale"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)

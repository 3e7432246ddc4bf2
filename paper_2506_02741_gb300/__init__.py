"""vtsplat: GB300-native differentiable splatting of view-tied isotropic
Gaussians (VTGaussian-SLAM, arXiv 2506.02741).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/vtsplat.h``); ``api`` is its PyTorch binding and ``autograd`` wraps
it in a ``torch.autograd.Function``.  Importing the package itself loads
nothing heavy, so the input generator ``synthetic`` can be used on its own.
"""

import importlib

__all__ = ["api", "autograd", "build", "synthetic", "tracking"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

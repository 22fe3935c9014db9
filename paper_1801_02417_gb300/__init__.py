"""GB300-native Polarized SARA primal-dual imager (arXiv:1801.02417).

The compute path is the CUDA library libpolsara.so (C ABI in include/polsara.h);
``binding`` marshals arguments to it, ``solver`` drives Algorithm 2 on top of it,
``inputs`` draws seeded synthetic problems. Importing the package does not load
the library; the first call that needs it does, and fails loudly if it is absent.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "binding", "solver"]

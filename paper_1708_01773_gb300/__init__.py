"""GB300-native cell integration and CSR assembly for grad-conforming Lagrangian
Q_p hexahedra (FEMPAR, arXiv 1708.01773).

The compute path is the CUDA library ``libfeasm.so`` (built from ``csrc/``);
``feasm`` is its thin ctypes binding, ``autograd`` the compliance
``torch.autograd.Function``, ``inputs`` the seeded synthetic workloads.
Importing the package loads nothing; ``feasm`` loads the library on first use
and raises if it is missing.
"""
__all__ = ["inputs", "feasm", "autograd"]

"""GB300 library for the displacement-probed estimator of Tr(P A^{-1}).

The compute path is the CUDA library libptrace.so (C ABI in include/ptrace.h);
``ptrace`` is its ctypes binding and ``autograd`` the torch.autograd wrapper.
``inputs`` generates the seeded synthetic gauge fields.  Importing the package
does not load the library; the first call that needs it does, and raises if
it has not been built.
"""
__all__ = ["ptrace", "inputs"]

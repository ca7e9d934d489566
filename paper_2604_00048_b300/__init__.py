"""B300-native Whittaker-Henderson smoother: banded SPD solve as a differentiable layer.

The compute path is the CUDA library built from csrc/ (C-ABI declared in include/ws.h);
this package only marshals arguments to it. There is no CPU fallback: importing
the binding fails loudly when the shared library is missing.
"""
__all__ = ["synth"]

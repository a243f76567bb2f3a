"""GB300-native hot path of the 2D-axisymmetric GR particle-in-cell method of
arXiv:2511.17701: GR pusher, charge-conserving deposit and GR Maxwell update as
sm_103a CUDA kernels behind the C ABI of include/grpic.h (libgrpic.so), with a
thin ctypes binding. PyTorch supplies device memory and streams only."""
from ._build import build
from .binding import (ADVANCE, FIELD_MONOPOLE, FIELD_USER, FIELD_VERTICAL, FIELD_WALD, FIELD_ZERO,
                      NPLANES, PREDICT, GrpicError, Sim, lib)


__all__ = ["build", "lib", "Sim", "GrpicError", "FIELD_ZERO", "FIELD_WALD", "FIELD_VERTICAL",
           "FIELD_USER", "FIELD_MONOPOLE", "PREDICT", "ADVANCE", "NPLANES", "PushAdjoint", "push_adjoint"]


def __getattr__(name):  # the autograd Function needs torch; import it on first use
    if name in ("PushAdjoint", "push_adjoint"):
        from . import adjoint
        return getattr(adjoint, name)
    raise AttributeError(name)

"""GB300-native long-range molecular dynamics after arXiv 1212.0262.

The force evaluation inside the fourth-order symplectic integrator of Sec. 3 for
the HMF (Eqs. 2, 5-7), Ring (Eqs. 1, 8-9) and 2D self-gravitating (Eq. 3)
models, and 3D self-gravitating particles and 1D self-gravitating sheets with the
same coupling, as
hand-written sm_103a CUDA kernels behind the C ABI of include/md.h.
"""
from . import binding
from .binding import MDError
from .system import Ensemble, ShardGroup, System, shard_range

HMF, RING, GRAV2D, GRAV3D, SHEET1D = 0, 1, 2, 3, 4
FP64, MIXED = 0, 1

__all__ = ["binding", "MDError", "System", "Ensemble", "ShardGroup", "shard_range", "HMF", "RING", "GRAV2D", "GRAV3D", "SHEET1D", "FP64", "MIXED"]

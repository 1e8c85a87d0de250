"""GB300-native hot path of 3-D PeriDEM (bond-based peridynamics with
critical-stretch breaking, nodal contact, rigid walls, velocity-Verlet) and its
bulk-stress MLP surrogate.  The compute runs in libpd.so (csrc/, sm_103a);
``pd`` is the ctypes binding and ``scenarios`` the seeded workloads."""
from . import scenarios  # noqa: F401

__all__ = ["scenarios", "pd"]

"""GB300-native DPD fluid step (cell-list binning, pair forces with a
stateless pair-symmetric noise, velocity-Verlet in periodic boxes) behind a
C ABI (libdpd.so).  See ``dpd`` for the single-box binding and ``batch`` for
the multi-box and served forms."""

from . import workloads  # noqa: F401

__all__ = ["workloads", "dpd"]

"""GB300-native synchronization check over simulated memory-access records.

The check (data races, redundant barriers, barrier divergence) is the
detection half of the memory-model method of arXiv 1905.01833, Sec. 3.2. It
runs in hand-written CUDA kernels for sm_103a behind the C ABI of
include/simulee.h; `simulee` is the thin Python binding of that ABI.
"""
from . import simulee
from .simulee import Checker, DeviceTrace, SimuleeError, to_device

__all__ = ["simulee", "Checker", "DeviceTrace", "SimuleeError", "to_device"]

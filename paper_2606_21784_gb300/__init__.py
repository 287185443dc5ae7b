"""GB300-native persistent call-auction engine (KineticSim's method).

The CUDA library ``_lib/libkineticsim.so`` (C ABI in ``include/kineticsim.h``)
runs the whole simulation; ``kineticsim`` is its ctypes binding and
``workloads`` describes the seeded synthetic ensembles.
"""
__all__ = ["kineticsim", "workloads", "build"]

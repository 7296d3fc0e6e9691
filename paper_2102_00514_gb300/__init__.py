"""GB300-native parallel iterated extended (IEKS) and cubature sigma-point
(IPLS) Kalman smoother (Yaghoobi et al., ICASSP 2021).

* ``pes``    - binding of the C ABI (``include/pes.h``, ``libpes.so``)
* ``synth``  - seeded synthetic coordinated-turn / bearings workloads
* ``build``  - in-tree build of the native libraries
"""
__all__ = ["pes", "synth", "build"]

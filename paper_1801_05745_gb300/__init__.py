"""GB300-native UFalcon lightcone library: particles -> (shell, HEALPix RING
pixel) -> per-shell count maps -> Born-approximation kappa -> moments, PDF and
covariance, with an adjoint for parameter gradients (Sgier et al., Sec. 2.3-3.3).

The compute runs in the CUDA shared library ``libufalcon_gb300.so`` built from
``csrc/``; :mod:`paper_1801_05745_gb300.api` is the Python binding of its C
ABI.  Importing this package does not load the library; ``api`` does, and it
raises if the library is missing.
"""
__all__ = ["api", "synth", "workloads"]

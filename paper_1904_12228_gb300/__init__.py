"""GB300-native differentiable Monte Carlo ray tracing with edge sampling.

The CUDA library is loaded lazily by :mod:`paper_1904_12228_gb300.drt`;
importing the package itself does not touch the GPU.
"""
__all__ = ["scenegen"]

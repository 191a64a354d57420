"""GB300-native differentiable spherical rasterizer of 2D Gaussian surfels
into LiDAR range images (the mapping hot path of "Real-Time LiDAR Gaussian
Splatting SLAM via Geometry-Aware Covariance Coupling").

Submodules are imported lazily: ``scenes`` (seeded synthetic inputs) has no
dependency on the compiled library; ``lib`` (the C-ABI binding), ``render``
(autograd functions), ``mapping`` (Adam mapping loop), ``batch`` (persistent
batched launch) and ``serve`` (serving loop) load ``liblgs.so`` and fail
loudly when it is missing.
"""
__all__ = ["scenes", "lib", "render", "mapping", "batch", "serve"]

"""GB300-native differentiable 3D Gaussian Splatting rasterizer with camera
pose gradients (the data-parallel hot path of joint pose + 3DGS optimisation).

The compute path is the C-ABI library ``libgsplat_gb300.so`` built from
``csrc/``; ``_lib`` binds it, ``autograd`` wraps it for torch. Submodules are
imported on demand so that ``synth`` (input generation) stays usable without
the compiled library.
"""
__all__ = ["synth", "_lib", "autograd", "pose", "build"]

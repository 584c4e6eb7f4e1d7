"""GB300-native renderer for the OSOG optical forward model (arxiv 2606.21381).

The hot path (particle footprints -> OPD composition -> exit wave -> pupil
filtering by FFT -> intensity) runs in the CUDA library libosog behind the
C ABI of ``include/osog.h``.  ``render.Renderer`` is the torch-facing entry;
``scenes`` draws seeded synthetic workloads.
"""
__all__ = ["Renderer", "scenes", "build"]


def __getattr__(name):
    if name == "Renderer":
        from .render import Renderer
        return Renderer
    raise AttributeError(name)

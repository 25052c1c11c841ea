"""GB300-native Splotch hot path (Dykes et al., "Splotch: porting and optimizing for
the Xeon Phi"): per-particle raster, tile binning, Gaussian splat and final transform
in hand-written sm_103a CUDA behind the C ABI of ``include/splotch.h``.

Submodules load lazily so that ``synth`` (input generation) imports without CUDA:
``render`` (Scene, Plan, RenderParams), ``build`` (compile the library), ``synth``.
"""
import importlib

__all__ = ["render", "build", "synth", "autotune", "serve"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

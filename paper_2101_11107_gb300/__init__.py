"""GB300-native D3Q27 central-Hermite-moment MRT lattice Boltzmann library.

Import is light: ``inputs`` (seeded geometry and waveforms) needs no GPU; ``lbm`` (the
binding of the CUDA C-ABI) loads the library on first use and raises if it is missing.
"""
import importlib

from . import inputs  # noqa: F401

__all__ = ["inputs", "lbm", "Domain"]


def __getattr__(name):
    if name == "lbm":
        return importlib.import_module(__name__ + ".lbm")
    if name == "Domain":
        return importlib.import_module(__name__ + ".lbm").Domain
    raise AttributeError(name)

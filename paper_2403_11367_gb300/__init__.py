"""GB300 (sm_103a) relocalization hot path of 3DGS-ReLoc (arXiv 2403.11367).

The compute path is the CUDA library behind include/reloc.h
(``_lib/libreloc.so``); ``reloc`` is its Python binding.  Build with
``paper_2403_11367_gb300.build.build()``.
"""
import importlib

__all__ = ["build", "reloc"]


def __getattr__(name):
    if name in ("reloc", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

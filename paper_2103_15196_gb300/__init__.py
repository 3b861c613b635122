"""GB300 (sm_103a) CSPH-TVD + Exner shallow-water/sediment solver.

The compute path is the in-tree CUDA library (``_lib/libswe.so``, C ABI in
``include/swe.h``); ``swe.Solver`` is its Python binding.  ``inputs`` builds
the seeded synthetic terrains and states.
"""


def __getattr__(name):
    if name in ("Solver", "SweError", "load_library"):
        from . import swe
        return getattr(swe, name)
    raise AttributeError(name)

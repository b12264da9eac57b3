"""B300-native (sm_103a) Super-Droplet Method coalescence step.

* ``paper_2101_06318_b300.sdm``     -- binding of libsdm.so (include/sdm.h)
* ``paper_2101_06318_b300.inputs``  -- seeded synthetic initial states
* ``paper_2101_06318_b300.build``   -- nvcc build of libsdm.so

The binding is imported lazily so that ``inputs`` can be used without a GPU.
"""
__all__ = ["sdm", "inputs", "build"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

"""GB300-native parallel orbital-updating (ParO) plane-wave Kohn-Sham hot path.

`paro` (the ctypes binding of libparo.so) is imported lazily so that the seeded input generators
in `inputs` can be used without the compiled library.
"""
__all__ = ["inputs", "paro"]

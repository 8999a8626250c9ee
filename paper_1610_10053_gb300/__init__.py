"""GB300-native implicit hydrodynamics JFNK inner loop (MUSIC benchmark paper).

The compute path lives in the CUDA library ``libmusic`` (``csrc/``) behind the
C ABI declared in ``include/music.h``; ``binding`` is its thin ctypes
binding.  Importing this package does not load the library: ``binding``
loads it on first use and raises if it is missing.
"""
__all__ = ["inputs", "binding", "build"]

"""GB300 (sm_103a) implementation of the time-dependent-basis in-situ compressor.

Submodules:
  tdb        - ctypes binding of libtdb (the C ABI in include/tdb.h)
  build_lib  - in-tree nvcc build of libtdb.so
  synth      - seeded synthetic snapshot streams (inputs only)
Nothing is imported eagerly, so importing the package never touches the GPU.
"""

__all__ = ["tdb", "build_lib", "synth"]

"""GB300-native time-explicit DG for the acoustic wave system on vertex-mapped pyramids.

The compute path lives in the CUDA shared library ``libpyrdg.so`` (sources in
``csrc/``, C-ABI in ``include/pyrdg.h``); ``binding`` is its thin ctypes layer.
``mesh`` holds the seeded synthetic inputs. Importing the package does not load
the library: ``from paper_1502_07703_gb300 import binding`` does, and fails
loudly when the library has not been built.
"""

__all__ = ["mesh", "binding", "build"]

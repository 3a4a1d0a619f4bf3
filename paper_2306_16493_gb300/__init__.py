"""GB300-native electron-phonon Wannier interpolation (EPWI) transport hot path.

Submodules are imported lazily so that the synthetic-input generator can be used
without loading the CUDA library:

* ``synth``  - seeded synthetic Wannier-basis systems (inputs only).
* ``epwi``   - ctypes binding of the C ABI in ``include/epwi.h`` (requires the
  compiled ``libepwi.so``; raises if it is missing).
"""

"""GB300-native Neural Incident Radiance Cache (NIRC) two-level Monte Carlo hot path.

* ``scenes``  -- seeded synthetic inputs (scenes, initial parameters, training batches)
* ``nirc``    -- thin ctypes binding of the C-ABI library ``libnirc.so``
  (CUDA kernels for sm_103a); importing it loads the library and fails loudly
  if it has not been built.
"""

"""GB300-native well-balanced diffuse-interface finite-volume solver.

The solver itself is the C-ABI library ``libfv`` (CUDA, sm_103a); ``fv`` is its
thin ctypes binding and ``cases`` builds seeded synthetic inputs.
"""

"""GB300-native PPML operator-splitting hydro step (Kulikov & Vorobyov, arXiv:1607.01105).

The compute path is ``libppml.so`` (hand-written sm_103a CUDA behind a C ABI declared in
``include/ppml.h``); ``paper_1607_01105_gb300.ppml`` is its thin ctypes binding.  Nothing
is imported eagerly, so the seeded input generators (``paper_1607_01105_gb300.inputs``)
stay usable on machines without a GPU.
"""

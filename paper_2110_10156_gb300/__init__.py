"""GB300-native all-shift NGF similarity (Cross-Sim-NGF hot path).

The compute path is the CUDA library ``libcs_ngf.so`` (sources in ``csrc/``,
C ABI in ``include/cs_ngf.h``); ``cs_ngf`` is its thin Python binding and
``synth`` builds seeded synthetic inputs.
"""

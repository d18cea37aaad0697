"""GB300-native batched solver for CAMP's coupled multiphase chemistry ODE system.

The CUDA path lives in ``libcamp.so`` (built from ``csrc/``) behind the C ABI
declared in ``include/camp.h``; ``camp`` is its thin Python binding.  Importing
this package does not load the library; ``workloads`` (seeded inputs) has no
dependency on it.
"""

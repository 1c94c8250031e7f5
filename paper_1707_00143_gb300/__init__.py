"""GB300-native (sm_103a) hot path of the Navigating Spreading-out Graph.

The compute lives in ``csrc/`` (hand-written CUDA behind a C ABI, declared in
``include/nsg.h``); ``capi`` is the thin ctypes binding with the same names.
``datagen`` draws the seeded synthetic inputs.  Importing the package loads
nothing; ``capi`` loads ``libnsg.so`` on first use and fails loudly if it is
missing.
"""

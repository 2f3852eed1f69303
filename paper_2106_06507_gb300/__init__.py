"""GB300-native Berends-Giele n-gluon tree amplitudes (colour-ordered with the
full colour sum, and colour-dressed with sampled colours).

The compute path is the C-ABI library ``libbg.so`` (hand-written sm_103a
CUDA); :mod:`paper_2106_06507_gb300.bg` is its thin ctypes binding.  Importing
this package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""

"""GB300-native (sm_103a) atomistic spin hot path of arXiv:1901.11350.

The compute path is the C-ABI library ``libspirit_gb.so`` built from
``csrc/``; :mod:`.binding` marshals arguments to it.  Importing the package
does not load the library; the first call that needs it does, and raises if
the CUDA extension is missing.
"""

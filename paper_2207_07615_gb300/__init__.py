"""GB300-native PLSS (projected linear systems solver, arXiv 2207.07615).

The compute path is a C-ABI CUDA library (libplss.so, sm_103a); the Python
binding in `plss` only marshals arguments. Importing this package does not
load the library; `plss.lib()` does, and fails loudly when it is missing.
"""

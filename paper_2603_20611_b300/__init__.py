"""B300-native (sm_103a) slice projection operator of GaussianPile (arXiv 2603.20611).

``binding`` holds the ctypes marshalling of the C ABI in ``include/gp.h`` (it
loads ``libgaussianpile.so`` and fails loudly without it); ``synth`` the seeded
synthetic inputs; ``build`` the nvcc build step.  Submodules are imported on
demand so that ``synth`` stays usable without the compiled library.
"""

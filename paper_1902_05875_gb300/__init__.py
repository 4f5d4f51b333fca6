"""GB300 Taylor-expansion FMM for the 3-D Helmholtz equation in layered media.

``tefmm`` is the binding of the C-ABI library (``include/tefmm.h``);
``workloads`` holds the seeded synthetic inputs.  Importing the package loads
nothing; ``tefmm.load()`` (or ``tefmm.Plan``) loads the CUDA library.
"""

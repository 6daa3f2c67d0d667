"""GB300-native hybrid lattice-Boltzmann / FENE-P droplet solver.

The compute path is the CUDA library ``liblbfe.so`` (built from ``csrc/``)
behind the C ABI declared in ``include/lbfe.h``; the Python modules here only
marshal arguments into it.  Importing the package does not load the library;
``paper_1411_2181_gb300.lbfe`` does, and fails loudly if it is missing.
"""

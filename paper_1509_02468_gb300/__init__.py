"""GB300-native bilateral-filter graph filters (Knyazev & Malyshev, 2015).

The compute path is the CUDA library ``libbf.so`` (C-ABI declared in ``include/bf.h``);
``paper_1509_02468_gb300.bf`` is its thin ctypes binding.  ``synth`` holds the seeded
input generators.  Importing this package does not load the library; importing ``bf``
does, and fails loudly if it is missing.
"""
__version__ = "0.1.0"

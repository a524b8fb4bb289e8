"""GB300-native Graph Normalization (arXiv 2605.05330): the WRGN iteration on a sparse
conflict graph, run until the state binarises into a maximal independent set.

The compute path is the CUDA library ``libgn.so`` (sources in ``csrc/``, C ABI in
``include/gn.h``).  ``gn`` is its thin Python binding; ``inputs`` holds the seeded
synthetic workload generators.  Importing this package does not load the library;
the first call into ``gn`` does, and fails loudly if it has not been built.
"""
__all__ = ["gn", "inputs"]

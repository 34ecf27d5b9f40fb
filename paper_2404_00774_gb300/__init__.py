"""GB300-native (sm_103a) implementation of the SOAR spilled-IVF hot path.

SOAR (Sun et al., "SOAR: Improved Indexing for Approximate Nearest Neighbor
Search", arXiv 2404.00774) assigns every datapoint to its nearest centroid
and to extra "spilled" centroids chosen by an orthogonality-amplified
residual loss (Theorem 3.1), and searches the resulting inverted-file index
by probing the top-t partitions, deduplicating spilled copies and keeping
the top-k inner products.

The compute lives in ``libsoar.so`` (CUDA, built by ``build.py``) behind the
C ABI of ``include/soar.h``; ``binding`` is its Python marshalling layer.
Importing this package loads nothing: call ``binding.load()``.
"""

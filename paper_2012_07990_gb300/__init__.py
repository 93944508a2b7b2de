"""g2: GB300-native frontier-driven graph traversal (edgeset.apply and the
algorithms built on it), a CUDA library behind a C ABI.

Importing the package loads nothing native; ``paper_2012_07990_gb300.g2``
loads ``libg2.so`` and fails loudly when it is missing.
"""

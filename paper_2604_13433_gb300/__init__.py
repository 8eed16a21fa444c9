"""PackSELL on GB300: delta-value packed sliced-ELLPACK SpMV, SpMM and PCG.

The compute path is the C-ABI library ``libpacksell.so`` (CUDA, sm_103a),
loaded by :mod:`paper_2604_13433_gb300.packsell`. Importing this package does
not load it; the first call through the binding does, and raises if the
library has not been built.
"""
__all__ = ["inputs", "packsell"]

"""GB300-native many-body MD (Tersoff, Stillinger-Weber) in the explicit pairwise-force
form of Fan et al., CPC 2017 (arXiv:1610.03343).

Importing the package is cheap: the CUDA library is loaded on first use of
`paper_1610_03343_gb300.md` (the ctypes binding), never at package import.
"""
__all__ = ["inputs", "md"]

"""GB300-native hybridised multigrid trace solver (lowest-order compatible FEM).

Importing the package is cheap: the CUDA library is loaded on first use by
`paper_2210_11797_gb300.hmg`, which fails loudly if it has not been built.
"""
__all__ = ["inputs", "hmg", "presets"]

"""GB300-native block-coordinate Frank-Wolfe for semi-relaxed optimal transport.

Importing the package loads nothing compiled; `paper_2103_05857_gb300.sr_ot`
loads the CUDA library (and fails loudly if it has not been built).
"""
__all__ = ["workloads"]

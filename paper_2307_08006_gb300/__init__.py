"""GB300-native multiple-walker lambda-ABF engine (arXiv 2307.08006).

Importing the package is cheap: the CUDA library is loaded on first use
by :mod:`paper_2307_08006_gb300.labf`.
"""
__all__ = ["synth"]

"""GB300-native dual-domain convolutional sparse coding (arXiv 1709.09479): coding ADMM and filter update.

Importing the package is cheap. The CUDA library is loaded on first use of ``paper_1709_09479_gb300.csc``.
"""

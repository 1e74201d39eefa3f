"""GB300-native backward-Euler Newton-Krylov-Schwarz step for the SEIRD
reaction-diffusion model (arXiv 2208.01839).

Importing the package does not load the CUDA library; ``paper_2208_01839_gb300.seird``
does, and raises if it is missing.
"""

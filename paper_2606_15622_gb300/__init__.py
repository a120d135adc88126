"""GB300-native cubic Fokker-Planck moment closure.

Importing the package loads nothing compiled; the CUDA library is loaded on
first use through :mod:`paper_2606_15622_gb300.api`.
"""

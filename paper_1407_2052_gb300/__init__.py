"""amrfd: GB300-native FP64 FD-MP5 update (Porth et al. 2014, Sec. 2) for Euler and ideal MHD+GLM.

Importing the package loads nothing compiled; `paper_1407_2052_gb300.amrfd`
loads the CUDA library (libamrfd.so) and fails loudly when it is missing.
"""

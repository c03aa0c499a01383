"""GB300-native unsplit PPM + HLLC hydro update behind a C ABI.

Importing the package is cheap: the CUDA library is loaded on first use by
`paper_2007_05218_gb300.hydro` (ctypes binding of include/hydro.h).
"""
__all__ = ["inputs", "hydro"]

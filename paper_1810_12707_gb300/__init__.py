"""GB300-native pseudo-spectral compressible MHD (isothermal), FP64 or mixed precision, through a
C ABI.

``paper_1810_12707_gb300.mhd`` binds the entry points of ``include/mhd.h``;
``paper_1810_12707_gb300.inputs`` generates the seeded initial conditions;
``paper_1810_12707_gb300.serving`` runs many independent runs with continuous batching;
``paper_1810_12707_gb300.build_lib`` compiles the sm_103a library.
Nothing is loaded at import time.
"""
__all__ = ["mhd", "inputs", "serving", "build_lib"]

"""GB300-native QAOA simulator (arXiv 2309.04841, "Fast Simulation of
High-Depth QAOA Circuits"): cost-vector precompute, phase + transverse-field
mixer layers, energy / ground-state overlap, adjoint gradient and a serving
loop, as hand-written sm_103a CUDA kernels behind a C ABI (include/qaoa.h)."""

"""GB300-native volumetric curvilinear lattice Boltzmann (H. Chen, section 2).

The compute lives in the CUDA library libvlb.so (C-ABI declared in
include/vlb.h); paper_2401_17183_gb300.vlb is its thin ctypes binding. The
library is loaded on first use, not at import, so the seeded input module
(paper_2401_17183_gb300.workloads) imports without a GPU.
"""

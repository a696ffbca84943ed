"""GB300-native hot path of the MXE method (Mendez & Ponga): phase-averaged
EAM free energy and gradients, FIRE relaxation and master-equation mass
transport, as a C-ABI CUDA library (`libmxe.so`, include/mxe.h) with a thin
ctypes binding (`paper_1910_01235_gb300.mxe`).

`workloads` (seeded synthetic inputs) imports without CUDA; `mxe` loads the
CUDA library and raises if it is missing -- there is no CPU fallback."""

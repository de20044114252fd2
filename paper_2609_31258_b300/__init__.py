"""MuCITE ion-pack step on B300 (sm_103a): C-ABI CUDA library
(libmucite.so) with a thin ctypes binding (`mucite`) and the seeded input
generators of the benchmark workloads (`workloads`)."""

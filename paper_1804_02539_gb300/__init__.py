"""GB300-native multigrid-preconditioned CG for multi-patch isogeometric Poisson problems
(Hofer & Takacs, "A parallel multigrid solver for multi-patch Isogeometric Analysis").

The compute path is the CUDA library libigamg.so (csrc/, C ABI in include/igamg.h);
`igamg` is its ctypes binding."""

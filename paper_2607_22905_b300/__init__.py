"""B300-native AlgMortar-PCG: the algebraic multiscale mortar preconditioner inside CG.

The compute path lives in `libalgmortar.so` (hand-written sm_103a CUDA behind a C ABI,
declared in include/algmortar.h).  `binding` marshals arguments to it; `solver` wraps it
for PyTorch users; the seeded synthetic TPFA Darcy systems come from the top-level `synth` module.  Importing the
package does not load the shared library; the first call that needs it does, and fails
loudly if it is missing.
"""
__all__ = ["binding", "solver"]

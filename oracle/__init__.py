"""CPU oracle for the Whittaker-Henderson smoother: test infrastructure only.

Two independent FP64 statements of what the GPU path computes:
  * oracle.dense  - the definition (Eqs. 1-5): dense Omega, LAPACK Cholesky;
  * oracle.banded - Algorithm 1 (banded in-place Cholesky) in plain C with OpenMP,
                    pinned to the dense one by the tests.
Only tests/, the smoke check and the benchmark's CPU-baseline leg may import this
package. The product path (the CUDA library and its Python binding) never does.
"""

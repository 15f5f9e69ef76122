"""FP64 CPU oracle for the Laplace-Beltrami layer-potential solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
tests/, the smoke check and the CPU-baseline leg of the benchmark may import,
call, link or execute it.  It shares no code, header, table or constant with
the CUDA library: it restates each step of the paper's method plainly, in
double precision, to give values the GPU path is compared against.

Modules (paper section in brackets):
  basis      orthonormal polynomials on T0, interpolation, differentiation [4]
  geometry   normals, weights, metric, mean curvature, near lists          [2, 4]
  quadrature adaptive self / near-patch corrected weights                  [4]
  farsum     C direct far sums for S, D, S', S''+D'                        [3, 4]
  layers     discretised potentials, the A2 and A3 operators               [3, 4.2, 4.3]
  gmres      GMRES, dense assembly and the mean-zero solve                 [6]
  hodge      surface div / grad and the harmonic-field decomposition       [2, 5]
  shape      gradient of an A3-solve loss with respect to node positions

Parity status: every function here is pinned by a closed form, an invariant
or a library special case in tests/test_oracle_*.py, except the corrected
weights themselves, whose only pin is their own convergence (tolerance and
rule order) and the closed forms of the potentials they produce.
"""

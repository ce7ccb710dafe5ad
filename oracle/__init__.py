"""CPU FP64 oracle for the vectorised parallel-in-time block solve.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, link or run
this package: only the tests, the smoke check and the CPU-baseline leg of the
benchmark do. It shares no code with the CUDA library; the only module both
import is `synth` (seeded random inputs, no solver arithmetic).

Every routine is a plain, slow, obviously-correct restatement of the paper
(Engwer, Schell & Dreier, "Vectorized Parallel in Time methods for low-order
discretizations with application to Porous Media problems", arXiv 2504.02117),
cited by section / equation / algorithm, in float64. Library primitives
(numpy matmul, scipy sparse products, sparse direct solves, triangular solves)
serve as single steps; there is no blocking or fusion beyond what the cited
definition states.

Modules
-------
coupling : DIRK tableau -> time-stepping matrices A1, A2, B0 (Sec. 2.1,
           Eq. general-system-time-steps, Eq. time-stepping-matrices-multiple-
           parallel-time-steps, Example ex:time-stepping-matrices), splitting
           (Eq. matrix-splitting), pipelined windows (Eq. matrix-equation-
           pipelining).
fv       : cell-centred finite-volume operators used as synthetic workloads
           (conv.-diffusion, nonlinear diffusion-reaction, Richards with the
           van Genuchten-Mualem relations, Eq. RelationshipsThetaK).
krylov   : CholQR2, block classical Gram-Schmidt (two passes), block GMRES with
           Householder least squares, Jacobi and ILU(0) preconditioners.
slab     : coupled residual (Sec. 2.2), all-at-once Kronecker system,
           sequential stepping, fixed-point / defect-correction slab solve
           (Eq. matrix-fixed-point-equation).
newton   : sequential Newton DIRK stepping and the pipelined block Newton
           time stepping of Algorithm 1.

Parity status: every function is pinned by a CPU test (tests/test_oracle_*.py)
except the ones whose header says "parity unpinned".
"""

"""FP64 CPU oracle for the 4D domain-decomposition factorization of det D.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the
CUDA library (no kernels, headers, tables or helpers); it takes its seeded
inputs from ``paper_2211_06902_gb300.synth``, which holds none of the method's
arithmetic.

Plain, slow and written to be checked by eye against the paper
(Saccardi & Giusti, "Four-dimensional domain decomposition for the
factorization of the fermion determinant", Lattice 2022):

* ``lattice``  - gamma matrices, the Wilson-Dirac operator D[U] of Sec. 1/3
                 (optionally with the site-local clover term), its
                 restrictions D_X = P_X D P_X and sparse matrices of them.
* ``geometry`` - the domain decomposition of Sec. 2 (Lambda0^a, Lambda1,
                 dLambda0, dPi, dPi1, Omega0^a, Phi1^a and exterior boundaries).
* ``dd``       - block and frame solves, the operator w = 1 - W_1 (Eqs. Wz,
                 offdiagW1), the roots u_k (Sec. 4), the multi-boson action
                 (Eqs. MBaction, localMB, globalMB), the dense log-det
                 factors of Eq. (detD), the stochastic samples of the
                 reweighting factor of Eq. (rw) and the force of the
                 factorized multi-boson action on the active links.
* ``md``       - block-local molecular dynamics of the active links (Sec. 4,
                 Eq. SFeffN; Sec. 5): pseudofermions for the block
                 determinants, their force, the SU(3) link update and the
                 leapfrog integrator.

Parity status: every function is pinned by a CPU test against closed forms,
identities of the paper or brute force.  W_1 is assembled from the blocks the
paper prints (Sec. 3); it is fixed by the printed upper-right block of Eq.
(offdiagW1), the gamma_5-hermiticity of diag(D^d, D^_{dPi1}) W_1 and the Schur
complement of Eq. (Dtilde), and it satisfies Eqs. (detD) and (WW).  The
molecular dynamics is pinned by the pseudofermion heat-bath identity, finite
differences of its action, SU(3) closure, time reversibility and the dt^2
scaling of the energy violation.
"""

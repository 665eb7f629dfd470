"""Plain FP64 CPU oracle for the displacement-probed estimator of Tr(P A^{-1}).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
link anything in this package.  The product path (the CUDA library and its
Python binding) never touches it, and this package imports nothing from the
product package.

Every function follows a passage of the paper (Switzer, Stathopoulos, Romero,
Laeuchli, Orginos, "Probing for the trace estimation of a permuted matrix
inverse corresponding to a lattice displacement", arXiv 2106.01275) and cites
it by section / equation / theorem.  The code is written for a reader to check
against the paper by eye: no blocking, fusion or reordering beyond what the
definition states.

Modules
-------
lattice      coordinates, storage index, displacement permutation P (Sec. 3)
stencil      displaced neighbourhood N(x,p,k), Eq. (8), multi-p union (Sec. 3.4)
colouring    greedy displaced distance-k colouring, Algorithm 1 (Sec. 3.1), nested variant
bounds       lower bounds on the colour count, Eq. (9), Thms 3.2-3.5, Eq. (13)
rng          SplitMix64 counter-based Z2 / Z4 noise (Sec. 1, Rademacher vectors)
probes       probing vectors, Eq. (4), unbiased form Eq. (5), spin-colour dilution
operators    shifted 4D Laplacian and Wilson-Dirac operators
solvers      textbook CG and BiCGStab in FP64, dense solve for tiny lattices
estimator    Hutchinson / probed trace estimate, statistics, Eqs. (1), (15)-(17)
variance     exact estimator variance, Eq. (2) generalised to non-symmetric B
gradient     adjoint gradient of the probed estimate (extension, not in the paper)
tiles        tile policy of Sec. 3.5 (Table 2)
clearance    clearance of a colouring at other displacements (Thm 3.6, Table 5)
deflation    deflation of the lowest singular triplets, Eq. (6) (Sec. 2.4)
evenodd      even-odd (Schur complement) preconditioning of both operators
clover       clover (Sheikholeslami-Wohlert) term of the Wilson-Dirac operator
multigrid    two-level aggregation multigrid preconditioner, right-preconditioned GMRES

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
value printed in the paper, a closed form, brute force or an invariant, except
where the header of the function says "parity unpinned".
"""

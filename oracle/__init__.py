"""Plain, slow FP64 CPU oracle for IDR(s)stab(l) and M(s)stab(l) (arXiv:1604.06043).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or
execute anything in this package: only the tests, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` use it.  It shares
no code with the CUDA path; both sides take their inputs from the seeded
generators in ``paper_1604_06043_gb300.problems``, which hold none of the
method's arithmetic.

Modules
-------
idrstab   Algorithm 1 (IDRstab) step by step, the Arnoldi start of level s, the
          M(s)stab sequence driver with the fetching point, a textbook BiCGStab
          (the s = l = 1 special case), and the small dense solves.
cnn       the 3D CNN used for the learned initial guess: convolution forward and
          backward, GELU, MSE loss and one Adam step, in FP64.
guess     the selection of a learned initial guess: the residual-minimising
          point of x_prev + span(directions), by its definition.
ilu       ILU(0) split preconditioning (Section 5.1): the factor by its
          definition (IKJ elimination restricted to A's pattern), triangular
          solves, the preconditioned operator and the preconditioned sequence.

Parity pins (see tests/test_oracle_*.py): dense LU on tiny systems, BiCGStab
equivalence for s = l = 1, the finite-termination levels of Section 5.2 (the
printed values in tests/golden/paper_finite_termination.json), the
invariants V = AU, P^T r^(i) = 0, Z^T r = 0, true = recursive residual, the MV
counts of Table 1, and for the CNN central finite differences, scipy's
correlate, tabulated normal-CDF values and the closed form of the first Adam
step; for the guess selection the exact correction in the span, the
closed form of a single direction and the orthogonality of the optimal
residual to A times the directions; for ILU(0) its defining equations checked by dense products, the exact
LU of a tridiagonal matrix, the known fill positions of the 5-point stencil
and dense triangular solves.  Parity unpinned: the MV counts on the synthetic convection-diffusion
sequences (the paper prints none for them) and the choice of fetching point
(the paper gives only a rule of thumb); those are fixed by agreement with this
oracle alone.
"""

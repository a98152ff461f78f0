"""The solve-level parity rule shared by the GPU tests.

Products with A agree within 2, or the two sides stop one cycle apart and the
stopping test was a threshold decision: the side that ran on had a residual
within a factor 10 of tol at the cycle end where the other stopped.

Why a cycle can differ: at s = 8, l = 4 on the 3D convection-diffusion
sequences the iteration amplifies rounding by many orders of magnitude within
a few cycles (the level vectors span ||A||^l; the oracle against itself under
another BLAS thread count or another summation order of its dot products
reaches residuals a factor 2-6 apart from the fourth cycle on), so whether the
last cycle end falls below tol or just above it is decided by rounding.

On the full-size 128^3 sequence even the residual clause does not hold between
two correct runs: the oracle under another BLAS thread count had a cycle whose
residual rose tenfold (4e-7) where its record stopped (3e-9), and needed one
cycle more.  The full-size tests therefore use one_cycle_apart and bound the
number of such systems by what the oracle shows against itself."""


def mvs_match(mvs, ref_mvs, hist, ref_hist, tol):
    """hist / ref_hist: relative residual at the start and at every cycle end."""
    if abs(mvs - ref_mvs) <= 2:
        return True
    cg, co = len(hist) - 1, len(ref_hist) - 1
    if abs(cg - co) != 1:
        return False
    other = ref_hist[cg] if cg < co else hist[co]
    return other <= 10 * tol


def one_cycle_apart(hist, ref_hist):
    """The two solves stopped at adjacent cycle ends."""
    return abs((len(hist) - 1) - (len(ref_hist) - 1)) == 1

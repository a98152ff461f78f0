"""The solve-level parity rule shared by the GPU tests.

Products with A agree within 2, or the two sides stop one cycle apart and the
stopping test was a threshold decision: the side that ran on had a residual
within a factor 10 of tol at the cycle end where the other stopped.  Two
correct FP64 paths (different summation orders; the oracle under another BLAS
thread count too) reach the last cycle ends with residuals that differ by a
few times once the level vectors span many orders of magnitude or the
recycled basis is ill-conditioned, so a test at tol falls one cycle apart."""


def mvs_match(mvs, ref_mvs, hist, ref_hist, tol):
    """hist / ref_hist: relative residual at the start and at every cycle end."""
    if abs(mvs - ref_mvs) <= 2:
        return True
    cg, co = len(hist) - 1, len(ref_hist) - 1
    if abs(cg - co) != 1:
        return False
    other = ref_hist[cg] if cg < co else hist[co]
    return other <= 10 * tol

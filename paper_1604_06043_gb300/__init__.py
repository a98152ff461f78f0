"""M(s)stab(l) / IDR(s)stab(l) for sequences of sparse linear systems on GB300.

The compute path is the C-ABI library ``libmsstab.so`` (hand-written CUDA for
sm_103a); :mod:`paper_1604_06043_gb300.msstab` is a thin ctypes binding to it.
:mod:`paper_1604_06043_gb300.problems` generates the seeded synthetic inputs.
"""

__all__ = ["problems"]

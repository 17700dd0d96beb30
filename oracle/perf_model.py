"""Oracle of the paper's performance model (section 4.1, Eq. 2-7) by brute force.

Test infrastructure only: imported by tests and never by the library.

For Neko the cost of a time step is linear in the number of elements on a
device (section 4.1), and the paper finds the modelled lowest run time T_min
"through a parameter search where we load balance the elements between the
different computing devices".  This module does exactly that search: every
split (E_1, ..., E_n) of E elements over n devices, each element costing c,
device i taking T_i = E_i c / P_i (its best performance P_i) and holding at
most Cmax_i; T_min is the smallest max_i T_i over the splits that fit.  It is
exponential in n and linear-to-quadratic in E: small cases only.
"""
from __future__ import annotations

import math


def _splits(E: int, n: int):
    if n == 1:
        yield (E,)
        return
    for a in range(E + 1):
        for rest in _splits(E - a, n - 1):
            yield (a,) + rest


def tmin_search(E: int, c: float, P, Cmax=None):
    """(T_min, best split in elements) by exhaustive search, or (inf, None)
    when no split fits the capacities."""
    n = len(P)
    cap = [math.inf if (Cmax is None or Cmax[i] is None or Cmax[i] <= 0) else Cmax[i] for i in range(n)]
    best, arg = math.inf, None
    for sp in _splits(E, n):
        if any(sp[i] * c > cap[i] for i in range(n)):
            continue
        T = max(sp[i] * c / P[i] for i in range(n))
        if T < best:
            best, arg = T, sp
    return best, arg

"""Window layout and kappa (oracle).

Test infrastructure (see the package header).

Sliding windows on S = Z^2 (Sec. 3.2): window (i, j) covers rows
[i*stride + o, i*stride + o + size) and columns [j*stride + o, ...).  kappa(R)
is the set of window indices whose region intersects R (Assumption 1, App. B);
Alg. 3 gives it per dimension as
    i_min = ceil((start - o - size + 1) / stride),
    i_max = floor((stop - 1 - o) / stride),
empty when i_min > i_max.  Floor and ceil are the mathematical ones (Python
integer division), which matters for negative coordinates.

Pins: brute force over every window of a box (tests/test_oracle_kappa.py).
"""
from __future__ import annotations


def _ceil_div(a: int, b: int) -> int:
    return -((-a) // b)


def kappa_1d(start: int, stop: int, size: int, stride: int, offset: int = 0):
    """Inclusive window-index range [i_min, i_max] for [start, stop), or None."""
    if stop <= start:
        return None
    i_min = _ceil_div(start - offset - size + 1, stride)
    i_max = (stop - 1 - offset) // stride
    if i_min > i_max:
        return None
    return i_min, i_max


def kappa(y0: int, x0: int, h: int, w: int, size: int, stride: int, offset: int = 0):
    """Sorted list of window indices (i, j) intersecting rows [y0, y0+h) and
    columns [x0, x0+w); i indexes rows, j columns."""
    ri = kappa_1d(y0, y0 + h, size, stride, offset)
    rj = kappa_1d(x0, x0 + w, size, stride, offset)
    if ri is None or rj is None:
        return []
    return [(i, j) for i in range(ri[0], ri[1] + 1) for j in range(rj[0], rj[1] + 1)]


def window_rect(i: int, j: int, size: int, stride: int, offset: int = 0):
    """(y0, x0, h, w) of window (i, j)."""
    return (i * stride + offset, j * stride + offset, size, size)


def cone_window_counts(y0: int, x0: int, h: int, w: int, size: int, stride: int,
                       steps: int, offset: int = 0):
    """Number of windows evaluated at each step (last step first) by a cold
    query of J_final over the region, following Alg. 1's recursion: the
    windows kappa(R) of the last step need J on the bounding box of their
    regions at the step before, and so on (Sec. 3.4 cone growth)."""
    counts = []
    ry0, rx0, rh, rw = y0, x0, h, w
    for _ in range(steps):
        ri = kappa_1d(ry0, ry0 + rh, size, stride, offset)
        rj = kappa_1d(rx0, rx0 + rw, size, stride, offset)
        if ri is None or rj is None:
            counts.append(0)
            break
        counts.append((ri[1] - ri[0] + 1) * (rj[1] - rj[0] + 1))
        ry0 = ri[0] * stride + offset
        rx0 = rj[0] * stride + offset
        rh = (ri[1] - ri[0]) * stride + size
        rw = (rj[1] - rj[0]) * stride + size
    return counts

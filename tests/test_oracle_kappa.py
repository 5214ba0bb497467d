"""Pins of kappa (Alg. 3) and of cone window counts (Lemma 4 / Thm 2)."""
import random

from oracle import kappa as K


def brute_kappa(y0, x0, h, w, size, stride, offset, span=60):
    out = []
    for i in range(-span, span):
        for j in range(-span, span):
            wy, wx = i * stride + offset, j * stride + offset
            if wy < y0 + h and y0 < wy + size and wx < x0 + w and x0 < wx + size:
                out.append((i, j))
    return out


def test_kappa_brute_force():
    rnd = random.Random(0)
    for _ in range(400):
        size = rnd.randint(1, 12)
        stride = rnd.randint(1, 12)
        offset = rnd.randint(-7, 7)
        y0, x0 = rnd.randint(-70, 60), rnd.randint(-70, 60)
        h, w = rnd.randint(1, 20), rnd.randint(1, 20)
        assert K.kappa(y0, x0, h, w, size, stride, offset) == brute_kappa(y0, x0, h, w, size, stride, offset, 200)


def test_kappa_gap_between_windows_is_empty():
    # stride larger than the window leaves pixels covered by no window
    assert K.kappa(5, 5, 1, 1, size=4, stride=10) == []
    assert K.kappa_1d(4, 10, 4, 10) is None
    assert K.kappa_1d(-3, -1, 4, 10) is None   # pixels -3,-2 lie in the gap [-6, 0)


def test_cone_counts_closed_form():
    # n x n tiles (tile = stride, window = 2 stride) aligned query: the last
    # step needs (n+1)^2 windows and each earlier step two more per side.
    for (n, s, K_) in [(4, 16, 4), (3, 8, 5), (1, 64, 20)]:
        counts = K.cone_window_counts(0, 0, n * s, n * s, 2 * s, s, K_)
        assert counts == [(n + 2 * k + 1) ** 2 for k in range(K_)]
    # the 64 x 64 query at the origin, 32/16 windows, 4 steps: 276 windows
    assert sum(K.cone_window_counts(0, 0, 64, 64, 32, 16, 4)) == 276


def test_cone_counts_bounded_independent_of_location():
    # Thm 2: cost of a window-sized query is bounded by M + M^2 + ... + M^T,
    # with M = |kappa(R_i)| = 9 for 50% overlap; and it is translation invariant
    rnd = random.Random(1)
    ref = None
    for _ in range(50):
        i, j = rnd.randint(-10 ** 6, 10 ** 6), rnd.randint(-10 ** 6, 10 ** 6)
        c = K.cone_window_counts(i * 16, j * 16, 32, 32, 32, 16, 4)
        ref = ref or c
        assert c == ref
        assert sum(c) <= 9 + 9 ** 2 + 9 ** 3 + 9 ** 4


def test_stride_overhead_matches_the_paper():
    # Over a large region the windows kappa selects cover every pixel
    # (H / s)^2 times: 4x at a 50% stride and 16/9 = 1.78x at 75%, the
    # overheads the paper prints (tests/golden/stride_overhead.txt).
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "stride_overhead.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert rows
    for size_s, stride_s, printed in rows:
        size, stride, printed = int(size_s), int(stride_s), float(printed)
        side = 1_000_000 * stride
        lo, hi = K.kappa_1d(0, side, size, stride)
        overhead = ((hi - lo + 1) * size / side) ** 2
        # edge windows add O(1e-6); the paper prints two decimals
        assert abs(overhead - printed) <= 0.005, (size, stride, overhead, printed)


def test_overlap_bound_and_recursive_cost_bound():
    # Assumption 2 / the recursive cost bound (Sec. "Constant-time cost"
    # appendix): a window region overlaps M windows, here exactly
    # (2 H/s - 1)^2 = 9 for H = 2s; a cold query of one window region costs
    # at most M + M^2 + ... + M^T window evaluations (c_t <= M (1 + c_{t+1}),
    # c_T = 0).  The lazy cone with its cache stays within that bound.
    size, stride = 32, 16
    rng = random.Random(3)
    for _ in range(20):
        i, j = rng.randint(-1000, 1000), rng.randint(-1000, 1000)
        assert len(K.kappa(*K.window_rect(i, j, size, stride), size, stride)) == 9
    M = 9
    for T in (1, 2, 4, 6):
        counts = K.cone_window_counts(*K.window_rect(5, -7, size, stride), size, stride, T)
        bound = sum(M ** k for k in range(1, T + 1))
        assert sum(counts) <= bound, (T, counts, bound)

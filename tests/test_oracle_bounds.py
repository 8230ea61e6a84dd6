"""The window searches' certificates, checked on the CPU against the
oracle's objective (definition mode): the bound a 1-D block of thresholds
or a 2-D cell of threshold pairs gets from the class sums at its ends (or
corners) must be at least the objective at every valid threshold inside it.

The bounds (as the GPU evaluates them): with N_1, Q_1 the count and the sum
of h^q of class 1 and N_2, Q_2 those of class 2, a = Q_1 / N_1^q and
b = Q_2 / N_2^q, phi = (1 - a b) / (q - 1). N_1, Q_1 never decrease and
N_2, Q_2 never increase as t (and s) grow, so over a block [t0, t1]
  q < 1: a b <= Q_1(t1) Q_2(t0) / (N_1(t0) N_2(t1))^q,
  q > 1: a b >= Q_1(t0) Q_2(t1) / (N_1(t1) N_2(t0))^q,
  q = 1: H_k = ln N_k - S_k / N_k (S = sum h ln h) with H_1 <= ln N_1(t1) -
         S_1(t0) / N_1(t1), H_2 <= ln N_2(t0) - S_2(t1) / N_2(t0),
and in 2-D the same with (t0, s0) and (t1, s1) as the corners of the cell.
A mistake in a corner, a direction or an exponent makes some block's bound
fall below its maximum on these histograms."""
import numpy as np
import pytest

import oracle

QS = [0.3, 0.8, 1.0, 1.5, 3.0]


def _terms(h, q):
    h = h.astype(np.float64)
    return h * np.log(np.where(h > 0, h, 1.0)) if q == 1.0 else np.where(h > 0, h ** q, 0.0)


def _bound(n1_lo, n1_hi, q1_lo, q1_hi, n2_lo, n2_hi, q2_lo, q2_hi, q):
    """Upper bound of phi from the extremes of the four class sums."""
    if n1_hi <= 0 or n2_hi <= 0:
        return -np.inf
    if q == 1.0:
        return (np.log(n1_hi) - q1_lo / n1_hi) + (np.log(n2_hi) - q2_lo / n2_hi)
    if q < 1.0:
        if n1_lo <= 0 or n2_lo <= 0:
            return np.inf
        ab = q1_hi * q2_hi / (n1_lo * n2_lo) ** q
    else:
        ab = q1_lo * q2_lo / (n1_hi * n2_hi) ** q
    return (1.0 - ab) / (q - 1.0)


def _hist1d(rng, L):
    h = rng.integers(0, 500, L)
    h[rng.random(L) < 0.3] = 0
    h[rng.integers(0, L)] += 5000
    return h.astype(np.int64)


@pytest.mark.parametrize("q", QS)
def test_1d_block_bounds_dominate_the_objective(q):
    rng = np.random.default_rng(int(q * 10))
    L, B = 48, 8
    for _ in range(20):
        h = _hist1d(rng, L)
        phi, valid = oracle.objective1d(h, q, mode="definition")
        w = _terms(h, q)
        N1, Q1 = np.cumsum(h), np.cumsum(w)
        N2, Q2 = h.sum() - N1, w.sum() - Q1      # class 2 of threshold t: levels t+1..L-1
        for t0 in range(0, L - 1, B):
            t1 = min(t0 + B - 1, L - 2)
            inside = valid[t0:t1 + 1]
            if not inside.any():
                continue
            ub = _bound(N1[t0], N1[t1], Q1[t0], Q1[t1], N2[t1], N2[t0], Q2[t1], Q2[t0], q)
            best = phi[t0:t1 + 1][inside].max()
            assert ub >= best - 1e-9 * max(abs(best), 1.0), (q, t0, ub, best)


@pytest.mark.parametrize("q", QS)
def test_2d_cell_bounds_dominate_the_objective(q):
    rng = np.random.default_rng(100 + int(q * 10))
    L, C = 14, 4
    for _ in range(12):
        h = rng.integers(0, 60, (L, L))
        h[rng.random((L, L)) < 0.4] = 0
        f = rng.integers(0, L, 400)
        np.add.at(h, (f, np.clip(f + rng.integers(-1, 2, 400), 0, L - 1)), 7)   # a diagonal ridge
        h = h.astype(np.int64)
        phi, valid = oracle.objective2d(h, q, mode="definition")
        w = _terms(h, q)
        NA = h.cumsum(0).cumsum(1)
        QA = w.cumsum(0).cumsum(1)
        NB = h[::-1, ::-1].cumsum(0).cumsum(1)[::-1, ::-1]   # sums over i >= t, j >= s
        QB = w[::-1, ::-1].cumsum(0).cumsum(1)[::-1, ::-1]
        for t0 in range(0, L - 1, C):
            for s0 in range(0, L - 1, C):
                t1, s1 = min(t0 + C - 1, L - 2), min(s0 + C - 1, L - 2)
                inside = valid[t0:t1 + 1, s0:s1 + 1]
                if not inside.any():
                    continue
                # quadrant B of (t, s) is i > t, j > s: the suffix sums at (t + 1, s + 1)
                ub = _bound(NA[t0, s0], NA[t1, s1], QA[t0, s0], QA[t1, s1],
                            NB[t1 + 1, s1 + 1], NB[t0 + 1, s0 + 1], QB[t1 + 1, s1 + 1], QB[t0 + 1, s0 + 1], q)
                best = phi[t0:t1 + 1, s0:s1 + 1][inside].max()
                assert ub >= best - 1e-9 * max(abs(best), 1.0), (q, t0, s0, ub, best)


def test_a_wrong_corner_is_caught():
    """Planting the classic mistake (class 2's sums taken at the same end as
    class 1's) makes some bound fall below the block maximum, so the checks
    above have teeth."""
    rng = np.random.default_rng(7)
    q, L, B = 0.8, 48, 8
    caught = False
    for _ in range(20):
        h = _hist1d(rng, L)
        phi, valid = oracle.objective1d(h, q, mode="definition")
        w = _terms(h, q)
        N1, Q1 = np.cumsum(h), np.cumsum(w)
        N2, Q2 = h.sum() - N1, w.sum() - Q1
        for t0 in range(0, L - 1, B):
            t1 = min(t0 + B - 1, L - 2)
            inside = valid[t0:t1 + 1]
            if not inside.any():
                continue
            wrong = _bound(N1[t0], N1[t1], Q1[t0], Q1[t1], N2[t0], N2[t1], Q2[t0], Q2[t1], q)
            if wrong < phi[t0:t1 + 1][inside].max() - 1e-9:
                caught = True
    assert caught

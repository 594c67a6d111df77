"""Pins of the regression oracle (oracle/regression.py): its operator
semantics against the operator netlists evaluated on plaintext bits, the
closed form against Eq. 2-3 in exact rational arithmetic, one gradient step
against the gradient of the loss of Eq. 14, gradient descent converging to
the line that generated the data, and the loss of Eq. 14 on known
residuals.  A last test plants plausible mistakes in the oracle and checks
that a pin fails on each."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import circuits as C
from oracle import regression as R


def _bits(v, k):
    return [(v >> i) & 1 for i in range(k)]


def _int(bits):
    k = len(bits)
    v = sum(int(b) << i for i, b in enumerate(bits))
    return v - (1 << k) if v >> (k - 1) else v


@pytest.mark.parametrize("k", [8, 16])
def test_operator_semantics_match_the_netlists(k):
    rng = np.random.default_rng(70 + k)
    lo, hi = -(1 << (k - 1)), (1 << (k - 1))
    pairs = [(int(a), int(b)) for a, b in rng.integers(lo, hi, size=(48, 2))]
    pairs += [(lo, 1), (hi - 1, -1), (lo, lo), (-7, 2), (7, -2), (-7, -2), (0, 5), (5, 1)]
    A = np.array([_bits(a & ((1 << k) - 1), k) for a, _ in pairs])
    B = np.array([_bits(b & ((1 << k) - 1), k) for _, b in pairs])
    add = C.eval_plain(C.build("add", k), A, B)
    sub = C.eval_plain(C.build("sub", k), A, B)
    mul = C.eval_plain(C.build("mul", k), A, B)
    div = C.eval_plain(C.build("div", k), A, B)
    for i, (a, b) in enumerate(pairs):
        assert _int(add[i]) == R.add(a, b, k)
        assert _int(sub[i]) == R.sub(a, b, k)
        assert _int(mul[i]) == a * b                     # the full 2k-bit product
        assert _int(mul[i][:k]) == R.mul(a, b, k)        # the application keeps its low k bits
        if b != 0 and not (a == lo and b == -1):
            assert _int(div[i][:k]) == R.div(a, b, k)   # the quotient half of the outputs


@pytest.mark.parametrize("slope,icpt", [(2, 1), (-3, 5), (1, -4), (0, 3)])
def test_closed_form_recovers_an_exact_line(slope, icpt):
    xs = [0, 1, 3, 4]                 # sum divisible by m: the mean is exact
    ys = [slope * x + icpt for x in xs]
    assert R.closed_form(xs, ys, 8) == (slope, icpt)


def _eq2(xs, ys):
    m = len(xs)
    xbar = Fraction(sum(xs), m)
    num = sum(Fraction(y) * (x - xbar) for x, y in zip(xs, ys))
    den = sum(Fraction(x * x) for x in xs) - Fraction(sum(xs) ** 2, m)
    return num, den


def test_closed_form_matches_eq2_when_the_mean_is_exact():
    """With sum x divisible by m and nothing wrapping, Num and Den are the
    exact numerator and denominator of Eq. 2, so omega = trunc(Num / Den) and
    b = trunc(sum (y - omega x) / m) (Eq. 3 with the integer slope)."""
    rng = np.random.default_rng(71)
    for _ in range(200):
        m = int(rng.integers(2, 9))
        xs = [int(v) for v in rng.integers(-6, 7, size=m)]
        xs[-1] += (-sum(xs)) % m      # make the sum divisible by m
        ys = [int(3 * x + v) for x, v in zip(xs, rng.integers(-3, 4, size=m))]
        num, den = _eq2(xs, ys)
        if den == 0 or max(abs(v) for v in xs + ys) > 40:
            continue
        k = 16
        omega, b = R.closed_form(xs, ys, k)
        q = num / den
        assert omega == int(q)        # int() truncates toward zero, like the divider
        r = Fraction(sum(y - omega * x for x, y in zip(xs, ys)), m)
        assert b == int(r)


def test_one_gradient_step_is_the_gradient_of_eq14():
    """From W = B = 0 one step moves W by -alpha (2/m) sum e_i x_i with
    e_i = -n y_i (n times the residual of the zero model), truncated."""
    xs, ys = [1, 2, 3, 4], [3, 5, 7, 9]
    n, a_num, a_den, m = 8, 1, 32, 4
    W, B = R.gradient_descent(xs, ys, 16, n, a_num, a_den, 1)
    gW = sum(-n * y * x for x, y in zip(xs, ys))
    gB = sum(-n * y for y in ys)
    assert W == -int(Fraction(2 * a_num * gW, a_den * m))
    assert B == -int(Fraction(2 * a_num * gB, a_den * m))


def test_gradient_descent_converges_to_the_generating_line():
    """Truncated steps stop once both updates round to zero; that fixed
    point fits every data point to within half a unit, and from there the
    iteration does not move."""
    xs = [1, 2, 3, 4]
    ys = [2 * x + 1 for x in xs]
    n, a_num, a_den = 100, 1, 16
    W, B = R.gradient_descent(xs, ys, 16, n, a_num, a_den, 200)
    assert max(abs(W * x + B - n * y) for x, y in zip(xs, ys)) < n // 2
    assert abs(W - 2 * n) <= n // 10
    assert R.gradient_descent(xs, ys, 16, n, a_num, a_den, 1, W, B) == (W, B)
    assert R.loss_gradient_descent(xs, ys, W, B, n, 16) == 0


def test_loss_of_eq14_on_known_residuals():
    xs, ys = [0, 1, 2, 3], [1, 4, 5, 6]      # residuals of y = 2x + 1: 0, 1, 0, -1
    assert R.loss_closed_form(xs, ys, 2, 1, 8) == (0 + 1 + 0 + 1) // 4
    assert R.loss_closed_form([0, 1], [1, 3], 2, 1, 8) == 0
    assert R.loss_closed_form(xs, [1, 6, 5, 10], 2, 1, 8) == (0 + 9 + 0 + 9) // 4


def test_wrap_and_division_edge_cases():
    assert R.wrap(128, 8) == -128 and R.wrap(-129, 8) == 127 and R.wrap(255, 8) == -1
    assert R.div(-7, 2, 8) == -3 and R.div(7, -2, 8) == -3 and R.div(-7, -2, 8) == 3
    with pytest.raises(ZeroDivisionError):
        R.div(3, 0, 8)
    with pytest.raises(OverflowError):
        R.div(-128, -1, 8)


def test_pins_catch_planted_mistakes(monkeypatch):
    """Floor instead of truncating division, a dropped factor 2 in the step,
    and the mean subtracted from y instead of x: each fails a pin above."""
    floor_div = lambda a, b, k: R.wrap(a // b, k)  # noqa: E731
    with monkeypatch.context() as mp:
        mp.setattr(R, "div", floor_div)
        with pytest.raises(AssertionError):
            test_operator_semantics_match_the_netlists(8)

    def gd_no_two(xs, ys, k, zoom, a_num, a_den, iters, w0=0, b0=0):
        m = len(xs)
        c1, c2 = a_num, a_den * m          # planted: 2 dropped
        ny = [R.mul(zoom, y, k) for y in ys]
        W, B = w0, b0
        for _ in range(iters):
            e = [R.sub(R.add(R.mul(W, x, k), B, k), t, k) for x, t in zip(xs, ny)]
            W = R.sub(W, R.div(R.mul(R.total([R.mul(v, x, k) for v, x in zip(e, xs)], k), c1, k), c2, k), k)
            B = R.sub(B, R.div(R.mul(R.total(e, k), c1, k), c2, k), k)
        return W, B

    with monkeypatch.context() as mp:
        mp.setattr(R, "gradient_descent", gd_no_two)
        with pytest.raises(AssertionError):
            test_one_gradient_step_is_the_gradient_of_eq14()

    def cf_wrong_center(xs, ys, k):
        m = len(xs)
        sx = R.total(xs, k)
        ybar = R.div(R.total(ys, k), m, k)   # planted: centre y instead of x
        num = R.total([R.mul(x, R.sub(y, ybar, k), k) for x, y in zip(xs, ys)], k)
        sxx = R.total([R.mul(x, x, k) for x in xs], k)
        den = R.sub(sxx, R.div(R.mul(sx, sx, k), m, k), k)
        omega = R.div(num, den, k)
        return omega, R.div(R.total([R.sub(y, R.mul(omega, x, k), k) for x, y in zip(xs, ys)], k), m, k)

    with monkeypatch.context() as mp:
        mp.setattr(R, "closed_form", cf_wrong_center)
        with pytest.raises(AssertionError):
            test_closed_form_matches_eq2_when_the_mean_is_exact()

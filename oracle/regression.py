"""Linear regression on k-bit two's-complement integers, step for step as the
encrypted application computes it (test infrastructure only: the oracle of
the regression application; it imports nothing from the product package).

Paper: Sec. 3.4 (unary linear regression: the closed form, Eq. 2-3; gradient
descent, Eq. 4-5), Sec. 4.6 (Algorithm 7: the closed form with the
homomorphic operators; Algorithm 8 with Eq. 12-14: gradient descent with the
learning rate and the parameters zoomed to integers), Sec. 5.5 (training and
evaluation, Table 8).

Every step is one of the k-bit operators of Sec. 4.3-4.5 with the semantics
of the operator netlists:
  add, sub  modulo 2^k;
  mul       the 2k-bit product, of which the application keeps the low k bits
            (every quantity stays at the operands' width);
  div       quotient truncated toward zero; a zero divisor, and -2^(k-1)
            divided by -1, are errors here (the divider's bits are
            unspecified there).
Public constants (m, n, 2 a_num, a_den m) enter as k-bit operands like
every other value, i.e. modulo 2^k.

Readings (the paper names the equations but not the operator sequence, and
prints Eq. 12 and Eq. 13 garbled -- the same right-hand side for b' and
omega', with the zoom applied inconsistently):

  closed form (Eq. 2, Eq. 3, Algorithm 7 steps 3-5), m data points:
    Sx = sum x_i;  xbar = Sx / m;  Num = sum y_i * (x_i - xbar);
    Den = sum x_i * x_i - (Sx * Sx) / m;  omega = Num / Den;
    b = (sum (y_i - omega * x_i)) / m
  gradient descent (Algorithm 8; the gradient of the loss of Eq. 14 with the
  parameters zoomed by n, W = n omega and B = n b, and a learning rate
  alpha = a_num / a_den):
    ny_i = n * y_i  (once);  W = B = 0  (Algorithm 8 step 3)
    per iteration:  e_i = W * x_i + B - ny_i          (n times the residual)
                    gW = sum e_i * x_i;  gB = sum e_i
                    W = W - (gW * c1) / c2;  B = B - (gB * c1) / c2
    with the public constants c1 = 2 a_num and c2 = a_den m (the factor 2/m
    of the gradient of Eq. 14 and the learning rate).
  evaluation (Eq. 14, the loss of the trained model):
    closed form:  r_i = y_i - (omega * x_i + b);  loss = (sum r_i * r_i) / m
    gradient descent:  r_i = y_i - (W * x_i + B) / n;  loss = (sum r_i * r_i) / m
"""


def wrap(v, k):
    """v modulo 2^k as a signed k-bit integer."""
    v &= (1 << k) - 1
    return v - (1 << k) if v >> (k - 1) else v


def add(a, b, k):
    return wrap(a + b, k)


def sub(a, b, k):
    return wrap(a - b, k)


def mul(a, b, k):
    return wrap(a * b, k)


def div(a, b, k):
    if b == 0:
        raise ZeroDivisionError("zero divisor: the divider's output is unspecified")
    if a == -(1 << (k - 1)) and b == -1:
        raise OverflowError("-2^(k-1) / -1 does not fit in k bits")
    q = abs(a) // abs(b)
    return wrap(-q if (a < 0) != (b < 0) else q, k)


def total(vals, k):
    s = 0
    for v in vals:
        s = add(s, v, k)
    return s


def closed_form(xs, ys, k):
    """(omega, b) of Eq. 2-3 in k-bit operators (Algorithm 7)."""
    m = len(xs)
    assert m == len(ys) and m >= 1
    xs = [wrap(x, k) for x in xs]
    ys = [wrap(y, k) for y in ys]
    mk = wrap(m, k)
    sx = total(xs, k)
    xbar = div(sx, mk, k)
    num = total([mul(y, sub(x, xbar, k), k) for x, y in zip(xs, ys)], k)
    sxx = total([mul(x, x, k) for x in xs], k)
    den = sub(sxx, div(mul(sx, sx, k), mk, k), k)
    omega = div(num, den, k)
    b = div(total([sub(y, mul(omega, x, k), k) for x, y in zip(xs, ys)], k), mk, k)
    return omega, b


def gradient_descent(xs, ys, k, zoom, a_num, a_den, iters, w0=0, b0=0):
    """(W, B) = (zoom * omega, zoom * b) after `iters` iterations (Algorithm 8)."""
    m = len(xs)
    assert m == len(ys) and m >= 1 and iters >= 0
    xs = [wrap(x, k) for x in xs]
    ys = [wrap(y, k) for y in ys]
    c1, c2 = wrap(2 * a_num, k), wrap(a_den * m, k)
    ny = [mul(zoom, y, k) for y in ys]
    W, B = wrap(w0, k), wrap(b0, k)
    for _ in range(iters):
        e = [sub(add(mul(W, x, k), B, k), t, k) for x, t in zip(xs, ny)]
        gW = total([mul(ei, x, k) for ei, x in zip(e, xs)], k)
        gB = total(e, k)
        W = sub(W, div(mul(gW, c1, k), c2, k), k)
        B = sub(B, div(mul(gB, c1, k), c2, k), k)
    return W, B


def loss_closed_form(xs, ys, omega, b, k):
    """Eq. 14 for the closed-form model: (sum (y_i - (omega x_i + b))^2) / m."""
    r = [sub(wrap(y, k), add(mul(omega, wrap(x, k), k), b, k), k) for x, y in zip(xs, ys)]
    return div(total([mul(v, v, k) for v in r], k), wrap(len(xs), k), k)


def loss_gradient_descent(xs, ys, W, B, zoom, k):
    """Eq. 14 for the zoomed model: (sum (y_i - (W x_i + B) / n)^2) / m."""
    r = [sub(wrap(y, k), div(add(mul(W, wrap(x, k), k), B, k), wrap(zoom, k), k), k) for x, y in zip(xs, ys)]
    return div(total([mul(v, v, k) for v in r], k), wrap(len(xs), k), k)

"""Encrypted linear regression (Sec. 4.6, Algorithms 7 and 8; training and
evaluation as measured in Sec. 5.5, Table 8) on multi-key ciphertexts.

Composed of the library's k-bit operators only (mk_add_kbit, mk_sub_kbit,
mk_mul_kbit, mk_div_kbit): every gate of every step runs in the library's
kernels.  This module sequences the operator calls, slices, replicates and
stacks ciphertext rows in device memory, and encodes public constants with
mk_trivial.  An integer is a [count][kbits][W] int32 tensor of bit
ciphertexts, least significant bit first (W = k*n + 1), on the context's
device; tensor copies run on torch's current stream, which must be the
context's stream (the Context default).

Step semantics (those of the operator netlists): + and - modulo 2^kbits,
* keeps the low kbits of the 2*kbits-bit product, / truncates toward zero.
The paper gives the equations, not the operator sequence, and prints Eq. 12
and Eq. 13 garbled; the sequences below are the readings:

  closed form (Eq. 2-3; Algorithm 7 steps 3-5), m data points:
    Sx = sum x_i;  xbar = Sx / m;  Num = sum y_i * (x_i - xbar);
    Den = sum x_i * x_i - (Sx * Sx) / m;  omega = Num / Den;
    b = (sum (y_i - omega * x_i)) / m
  gradient descent (Algorithm 8: the gradient of the loss of Eq. 14 with
  the parameters zoomed by n, W = n omega, B = n b, learning rate
  a_num / a_den, public c1 = 2 a_num, c2 = a_den m):
    ny_i = n * y_i;  W = w0, B = b0;  per iteration
    e_i = W * x_i + B - ny_i;  gW = sum e_i * x_i;  gB = sum e_i;
    W = W - (gW * c1) / c2;  B = B - (gB * c1) / c2
  evaluation (the loss of Eq. 14 for the trained model):
    closed form        r_i = y_i - (omega * x_i + b)
    gradient descent   r_i = y_i - (W * x_i + B) / n
    loss = (sum r_i * r_i) / m

Independent operator instances of one step share a call (more operand
pairs, the same number of netlist levels): the operators are evaluated
level by level over all their pairs, so a call costs its netlist depth in
launches whatever its width.  For the same reason the calls here, with one
to a few pairs, suit the context's shallow netlist family
(ctx.set_circuit_style("shallow")); the results do not depend on it.
"""
import numpy as np
import torch

from .workloads import bits_to_int, int_to_bits


def encrypt_integers(ctx, values, kbits, party, seed, device="cuda"):
    """SymEnc by `party` of each integer's bits: [len(values)][kbits][W]."""
    ct = ctx.encrypt(party, int_to_bits(values, kbits).reshape(-1), seed)
    return torch.from_numpy(ct.view(np.int32)).reshape(len(values), kbits, ctx.W).to(device)


def decrypt_integers(ctx, ct):
    """SymDec (every party's secret) of [count][kbits][W] to signed integers."""
    count, kbits = ct.shape[0], ct.shape[1]
    return bits_to_int(ctx.decrypt(ct.reshape(count * kbits, -1).contiguous()).reshape(count, kbits))


class Operators:
    """The k-bit operators of one context at one width on [P][kbits][W]
    tensors (fresh contiguous outputs), with the application's semantics."""

    def __init__(self, ctx, kbits, device):
        self.ctx, self.k, self.device = ctx, kbits, device
        self.calls = {"add": 0, "sub": 0, "mul": 0, "div": 0}

    def _new(self, pairs, rows):
        return torch.empty((pairs, rows, self.ctx.W), dtype=torch.int32, device=self.device)

    def _prep(self, a, b):
        """Contiguous, 16-byte aligned operands (the ABI's pointer rule: a
        row slice of a [count][kbits][W] tensor starts at a multiple of
        4 kbits W bytes, which need not be one)."""
        if a.shape != b.shape or a.shape[1] != self.k or a.dtype != torch.int32:
            raise ValueError("operands must be int32 [pairs][kbits][W] of one shape")
        return tuple(t.clone() if t.data_ptr() % 16 else t for t in (a.contiguous(), b.contiguous()))

    def add(self, a, b):
        a, b = self._prep(a, b)
        out = self._new(a.shape[0], self.k)
        self.ctx.add_kbit(self.k, a, b, out)
        self.calls["add"] += 1
        return out

    def sub(self, a, b):
        a, b = self._prep(a, b)
        out = self._new(a.shape[0], self.k)
        self.ctx.sub_kbit(self.k, a, b, out)
        self.calls["sub"] += 1
        return out

    def mul(self, a, b):
        """The low kbits of the product."""
        a, b = self._prep(a, b)
        out = self._new(a.shape[0], 2 * self.k)
        self.ctx.mul_kbit(self.k, a, b, out)
        self.calls["mul"] += 1
        return out[:, :self.k].contiguous()

    def div(self, a, b):
        """The truncating quotient."""
        a, b = self._prep(a, b)
        q = self._new(a.shape[0], self.k)
        r = self._new(a.shape[0], self.k)
        self.ctx.div_kbit(self.k, a, b, q, r)
        self.calls["div"] += 1
        return q

    def sums(self, v):
        """Sums along axis 1 of [G][m][kbits][W]: [G][kbits][W], by a pairwise
        tree whose levels add all G groups in one call."""
        G, m = v.shape[0], v.shape[1]
        while m > 1:
            h = m // 2
            s = self.add(v[:, :h].reshape(G * h, self.k, -1), v[:, h:2 * h].reshape(G * h, self.k, -1))
            s = s.reshape(G, h, self.k, -1)
            v = torch.cat([s, v[:, 2 * h:]], dim=1) if m % 2 else s
            m = v.shape[1]
        return v[:, 0].contiguous()

    def public(self, value, count):
        """count copies of a public integer as noiseless ciphertexts."""
        rows = self.ctx.trivial(np.tile(int_to_bits([value], self.k)[0], count))
        return torch.from_numpy(rows.view(np.int32)).reshape(count, self.k, -1).to(self.device)


def _check_data(cx, cy, kbits):
    if cx.dim() != 3 or cx.shape != cy.shape or cx.shape[1] != kbits or cx.shape[0] < 1:
        raise ValueError("cx, cy: [m][kbits][W] with m >= 1")
    return cx.shape[0]


def _rep(a, count):
    """[1][kbits][W] -> [count][kbits][W] (a copy)."""
    return a.expand(count, -1, -1).contiguous()


def closed_form(ctx, kbits, cx, cy):
    """Algorithm 7: encrypted (omega, b) [1][kbits][W] each, from cx, cy
    [m][kbits][W].  Returns (omega, b, operator calls)."""
    ops = Operators(ctx, kbits, cx.device)
    m = _check_data(cx, cy, kbits)
    xx = ops.mul(cx, cx)                                        # x_i * x_i
    sx, sxx = ops.sums(torch.stack([cx, xx])).split(1)          # Sx, sum x_i^2
    sx2 = ops.mul(sx, sx)                                       # Sx * Sx
    xbar, t = ops.div(torch.cat([sx, sx2]), ops.public(m, 2)).split(1)
    diff = ops.sub(torch.cat([cx, sxx]), torch.cat([_rep(xbar, m), t]))
    d, den = diff[:m], diff[m:]                                 # x_i - xbar;  Den
    num = ops.sums(ops.mul(cy, d)[None])                        # Num
    omega = ops.div(num, den)
    r = ops.sub(cy, ops.mul(_rep(omega, m), cx))                # y_i - omega * x_i
    b = ops.div(ops.sums(r[None]), ops.public(m, 1))
    return omega, b, ops.calls


def gradient_descent(ctx, kbits, cx, cy, zoom, a_num, a_den, iters, w0=0, b0=0):
    """Algorithm 8: encrypted zoomed parameters (W, B) [1][kbits][W] each
    after `iters` iterations.  Returns (W, B, operator calls)."""
    ops = Operators(ctx, kbits, cx.device)
    m = _check_data(cx, cy, kbits)
    ny = ops.mul(ops.public(zoom, m), cy)                       # n * y_i
    c1, c2 = ops.public(2 * a_num, 2), ops.public(a_den * m, 2)
    wb = torch.cat([ops.public(w0, 1), ops.public(b0, 1)])      # [W; B]
    for _ in range(iters):
        e = ops.sub(ops.add(ops.mul(_rep(wb[:1], m), cx), _rep(wb[1:], m)), ny)
        g = ops.sums(torch.stack([ops.mul(e, cx), e]))           # [gW; gB]
        wb = ops.sub(wb, ops.div(ops.mul(g, c1), c2))
    return wb[:1].contiguous(), wb[1:].contiguous(), ops.calls


def loss_closed_form(ctx, kbits, cx, cy, omega, b):
    """Eq. 14 for the closed-form model: (sum (y_i - (omega x_i + b))^2) / m."""
    ops = Operators(ctx, kbits, cx.device)
    m = _check_data(cx, cy, kbits)
    r = ops.sub(cy, ops.add(ops.mul(_rep(omega, m), cx), _rep(b, m)))
    return ops.div(ops.sums(ops.mul(r, r)[None]), ops.public(m, 1)), ops.calls


def loss_gradient_descent(ctx, kbits, cx, cy, W, B, zoom):
    """Eq. 14 for the zoomed model: (sum (y_i - (W x_i + B) / n)^2) / m."""
    ops = Operators(ctx, kbits, cx.device)
    m = _check_data(cx, cy, kbits)
    pred = ops.div(ops.add(ops.mul(_rep(W, m), cx), _rep(B, m)), ops.public(zoom, m))
    r = ops.sub(cy, pred)
    return ops.div(ops.sums(ops.mul(r, r)[None]), ops.public(m, 1)), ops.calls

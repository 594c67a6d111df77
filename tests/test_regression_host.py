"""The encrypted regression's orchestration (paper_2205_05825_gb300/
regression.py) on the CPU: the module runs unchanged against a stand-in
context whose "ciphertexts" are noiseless rows (zero mask, b = m/4) and whose
operators evaluate the operator netlists on the decoded plaintext bits.
This checks the call sequence, the row layouts, slicing, stacking,
replication and public constants against the regression oracle; the
encrypted arithmetic itself is checked on the GPU
(tests/test_gpu_regression.py)."""
import numpy as np
import pytest
import torch

from oracle import circuits as C
from oracle import regression as R

W_TEST = 5  # stand-in ciphertext width (mask of 4 words + b)


class PlainContext:
    def __init__(self, style="array"):
        self.W = W_TEST
        self.style = style
        self.nets = {}

    def _net(self, op, k):
        if (op, k) not in self.nets:
            self.nets[(op, k)] = C.build(op, k, self.style)
        return self.nets[(op, k)]

    def trivial(self, bits):
        out = np.zeros((len(bits), self.W), np.uint32)
        out[:, -1] = (np.asarray(bits, np.uint32) & 1) << 30
        return out

    def encrypt(self, party, bits, seed):
        return self.trivial(bits)

    def decrypt(self, ct):
        ct = ct.numpy() if isinstance(ct, torch.Tensor) else ct
        return ((ct[:, -1].astype(np.uint32) >> 30) & 1).astype(np.uint8)

    @staticmethod
    def _bits(t, kbits, pairs):
        assert t.dtype == torch.int32 and t.is_contiguous() and t.numel() == pairs * kbits * W_TEST
        assert t.data_ptr() % 16 == 0, "the ABI wants 16-byte aligned operands"
        v = t.reshape(pairs, kbits, W_TEST).numpy().view(np.uint32)
        assert not v[..., :-1].any(), "stand-in ciphertexts have zero masks"
        return ((v[..., -1] >> 30) & 1).astype(np.int64)

    def _run(self, op, kbits, a, b, outs):
        pairs = a.numel() // (kbits * self.W)
        res = C.eval_plain(self._net(op, kbits), self._bits(a, kbits, pairs), self._bits(b, kbits, pairs))
        col = 0
        for o in outs:
            rows = o.numel() // (pairs * self.W)
            assert o.is_contiguous() and o.shape[0] == pairs
            o.zero_()
            o.reshape(pairs, rows, self.W)[..., -1] = torch.from_numpy((res[:, col:col + rows] << 30).astype(np.int32))
            col += rows
        assert col == res.shape[1]

    def add_kbit(self, k, a, b, out):
        self._run("add", k, a, b, [out])

    def sub_kbit(self, k, a, b, out):
        self._run("sub", k, a, b, [out])

    def mul_kbit(self, k, a, b, out):
        self._run("mul", k, a, b, [out])

    def div_kbit(self, k, a, b, q, r):
        self._run("div", k, a, b, [q, r])


def _enc(ctx, vals, k):
    from paper_2205_05825_gb300 import regression as G
    return G.encrypt_integers(ctx, vals, k, 0, 1, device="cpu")


@pytest.mark.parametrize("m", [1, 2, 3, 4, 7])
def test_closed_form_orchestration_matches_the_oracle(m):
    from paper_2205_05825_gb300 import regression as G
    rng = np.random.default_rng(80 + m)
    ctx = PlainContext()
    checked = 0
    for _ in range(6):
        xs = [int(v) for v in rng.integers(-4, 5, size=m)]
        ys = [int(2 * x + v) for x, v in zip(xs, rng.integers(-2, 3, size=m))]
        try:
            ref = R.closed_form(xs, ys, 8)
        except (ZeroDivisionError, OverflowError):
            assert len(set(xs)) == 1     # all x equal (always at m = 1): Den = 0, no slope
            continue
        checked += 1
        omega, b, calls = G.closed_form(ctx, 8, _enc(ctx, xs, 8), _enc(ctx, ys, 8))
        got = (int(G.decrypt_integers(ctx, omega)[0]), int(G.decrypt_integers(ctx, b)[0]))
        assert got == ref
        assert calls["div"] == 3 and calls["mul"] == 4 and calls["sub"] == 2
        loss, _ = G.loss_closed_form(ctx, 8, _enc(ctx, xs, 8), _enc(ctx, ys, 8), omega, b)
        assert int(G.decrypt_integers(ctx, loss)[0]) == R.loss_closed_form(xs, ys, ref[0], ref[1], 8)
    assert checked >= (0 if m == 1 else 3)


@pytest.mark.parametrize("m,iters", [(1, 2), (4, 3), (5, 2)])
def test_gradient_descent_orchestration_matches_the_oracle(m, iters):
    from paper_2205_05825_gb300 import regression as G
    rng = np.random.default_rng(90 + m)
    ctx = PlainContext()
    xs = [int(v) for v in rng.integers(-3, 5, size=m)]
    ys = [int(2 * x + 1 + v) for x, v in zip(xs, rng.integers(-1, 2, size=m))]
    k, n, a_num, a_den = 16, 50, 1, 16
    Wc, Bc, calls = G.gradient_descent(ctx, k, _enc(ctx, xs, k), _enc(ctx, ys, k), n, a_num, a_den, iters)
    W, B = R.gradient_descent(xs, ys, k, n, a_num, a_den, iters)
    assert (int(G.decrypt_integers(ctx, Wc)[0]), int(G.decrypt_integers(ctx, Bc)[0])) == (W, B)
    assert calls["div"] == iters and calls["mul"] == 1 + 3 * iters
    loss, _ = G.loss_gradient_descent(ctx, k, _enc(ctx, xs, k), _enc(ctx, ys, k), Wc, Bc, n)
    assert int(G.decrypt_integers(ctx, loss)[0]) == R.loss_gradient_descent(xs, ys, W, B, n, k)


def test_gradient_descent_from_given_start_and_wrapping_constants():
    """A start point other than zero, and a zoom and data count that wrap
    at 8 bits (public constants are k-bit operands)."""
    from paper_2205_05825_gb300 import regression as G
    ctx = PlainContext()
    xs, ys = [1, -2, 3], [3, -3, 7]
    k = 8
    Wc, Bc, _ = G.gradient_descent(ctx, k, _enc(ctx, xs, k), _enc(ctx, ys, k), 300, 1, 100, 2, w0=5, b0=-3)
    assert (int(G.decrypt_integers(ctx, Wc)[0]), int(G.decrypt_integers(ctx, Bc)[0])) == \
        R.gradient_descent(xs, ys, k, 300, 1, 100, 2, w0=5, b0=-3)


def test_odd_width_operands_stay_aligned():
    """At 3 bits a row slice starts at a multiple of 4 * 3 * W bytes, not of
    16: the module copies such operands before a call."""
    from paper_2205_05825_gb300 import regression as G
    ctx = PlainContext()
    xs, ys = [0, 1, 2], [1, 2, 3]     # the data count is an operand too: m <= 3 at 3 bits
    k = 3
    got = G.closed_form(ctx, k, _enc(ctx, xs, k), _enc(ctx, ys, k))
    ref = R.closed_form(xs, ys, k)
    assert (int(G.decrypt_integers(ctx, got[0])[0]), int(G.decrypt_integers(ctx, got[1])[0])) == ref


def test_integer_bit_codecs():
    from paper_2205_05825_gb300 import workloads as W
    vals = [0, 1, -1, 127, -128, 5, -77]
    bits = W.int_to_bits(vals, 8)
    assert bits.shape == (7, 8) and list(W.bits_to_int(bits)) == vals
    assert list(W.bits_to_int(W.int_to_bits([128, -129], 8))) == [-128, 127]


def test_bad_shapes_are_refused():
    from paper_2205_05825_gb300 import regression as G
    ctx = PlainContext()
    x = _enc(ctx, [1, 2], 8)
    with pytest.raises(ValueError):
        G.closed_form(ctx, 8, x, _enc(ctx, [1, 2, 3], 8))
    with pytest.raises(ValueError):
        G.gradient_descent(ctx, 16, x, x, 10, 1, 10, 1)


def test_both_netlist_families_give_the_same_models():
    """The application on the shallow netlists equals the oracle as on the
    array ones (the families compute the same functions)."""
    from paper_2205_05825_gb300 import regression as G
    from paper_2205_05825_gb300 import workloads as W
    xs, ys = W.unary_regression_data(6, 2, 1, -3, 4, 1, config_id=61)
    for style in ("array", "shallow"):
        ctx = PlainContext(style)
        om, b, _ = G.closed_form(ctx, 8, _enc(ctx, xs, 8), _enc(ctx, ys, 8))
        assert (int(G.decrypt_integers(ctx, om)[0]), int(G.decrypt_integers(ctx, b)[0])) == R.closed_form(xs, ys, 8)
        Wc, Bc, _ = G.gradient_descent(ctx, 16, _enc(ctx, xs, 16), _enc(ctx, ys, 16), 100, 1, 16, 2)
        assert (int(G.decrypt_integers(ctx, Wc)[0]), int(G.decrypt_integers(ctx, Bc)[0])) == \
            R.gradient_descent(xs, ys, 16, 100, 1, 16, 2)

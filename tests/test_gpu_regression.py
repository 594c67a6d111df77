"""The encrypted linear regression (Algorithms 7 and 8) on the GPU at the toy
parameter set, two parties: x encrypted by party 0, y by party 1 (each
participant contributes its own data, Sec. 5.5).  The decrypted model and
loss equal the regression oracle's integer emulation exactly: every operator
is an exact circuit, so any gate that decrypted wrongly would show."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx2(gpu_ready):
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    for i, s in enumerate(W.party_seeds(2)):
        ctx.keygen(i, s)
    yield ctx
    ctx.close()


def _enc(ctx, xs, ys, k, cfg):
    from paper_2205_05825_gb300 import regression as G
    from paper_2205_05825_gb300 import workloads as W
    return (G.encrypt_integers(ctx, xs, k, 0, W.encryption_seed(cfg, 0)),
            G.encrypt_integers(ctx, ys, k, 1, W.encryption_seed(cfg, 1)))


def _dec(ctx, ct):
    from paper_2205_05825_gb300 import regression as G
    return int(G.decrypt_integers(ctx, ct)[0])


@pytest.mark.parametrize("style", ["array", "shallow"])
@pytest.mark.parametrize("case", ["exact line", "noisy"])
def test_closed_form_8bit_equals_the_oracle(ctx2, case, style):
    from oracle import regression as R
    from paper_2205_05825_gb300 import regression as G
    from paper_2205_05825_gb300 import workloads as W
    if case == "exact line":
        xs, ys = [0, 1, 3, 4], [1, 3, 7, 9]           # y = 2x + 1, mean of x exact
    else:
        xs, ys = W.unary_regression_data(6, 2, 1, -3, 4, 1, config_id=61)
    k = 8
    cx, cy = _enc(ctx2, xs, ys, k, 60)
    ctx2.set_circuit_style(style)
    try:
        omega, b, calls = G.closed_form(ctx2, k, cx, cy)
        ref = R.closed_form(xs, ys, k)
        assert (_dec(ctx2, omega), _dec(ctx2, b)) == ref
        if case == "exact line":
            assert ref == (2, 1)
        loss, _ = G.loss_closed_form(ctx2, k, cx, cy, omega, b)
        ctx2.sync()
    finally:
        ctx2.set_circuit_style("array")
    assert _dec(ctx2, loss) == R.loss_closed_form(xs, ys, ref[0], ref[1], k)


@pytest.mark.parametrize("style", ["array", "shallow"])
def test_gradient_descent_16bit_equals_the_oracle(ctx2, style):
    from oracle import regression as R
    from paper_2205_05825_gb300 import regression as G
    from paper_2205_05825_gb300 import workloads as W
    xs, ys = W.unary_regression_data(4, 2, 1, 1, 4, 0, config_id=62)
    k, n, a_num, a_den, iters = 16, 100, 1, 16, 2
    cx, cy = _enc(ctx2, xs, ys, k, 63)
    ctx2.set_circuit_style(style)
    try:
        Wc, Bc, calls = G.gradient_descent(ctx2, k, cx, cy, n, a_num, a_den, iters)
        W_, B_ = R.gradient_descent(xs, ys, k, n, a_num, a_den, iters)
        assert (_dec(ctx2, Wc), _dec(ctx2, Bc)) == (W_, B_)
        assert calls["div"] == iters
        loss, _ = G.loss_gradient_descent(ctx2, k, cx, cy, Wc, Bc, n)
        ctx2.sync()
    finally:
        ctx2.set_circuit_style("array")
    assert _dec(ctx2, loss) == R.loss_gradient_descent(xs, ys, W_, B_, n, k)

"""Parameter sets, seeds and seeded synthetic inputs.

This module holds no arithmetic of the method: it only names the workloads
(parameter sets after Table 7 of the paper, party counts, batch sizes) and draws
the plaintext inputs (bits, gate types, integer operands) from fixed seeds.
Both the test suite and the benchmark take their inputs from here, for the
GPU library and for the CPU oracle alike.

The paper publishes no dataset: every input is synthetic.
"""
import numpy as np

# Seeds.  The CRS seed and per-party key seeds are the ones every workload uses.
CRS_SEED = 0x22050582
PARTY_SEED_BASE = 0x5825_0000
INPUT_SEED_BASE = 0xB175_0000

GATE_NAMES = ("AND", "OR", "NAND", "NOR", "XOR", "XNOR")


def party_seeds(k):
    return [PARTY_SEED_BASE + p for p in range(k)]


def _p(n, N, k, sigma_lwe, sigma_rlwe, bg_bit=8, d=3, ks_bit=2, t=8):
    return dict(n=n, N=N, k=k, bg_bit=bg_bit, d=d, ks_bit=ks_bit, t=t,
                sigma_lwe=float(sigma_lwe), sigma_rlwe=float(sigma_rlwe))


def toy_params(k=2):
    """Toy set: LWE n = 64, ring N = 256, base 2^8, d = 3, key-switch base 2^2,
    t = 8, Gaussian noise sigma = 2^-25 for both LWE and RLWE samples."""
    return _p(64, 256, k, 2.0 ** -25, 2.0 ** -25)


# RLWE noise per party count for the full-size set.  At the stated 2^-25 the
# bootstrap's output noise exceeds the 1/8 decision margin (see the design
# notes); each party count takes the largest sigma from the ladder
# {2^-25, 2^-28, 2^-30, 2^-32} whose predicted XOR-of-outputs margin is at
# least 6 standard deviations.
FULL_SIGMA_RLWE = {1: 2.0 ** -28, 2: 2.0 ** -30, 3: 2.0 ** -30, 4: 2.0 ** -32, 8: 2.0 ** -32}


def full_params(k=2):
    """Full-size set: n = 560, N = 1024, base 2^8, d = 3, key-switch base 2^2,
    t = 8, LWE sigma = 2^-15, RLWE sigma per party count (FULL_SIGMA_RLWE)."""
    return _p(560, 1024, k, 2.0 ** -15, FULL_SIGMA_RLWE.get(k, 2.0 ** -32))


def paper_params(k=2):
    """Table 7 verbatim: n = 560, alpha = 3.05e-5, B' = 2^2, d' = 8, N = 1024,
    beta = 3.72e-9, B = 2^9, d = 3."""
    return _p(560, 1024, k, 3.05e-5, 3.72e-9, bg_bit=9)


def tiny_params(k=2, sigma=0.0):
    """Smallest set used by the oracle's unit pins (fast on one core)."""
    return _p(16, 64, k, sigma, sigma)


# ----------------------------------------------------------------------------- inputs
def rng(config_id):
    return np.random.default_rng(INPUT_SEED_BASE + config_id)


def truth_table_inputs():
    """The 6 gates x 4 input pairs of the toy configuration (c1 by party 0,
    c2 by party 1), in a fixed order: returns (gate_ids, bits1, bits2)."""
    g, b1, b2 = [], [], []
    for gi in range(6):
        for m1 in (0, 1):
            for m2 in (0, 1):
                g.append(gi)
                b1.append(m1)
                b2.append(m2)
    return (np.array(g, np.int32), np.array(b1, np.uint8), np.array(b2, np.uint8))


def random_gates(count, config_id=2):
    """Uniform gate types and uniform input bits: returns (types, bits1, bits2)."""
    r = rng(config_id)
    types = r.integers(0, 6, size=count).astype(np.int32)
    b1 = r.integers(0, 2, size=count).astype(np.uint8)
    b2 = r.integers(0, 2, size=count).astype(np.uint8)
    return types, b1, b2


def random_operands(kbits, count, config_id=3):
    """Uniform signed kbits-bit integers (two's complement range)."""
    r = rng(config_id * 1000 + kbits)
    lo, hi = -(1 << (kbits - 1)), (1 << (kbits - 1))
    return (r.integers(lo, hi, size=count).astype(np.int64),
            r.integers(lo, hi, size=count).astype(np.int64))


def int_to_bits(vals, kbits):
    """LSB-first two's-complement bit planes: [count][kbits] uint8."""
    vals = np.asarray(vals, np.int64)
    return ((vals[:, None] >> np.arange(kbits)) & 1).astype(np.uint8)


def bits_to_int(bits):
    """Inverse of int_to_bits (signed)."""
    bits = np.asarray(bits, np.int64)
    kbits = bits.shape[-1]
    v = (bits << np.arange(kbits)).sum(axis=-1)
    return np.where(v >= (1 << (kbits - 1)), v - (1 << kbits), v)


def encryption_seed(config_id, party, stream=0):
    return INPUT_SEED_BASE + (config_id << 12) + (party << 4) + stream


# ----------------------------------------------------------------------------- serving (regression requests)
def wrap_int(v, bits=16):
    """Two's-complement wrap of Python/numpy integers to `bits` bits."""
    v = np.asarray(v, np.int64) % (1 << bits)
    return np.where(v >= 1 << (bits - 1), v - (1 << bits), v)


def regression_data(samples=64, features=4, config_id=5):
    """Synthetic linear-regression data (the paper's is unpublished): integer
    features uniform in [-16, 16], integer weights, y = w.x + noise in [-2, 2]."""
    r = rng(config_id)
    X = r.integers(-16, 17, size=(samples, features)).astype(np.int64)
    w = r.integers(-4, 5, size=features).astype(np.int64)
    y = X @ w + r.integers(-2, 3, size=samples)
    return X, w, y


def unary_regression_data(m, slope, intercept, x_lo, x_hi, noise, config_id=6):
    """m points of the unary model (Sec. 3.4): x uniform in [x_lo, x_hi],
    y = slope x + intercept + noise uniform in [-noise, noise] (the paper's
    data, linear with random noise, is unpublished)."""
    r = rng(config_id)
    x = r.integers(x_lo, x_hi + 1, size=m).astype(np.int64)
    y = slope * x + intercept + r.integers(-noise, noise + 1, size=m)
    return [int(v) for v in x], [int(v) for v in y]


def gd_request_stream(count, bits=16, config_id=5):
    """`count` single-operation requests (op, a, b) drawn from one integer
    gradient-descent step on regression_data, in the step's own proportions:
    products x*w and err*x (mul), partial sums and gradient sums (add),
    residuals (sub) and the per-feature scaling of the gradient (div)."""
    X, w, y = regression_data(config_id=config_id)
    m, f = X.shape
    ops = []
    for i in range(m):
        acc = 0
        for j in range(f):
            ops.append(("mul", int(X[i, j]), int(w[j])))
            if j:
                ops.append(("add", int(acc), int(X[i, j] * w[j])))
            acc += int(X[i, j] * w[j])
        ops.append(("sub", int(acc), int(y[i])))
        err = acc - int(y[i])
        for j in range(f):
            ops.append(("mul", int(err), int(X[i, j])))
    for j in range(f):
        grad = int((X @ w - y) @ X[:, j])
        ops.append(("div", grad, m))
    r = rng(config_id * 7 + 1)
    pick = r.choice(len(ops), size=count, replace=count > len(ops))
    out = []
    for k_ in pick:
        op, a, b = ops[k_]
        a, b = int(wrap_int(a, bits)), int(wrap_int(b, bits))
        if op == "div" and b == 0:
            b = 1
        out.append((op, a, b))
    return out


def expected_result(op, a, b, bits=16):
    """Native two's-complement result of one request (q, r for div)."""
    if op == "add":
        return int(wrap_int(a + b, bits))
    if op == "sub":
        return int(wrap_int(a - b, bits))
    if op == "mul":
        return int(a * b)
    q = int(np.trunc(a / b))
    return q, a - q * b


def poisson_arrivals(count, rate, config_id=5):
    """Arrival times (seconds) of a Poisson process of the given rate."""
    r = rng(config_id * 13 + 2)
    return np.cumsum(r.exponential(1.0 / rate, size=count))

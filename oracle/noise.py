"""Output noise of the oracle's bootstrapped gates (test infrastructure).

Measures, with the oracle alone, the phase error of gate outputs at the
full-size parameters (n = 560, N = 1024, base 2^8, d = 3, key switch base
2^2, t = 8, LWE sigma 2^-15) for a given party count k and RLWE sigma:
every output of gate bit m should have phase m/4 (Sec. 3.2: SymDec reads
the bit from the phase; the bootstrap maps its window onto 0 or 1/4), and
its error e = phase - m/4 (as a signed torus value) is the noise that the
next gate's linear part consumes.  The worst consumer is XOR (Eq. 10, with
the reading of its constant): its input phase carries 2 (e1 - e2), of
standard deviation 2 sqrt(2) sigma_out, against the 1/8 half-width of the
decision window.  The script reports sigma_out and z = (1/8) / (2 sqrt(2)
sigma_out); the presets take the largest RLWE sigma of the ladder
{2^-25, 2^-28, 2^-30, 2^-32} with z >= 6.

Inputs are joint-key encryptions (every party block uniform), so all k n
CMux steps of the blind rotation run.  Seeds come from
paper_2205_05825_gb300/workloads.py (parameters and seeds only).

    python -m oracle.noise --parties 4 --sigma-log2 -30 --gates 48
"""
import argparse
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as o  # noqa: E402
from paper_2205_05825_gb300 import workloads as W  # noqa: E402

TRUTH = [lambda a, b: a & b, lambda a, b: a | b, lambda a, b: 1 - (a & b),
         lambda a, b: 1 - (a | b), lambda a, b: a ^ b, lambda a, b: 1 - (a ^ b)]


def output_errors(params, keys, types, b1, b2, out):
    """Signed torus error (as a fraction of the torus) of each output phase
    against m/4 for the gate's plaintext result m."""
    ph = o.phase(params, keys, out).astype(np.int64)
    m = np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)], np.int64)
    err = (ph - m * (1 << 30)) & 0xFFFFFFFF
    err = np.where(err >= 1 << 31, err - (1 << 32), err)
    return err.astype(np.float64) / 2.0 ** 32


def measure(k, sigma_rlwe, gates, seed_config=90, threads=None):
    params = W.full_params(k)
    params["sigma_rlwe"] = float(sigma_rlwe)
    keys = o.keygen(params, W.CRS_SEED, W.party_seeds(k), nthreads=threads)
    types, b1, b2 = W.random_gates(gates, config_id=seed_config)
    c1 = o.encrypt_joint(params, keys, b1, W.encryption_seed(seed_config, 0))
    c2 = o.encrypt_joint(params, keys, b2, W.encryption_seed(seed_config, 1))
    t0 = time.perf_counter()
    out = o.gates(params, keys, types, c1, c2, nthreads=threads)
    dt = time.perf_counter() - t0
    e = output_errors(params, keys, types, b1, b2, out)
    sd = float(np.sqrt(np.mean(e * e)))
    z = 0.125 / (2.0 * math.sqrt(2.0) * sd) if sd > 0 else float("inf")
    ok = bool(np.array_equal(o.decrypt(params, keys, out),
                             np.array([TRUTH[int(t)](int(x), int(y)) for t, x, y in zip(types, b1, b2)],
                                      np.uint8)))
    return {"parties": k, "sigma_rlwe_log2": math.log2(sigma_rlwe), "gates": gates, "sigma_out": sd,
            "max_abs_err": float(np.max(np.abs(e))), "xor_margin_z": z, "decrypt_ok": ok, "seconds": dt}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--parties", type=int, nargs="+", default=[4])
    ap.add_argument("--sigma-log2", type=float, nargs="+", default=[-30.0])
    ap.add_argument("--gates", type=int, default=48)
    args = ap.parse_args()
    for k in args.parties:
        for s in args.sigma_log2:
            print(measure(k, 2.0 ** s, args.gates), flush=True)


if __name__ == "__main__":
    main()

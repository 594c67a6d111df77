"""Independent reference helpers for the oracle pins (Python integers, no
shared code with the oracle or the library)."""
import numpy as np

M32 = (1 << 32) - 1


def negacyclic(p, q):
    """p * q in Z[X]/(X^N + 1) mod 2^32: full product, then X^N -> -1."""
    N = len(p)
    full = np.convolve(np.array([int(x) for x in p], dtype=object), np.array([int(x) for x in q], dtype=object))
    out = [0] * N
    for i, v in enumerate(full):
        if i < N:
            out[i] += v
        else:
            out[i - N] -= v
    return np.array([x & M32 for x in out], dtype=np.uint32)


def rlwe_phase(c, z):
    """c_0 + sum_j c_j * z_j for c [(k+1), N] and z [k, N]."""
    ph = np.array([int(x) for x in c[0]], dtype=object)
    for j in range(1, len(c)):
        ph = ph + np.array([int(x) for x in negacyclic(c[j], z[j - 1])], dtype=object)
    return np.array([x & M32 for x in ph], dtype=np.uint32)


def signed32(x):
    x = np.asarray(x, dtype=np.int64) & M32
    return np.where(x >= 1 << 31, x - (1 << 32), x)


def torus_dist(a, b):
    """|a - b| on the torus, in torus32 units."""
    return np.abs(signed32(np.asarray(a, np.int64) - np.asarray(b, np.int64)))

"""ctypes wrapper of the CPU oracle (test infrastructure only).

The oracle is the plain, slow reference implementation of multi-key TFHE gate
bootstrapping written from the paper (arXiv 2205.05825, Sec. 3.2, Sec. 4.1-4.2,
Eq. 6-11, Algorithms 1-2, Table 1, Table 7); see ``mk_oracle.c`` for the
definitions and the readings of points the paper leaves open.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may import
this module.  It imports nothing from the product package.
"""
import ctypes
import os

import numpy as np

from . import build as _build

U32P = ctypes.POINTER(ctypes.c_uint32)
I32P = ctypes.POINTER(ctypes.c_int32)
U8P = ctypes.POINTER(ctypes.c_uint8)

GATES = {"AND": 0, "OR": 1, "NAND": 2, "NOR": 3, "XOR": 4, "XNOR": 5}


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("N", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("bg_bit", ctypes.c_uint32), ("d", ctypes.c_uint32), ("ks_bit", ctypes.c_uint32),
                ("t", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("sigma_lwe", ctypes.c_double), ("sigma_rlwe", ctypes.c_double)]

    @classmethod
    def from_dict(cls, p):
        return cls(p["n"], p["N"], p["k"], p["bg_bit"], p["d"], p["ks_bit"], p["t"], 0,
                   float(p["sigma_lwe"]), float(p["sigma_rlwe"]))

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


_lib = None


def lib():
    global _lib
    if _lib is None:
        # MK_ORACLE_LIB points the tests at a deliberately broken copy of the
        # oracle (mutant checks of the pins); normal use builds mk_oracle.c.
        path = os.environ.get("MK_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(Params)
        sig = {
            "orc_params_check": (ctypes.c_int, [P]),
            "orc_philox4x32_10": (None, [U32P, U32P, U32P]),
            "orc_word": (ctypes.c_uint32, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]),
            "orc_normal": (ctypes.c_double, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]),
            "orc_gauss32": (ctypes.c_uint32, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                              ctypes.c_double]),
            "orc_negacyclic_mul": (None, [ctypes.c_uint32, U32P, U32P, U32P]),
            "orc_monomial_mul": (None, [ctypes.c_uint32, ctypes.c_uint32, U32P, U32P]),
            "orc_gadget_decompose": (None, [P, ctypes.c_uint32, I32P]),
            "orc_keygen_crs": (None, [P, ctypes.c_uint64, U32P]),
            "orc_keygen_party": (None, [P, U32P, ctypes.c_uint64, U32P, U32P, U32P, U32P, U32P,
                                        ctypes.c_int]),
            "orc_encrypt": (None, [P, ctypes.c_uint32, U32P, ctypes.c_uint64, U8P, ctypes.c_size_t,
                                   U32P]),
            "orc_encrypt_joint": (None, [P, U32P, ctypes.c_uint64, U8P, ctypes.c_size_t, U32P]),
            "orc_phase": (ctypes.c_uint32, [P, U32P, U32P]),
            "orc_decrypt": (None, [P, U32P, U32P, ctypes.c_size_t, U8P]),
            "orc_mod_to_t": (ctypes.c_uint32, [ctypes.c_int32, ctypes.c_uint32]),
            "orc_lwe_add": (None, [P, U32P, U32P, U32P]),
            "orc_lwe_sub": (None, [P, U32P, U32P, U32P]),
            "orc_lwe_mul": (None, [P, U32P, ctypes.c_int32, U32P, U32P]),
            "orc_gate_linear": (ctypes.c_int, [P, ctypes.c_int, U32P, U32P, U32P]),
            "orc_lin_comb": (None, [P, ctypes.c_uint32, ctypes.c_int32, U32P, ctypes.c_int32, U32P,
                                    U32P]),
            "orc_not": (None, [P, U32P, U32P]),
            "orc_mod_switch": (ctypes.c_uint32, [P, ctypes.c_uint32]),
            "orc_sample_extract": (None, [P, U32P, U32P]),
            "orc_hybrid_product_flat": (None, [P, U32P, U32P, U32P, U32P, ctypes.c_uint32, U32P]),
            "orc_gates": (ctypes.c_int, [P, I32P, U32P, U32P, ctypes.c_size_t, U32P, U32P, U32P,
                                         U32P, U32P, ctypes.c_int]),
            "orc_blind_rotate_batch": (None, [P, U32P, ctypes.c_size_t, U32P, U32P, U32P,
                                              ctypes.c_int64, U32P, ctypes.c_int]),
            "orc_bootstrap_batch": (None, [P, U32P, ctypes.c_size_t, U32P, U32P, U32P, U32P,
                                           ctypes.c_int]),
            "orc_keyswitch_batch": (None, [P, U32P, U32P, ctypes.c_size_t, U32P, ctypes.c_int]),
            "orc_max_threads": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(U32P)


def _p(params):
    return ctypes.byref(params if isinstance(params, Params) else Params.from_dict(params))


def default_threads():
    return int(os.environ.get("MK_ORACLE_THREADS", "0")) or lib().orc_max_threads()


# ----------------------------------------------------------------------------- RNG
def philox(ctr, key):
    c, cp = _u32(ctr)
    k_, kp = _u32(key)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(cp, kp, out.ctypes.data_as(U32P))
    return out


def word(seed, tag, q):
    return int(lib().orc_word(seed, tag, q))


def normal(seed, tag, q):
    return float(lib().orc_normal(seed, tag, q))


def gauss32(seed, tag, q, sigma):
    return int(lib().orc_gauss32(seed, tag, q, sigma))


# ----------------------------------------------------------------------------- polynomials
def negacyclic_mul(p, q):
    p, pp = _u32(p)
    q, qp = _u32(q)
    out = np.zeros(len(p), np.uint32)
    lib().orc_negacyclic_mul(len(p), pp, qp, out.ctypes.data_as(U32P))
    return out


def monomial_mul(e, p):
    p, pp = _u32(p)
    out = np.zeros(len(p), np.uint32)
    lib().orc_monomial_mul(len(p), e, pp, out.ctypes.data_as(U32P))
    return out


def gadget_decompose(params, x):
    d = params["d"] if isinstance(params, dict) else params.d
    out = np.zeros(d, np.int32)
    lib().orc_gadget_decompose(_p(params), int(x) & 0xFFFFFFFF, out.ctypes.data_as(I32P))
    return out


def mod_switch(params, x):
    return int(lib().orc_mod_switch(_p(params), int(x) & 0xFFFFFFFF))


def mod_to_t(num, den):
    return int(lib().orc_mod_to_t(num, den))


# ----------------------------------------------------------------------------- keys
class Keys:
    """All parties' key material as produced by the oracle's key generator."""

    def __init__(self, params, crs, s, z, pk, bk, ks):
        self.params = params
        self.crs, self.s, self.z, self.pk, self.bk, self.ks = crs, s, z, pk, bk, ks

    @property
    def s_all(self):
        return np.ascontiguousarray(self.s.reshape(-1))


def key_shapes(params):
    n, N, k, d, t = params["n"], params["N"], params["k"], params["d"], params["t"]
    nb = (1 << params["ks_bit"]) - 1
    return dict(crs=(d, N), s=(k, n), z=(k, N), pk=(k, d, N), bk=(k, n, 3, d, N),
                ks=(k, N, t, nb, n + 1))


def keygen(params, crs_seed, party_seeds, nthreads=None):
    """MKTFHE.Setup + MKTFHE.KeyGen for every party (Sec. 3.2)."""
    nthreads = default_threads() if nthreads is None else nthreads
    sh = key_shapes(params)
    crs = np.zeros(sh["crs"], np.uint32)
    lib().orc_keygen_crs(_p(params), crs_seed, crs.ctypes.data_as(U32P))
    arrs = {name: np.zeros(sh[name], np.uint32) for name in ("s", "z", "pk", "bk", "ks")}
    for i, seed in enumerate(party_seeds):
        lib().orc_keygen_party(_p(params), crs.ctypes.data_as(U32P), seed,
                               *[arrs[nm][i].ctypes.data_as(U32P) for nm in ("s", "z", "pk", "bk", "ks")],
                               nthreads)
    return Keys(params, crs, arrs["s"], arrs["z"], arrs["pk"], arrs["bk"], arrs["ks"])


# ----------------------------------------------------------------------------- enc / dec
def ct_width(params):
    return params["k"] * params["n"] + 1


def encrypt(params, keys, party, bits, seed):
    bits = np.ascontiguousarray(bits, np.uint8)
    out = np.zeros((len(bits), ct_width(params)), np.uint32)
    s, sp = _u32(keys.s[party])
    lib().orc_encrypt(_p(params), party, sp, seed, bits.ctypes.data_as(U8P), len(bits),
                      out.ctypes.data_as(U32P))
    return out


def encrypt_joint(params, keys, bits, seed):
    bits = np.ascontiguousarray(bits, np.uint8)
    out = np.zeros((len(bits), ct_width(params)), np.uint32)
    s, sp = _u32(keys.s_all)
    lib().orc_encrypt_joint(_p(params), sp, seed, bits.ctypes.data_as(U8P), len(bits),
                            out.ctypes.data_as(U32P))
    return out


def phase(params, keys, ct):
    ct = np.ascontiguousarray(ct, np.uint32).reshape(-1, ct_width(params))
    s, sp = _u32(keys.s_all)
    return np.array([lib().orc_phase(_p(params), sp, row.ctypes.data_as(U32P)) for row in ct],
                    dtype=np.uint32)


def decrypt(params, keys, ct):
    ct, cp = _u32(np.asarray(ct).reshape(-1, ct_width(params)))
    out = np.zeros(len(ct), np.uint8)
    s, sp = _u32(keys.s_all)
    lib().orc_decrypt(_p(params), sp, cp, len(ct), out.ctypes.data_as(U8P))
    return out


# ----------------------------------------------------------------------------- gates
def _row_op(fn, params, *rows):
    rows = [_u32(r) for r in rows]
    out = np.zeros(ct_width(params), np.uint32)
    fn(_p(params), *[r[1] for r in rows], out.ctypes.data_as(U32P))
    return out


def lwe_add(params, c1, c2):
    return _row_op(lib().orc_lwe_add, params, c1, c2)


def lwe_sub(params, c1, c2):
    return _row_op(lib().orc_lwe_sub, params, c1, c2)


def lwe_mul(params, c1, kk, c2):
    a, ap = _u32(c1)
    b, bp = _u32(c2)
    out = np.zeros(ct_width(params), np.uint32)
    lib().orc_lwe_mul(_p(params), ap, kk, bp, out.ctypes.data_as(U32P))
    return out


def gate_linear(params, gate, c1, c2):
    a, ap = _u32(c1)
    b, bp = _u32(c2)
    out = np.zeros(ct_width(params), np.uint32)
    rc = lib().orc_gate_linear(_p(params), GATES[gate] if isinstance(gate, str) else gate, ap, bp,
                               out.ctypes.data_as(U32P))
    assert rc == 0
    return out


def lin_comb(params, cst, s1, c1, s2, c2):
    a, ap = _u32(c1)
    b, bp = _u32(c2)
    out = np.zeros(ct_width(params), np.uint32)
    lib().orc_lin_comb(_p(params), cst & 0xFFFFFFFF, s1, ap, s2, bp, out.ctypes.data_as(U32P))
    return out


def mk_not(params, c):
    return _row_op(lib().orc_not, params, c)


def sample_extract(params, acc):
    a, ap = _u32(acc)
    out = np.zeros(params["k"] * params["N"] + 1, np.uint32)
    lib().orc_sample_extract(_p(params), ap, out.ctypes.data_as(U32P))
    return out


def hybrid_product(params, keys, c, party, j):
    """HP of the MK RLWE ciphertext c [(k+1), N] with BK_{party, j} (party 1..k)."""
    c, cp = _u32(c)
    bk, bkp = _u32(keys.bk[party - 1, j])
    crs, crsp = _u32(keys.crs)
    pk, pkp = _u32(keys.pk)
    out = np.zeros_like(c)
    lib().orc_hybrid_product_flat(_p(params), cp, bkp, crsp, pkp, party, out.ctypes.data_as(U32P))
    return out


def gates(params, keys, types, c1, c2, nthreads=None):
    nthreads = default_threads() if nthreads is None else nthreads
    types = np.ascontiguousarray(types, np.int32)
    c1, c1p = _u32(c1)
    c2, c2p = _u32(c2)
    out = np.zeros_like(c1)
    crs, crsp = _u32(keys.crs)
    pk, pkp = _u32(keys.pk)
    bk, bkp = _u32(keys.bk)
    ks, ksp = _u32(keys.ks)
    rc = lib().orc_gates(_p(params), types.ctypes.data_as(I32P), c1p, c2p, len(types), crsp, pkp,
                         bkp, ksp, out.ctypes.data_as(U32P), nthreads)
    assert rc == 0
    return out


def modswitch_input(params, c):
    """The blind rotation's input: every word mod-switched, b after the -1/4 shift."""
    c = np.asarray(c, np.uint32).reshape(-1, ct_width(params))
    out = np.zeros_like(c)
    for g in range(len(c)):
        for x in range(c.shape[1] - 1):
            out[g, x] = mod_switch(params, c[g, x])
        out[g, -1] = mod_switch(params, (int(c[g, -1]) - (1 << 30)) & 0xFFFFFFFF)
    return out


def blind_rotate(params, keys, abar, max_steps=-1, nthreads=None):
    nthreads = default_threads() if nthreads is None else nthreads
    abar, ap = _u32(np.asarray(abar).reshape(-1, ct_width(params)))
    out = np.zeros((len(abar), params["k"] + 1, params["N"]), np.uint32)
    crs, crsp = _u32(keys.crs)
    pk, pkp = _u32(keys.pk)
    bk, bkp = _u32(keys.bk)
    lib().orc_blind_rotate_batch(_p(params), ap, len(abar), crsp, pkp, bkp, max_steps,
                                 out.ctypes.data_as(U32P), nthreads)
    return out


def bootstrap(params, keys, c, nthreads=None):
    nthreads = default_threads() if nthreads is None else nthreads
    c, cp = _u32(np.asarray(c).reshape(-1, ct_width(params)))
    out = np.zeros((len(c), params["k"] * params["N"] + 1), np.uint32)
    crs, crsp = _u32(keys.crs)
    pk, pkp = _u32(keys.pk)
    bk, bkp = _u32(keys.bk)
    lib().orc_bootstrap_batch(_p(params), cp, len(c), crsp, pkp, bkp, out.ctypes.data_as(U32P),
                              nthreads)
    return out


def keyswitch(params, keys, lwe, nthreads=None):
    nthreads = default_threads() if nthreads is None else nthreads
    lwe, lp = _u32(np.asarray(lwe).reshape(-1, params["k"] * params["N"] + 1))
    out = np.zeros((len(lwe), ct_width(params)), np.uint32)
    ks, ksp = _u32(keys.ks)
    lib().orc_keyswitch_batch(_p(params), ksp, lp, len(lwe), out.ctypes.data_as(U32P), nthreads)
    return out

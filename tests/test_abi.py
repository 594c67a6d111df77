"""The C-ABI library builds, loads without a GPU, and exports every function
include/*.h declares; host-only contexts work without a device."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mk_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import build
    build.build()
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2205_05825_gb300 import binding as B
    assert set(declared_functions()) <= set(B._SIGS)


def test_host_only_context_errors_and_presets(lib):
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    assert B.preset("toy", 2) == W.toy_params(2)
    assert B.preset("full", 2) == W.full_params(2)
    assert B.preset("full", 4) == W.full_params(4)
    ctx = B.Context(W.toy_params(2), W.CRS_SEED, device=-1)
    with pytest.raises(B.MkError, match="MK_ESTATE"):
        ctx.encrypt(0, np.array([1], np.uint8), 1)
    with pytest.raises(B.MkError, match="MK_EINVAL"):
        ctx.keygen(5, 1)
    ctx.keygen(0, 1)
    ctx.keygen(1, 2)
    blob = ctx.save_keys()
    bad = blob.copy()
    bad[100] ^= 1
    ctx2 = B.Context(W.toy_params(2), W.CRS_SEED, device=-1)
    with pytest.raises(B.MkError, match="MK_EFORMAT"):
        ctx2.load_keys(bad)
    with pytest.raises(B.MkError, match="MK_EFORMAT"):
        ctx2.load_keys(blob[:-9])
    ctx2.load_keys(blob)
    assert np.array_equal(ctx2.export_party(1)["bk"], ctx.export_party(1)["bk"])
    pub = ctx.save_keys(include_secrets=False)
    ctx3 = B.Context(W.toy_params(2), W.CRS_SEED, device=-1)
    ctx3.load_keys(pub)
    with pytest.raises(B.MkError, match="MK_ESTATE"):
        ctx3.export_party(0, parts=("s",))
    bad_params = dict(W.toy_params(2), N=512)
    with pytest.raises(B.MkError, match="MK_EPARAMS"):
        B.Context(bad_params, 1, device=-1)


def test_library_keygen_and_encrypt_byte_equal_to_oracle():
    """Host key generation and SymEnc of the library equal the oracle's
    (same seeds, same Philox streams, same Box-Muller samples)."""
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    keys = o.keygen(P, W.CRS_SEED, W.party_seeds(2))
    ctx = B.Context(P, W.CRS_SEED, device=-1)
    for i, s in enumerate(W.party_seeds(2)):
        ctx.keygen(i, s)
    assert np.array_equal(ctx.export_crs(), keys.crs)
    for i in range(2):
        e = ctx.export_party(i)
        for nm in ("s", "z", "pk", "bk", "ks"):
            assert np.array_equal(e[nm], getattr(keys, nm)[i]), nm
    bits = np.array([0, 1, 1, 0, 1, 0, 0, 1], np.uint8)
    assert np.array_equal(ctx.encrypt(1, bits, 99), o.encrypt(P, keys, 1, bits, 99))
    assert np.array_equal(ctx.encrypt_joint(bits, 98), o.encrypt_joint(P, keys, bits, 98))
    c = o.encrypt(P, keys, 0, bits, 97)
    assert np.array_equal(ctx.decrypt(c), bits)
    assert np.array_equal(ctx.phase(c), o.phase(P, keys, c))


def test_trivial_ciphertexts_of_public_bits():
    """mk_trivial: zero mask, b = m/4, no secret needed; the oracle decrypts
    it to the bit under the parties' keys with phase exactly m/4, and its
    gates treat it like any other ciphertext of that bit."""
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.toy_params(2)
    keys = o.keygen(P, W.CRS_SEED, W.party_seeds(2))
    ctx = B.Context(P, W.CRS_SEED, device=-1)    # no keys at all
    bits = np.array([1, 0, 1, 1, 0, 3, 2], np.uint8)  # only the lowest bit counts
    t = ctx.trivial(bits)
    assert t.shape == (len(bits), ctx.W) and not t[:, :-1].any()
    assert np.array_equal(o.phase(P, keys, t), (bits & 1).astype(np.uint32) << 30)
    assert np.array_equal(o.decrypt(P, keys, t), bits & 1)
    x = o.encrypt(P, keys, 0, np.array([1, 0, 1, 0], np.uint8), 55)
    one, zero = ctx.trivial([1, 1, 1, 1]), ctx.trivial([0, 0, 0, 0])
    g = np.array([0, 0, 4, 4], np.int32)         # AND, AND, XOR, XOR
    out = o.gates(P, keys, g, x, np.concatenate([one[:2], zero[:2]]))
    assert list(o.decrypt(P, keys, out)) == [1, 0, 1, 0]


def test_trivial_argument_errors(lib):
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    ctx = B.Context(W.toy_params(2), W.CRS_SEED, device=-1)
    einval = -1
    assert ctx.L.mk_trivial(ctx.h, None, 3, None) == einval    # null pointers with count > 0
    assert ctx.L.mk_trivial(ctx.h, None, 0, None) == B.MK_OK   # nothing to do
    assert ctx.L.mk_trivial(None, None, 0, None) == einval     # no context
    assert ctx.trivial(np.zeros(0, np.uint8)).shape == (0, ctx.W)


def test_circuit_style_setting(lib):
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    ctx = B.Context(W.toy_params(2), W.CRS_SEED, device=-1)
    assert ctx.get_circuit_style() == "array"
    ctx.set_circuit_style("shallow")
    assert ctx.get_circuit_style() == "shallow"
    with pytest.raises(B.MkError):
        ctx.set_circuit_style(7)
    assert ctx.get_circuit_style() == "shallow"
    with pytest.raises(B.MkError):
        B.circuit_netlist("add", 8, 5)


def test_gate_lin_records_match_oracle_linear_part():
    """mk_gate_lin (the library's Eq. 6-11 records, with NOT folded in on
    request) gives the oracle's linear combination of two ciphertexts, for
    every gate type and input negation."""
    import numpy as np
    from oracle import oracle as o
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.tiny_params(2)
    rng = np.random.default_rng(5)
    c1 = rng.integers(0, 1 << 32, size=o.ct_width(P), dtype=np.uint64).astype(np.uint32)
    c2 = rng.integers(0, 1 << 32, size=o.ct_width(P), dtype=np.uint64).astype(np.uint32)
    for t in range(6):
        for na in (False, True):
            for nb in (False, True):
                cst, s1, s2 = B.gate_lin(t, na, nb)
                a = o.mk_not(P, c1) if na else c1
                b = o.mk_not(P, c2) if nb else c2
                assert np.array_equal(o.lin_comb(P, cst, s1, c1, s2, c2), o.gate_linear(P, t, a, b))
    with pytest.raises(B.MkError):
        B.gate_lin(6)

"""The pins must catch plausible mistakes: each case plants one mistake in a
copy of the oracle's C source (on the CPU), builds it, and runs the pin suite
against that copy, which must fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mk_oracle.c")

MUTANTS = [
    ("hybrid product: +<u_0, a> instead of -<u_0, a>",
     "for (uint32_t m = 0; m < N; ++m) negu[m] = 0u - ul[m];", "for (uint32_t m = 0; m < N; ++m) negu[m] = ul[m];"),
    ("hybrid product: f1 added to c'_0 instead of c'_i",
     "out + (size_t)party * N);   /* c'_i += <w, f1> */", "out);   /* c'_i += <w, f1> */"),
    ("negacyclic product: wrap added instead of subtracted",
     "for (uint32_t j = N - i; j < N; ++j) r[i + j - N] -= pi * q[j];",
     "for (uint32_t j = N - i; j < N; ++j) r[i + j - N] += pi * q[j];"),
    ("SampleExtract: a_i[m] = +c_i[N-m]", "for (uint32_t m = 1; m < N; ++m) ai[m] = 0u - ci[N - m];",
     "for (uint32_t m = 1; m < N; ++m) ai[m] = ci[N - m];"),
    ("blind rotation: X^{+e} instead of X^{-e}",
     "orc_monomial_mul(N, (2 * N - e) % (2 * N), acc + (size_t)p * N, rot + (size_t)p * N);",
     "orc_monomial_mul(N, e, acc + (size_t)p * N, rot + (size_t)p * N);"),
    ("key switch: no rounding offset", "const uint32_t round_off = 1u << (32 - prec - 1);",
     "const uint32_t round_off = 0;"),
    ("gadget: no rounding at the last digit", "offset += 1u << (32 - P->bg_bit * P->d - 1); /* rounding */",
     "offset += 0; /* rounding */"),
    ("NOR with the printed constant 1/8", "lwe_trivial(P, orc_mod_to_t(3, 8), tr);",
     "lwe_trivial(P, orc_mod_to_t(1, 8), tr);"),
    ("bootstrap without the -1/4 window shift", "abar[W - 1] = orc_mod_switch(P, c[W - 1] - (1u << 30));",
     "abar[W - 1] = orc_mod_switch(P, c[W - 1]);"),
    ("public key sign", "pk[(size_t)l * N + m] = (0u - tmp[m]) +", "pk[(size_t)l * N + m] = tmp[m] +"),
    ("Philox: key schedule constant", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;"),
    ("mod switch truncates", "return (uint32_t)((((uint64_t)x + (1ull << (sh - 1))) >> sh) & (2u * P->N - 1));",
     "return (uint32_t)((((uint64_t)x) >> sh) & (2u * P->N - 1));"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(desc, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + desc
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           str(mut), "-o", str(lib), "-lm"])
    env = dict(os.environ, MK_ORACLE_LIB=str(lib), MK_ORACLE_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "pins did not catch: " + desc

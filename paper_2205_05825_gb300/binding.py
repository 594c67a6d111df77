"""Thin ctypes binding of ``libmktfhe.so`` (the C ABI in include/mk_tfhe.h).

Argument marshalling only: every step of a gate runs in the library's CUDA
kernels.  Device buffers are torch tensors (uint32 as torch.int32 storage);
host buffers are numpy arrays.  Loading fails loudly when the library has not
been built -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MK_OK = 0
ERRORS = {-1: "MK_EINVAL", -2: "MK_ENOMEM", -3: "MK_EPARAMS", -4: "MK_ETIMEOUT", -5: "MK_EDEVICE",
          -6: "MK_ESTATE", -7: "MK_EFORMAT"}
GATES = {"AND": 0, "OR": 1, "NAND": 2, "NOR": 3, "XOR": 4, "XNOR": 5}
PRESETS = {"toy": 0, "full": 1, "paper": 2}
NUM_VARIANTS = 9
FORMS = {"ntt": 0, "ntt2": 1, "fft": 2, "tc": 3}
CLUSTER_MODES = {"auto": 0, "off": 1, "on": 2}
CIRCUIT_STYLES = {"array": 0, "shallow": 1, "paper": 2, "nand": 3}

U32P = ctypes.POINTER(ctypes.c_uint32)
U8P = ctypes.POINTER(ctypes.c_uint8)
VP = ctypes.c_void_p


class MkParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("N", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("bg_bit", ctypes.c_uint32), ("d", ctypes.c_uint32), ("ks_bit", ctypes.c_uint32),
                ("t", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("sigma_lwe", ctypes.c_double), ("sigma_rlwe", ctypes.c_double)]

    @classmethod
    def from_dict(cls, p):
        return cls(p["n"], p["N"], p["k"], p["bg_bit"], p["d"], p["ks_bit"], p["t"], 0,
                   float(p["sigma_lwe"]), float(p["sigma_rlwe"]))

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class MkLin(ctypes.Structure):
    _fields_ = [("cst", ctypes.c_uint32), ("s1", ctypes.c_int32), ("s2", ctypes.c_int32)]


class MkError(RuntimeError):
    pass


_SIGS = {
    "mk_params_preset": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(MkParams)]),
    "mk_ctx_create": (ctypes.c_int, [ctypes.POINTER(MkParams), ctypes.c_uint64, ctypes.c_int, VP,
                                     ctypes.POINTER(VP)]),
    "mk_ctx_destroy": (ctypes.c_int, [VP]),
    "mk_ctx_set_stream": (ctypes.c_int, [VP, VP]),
    "mk_ctx_get_params": (ctypes.c_int, [VP, ctypes.POINTER(MkParams)]),
    "mk_ctx_set_form": (ctypes.c_int, [VP, ctypes.c_int]),
    "mk_ctx_get_form": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int)]),
    "mk_ctx_set_batch": (ctypes.c_int, [VP, ctypes.c_uint32]),
    "mk_last_error": (ctypes.c_char_p, [VP]),
    "mk_sync": (ctypes.c_int, [VP]),
    "mk_keygen": (ctypes.c_int, [VP, ctypes.c_uint32, ctypes.c_uint64]),
    "mk_import_crs": (ctypes.c_int, [VP, U32P]),
    "mk_import_party": (ctypes.c_int, [VP, ctypes.c_uint32, U32P, U32P, U32P, U32P, U32P]),
    "mk_export_crs": (ctypes.c_int, [VP, U32P]),
    "mk_export_party": (ctypes.c_int, [VP, ctypes.c_uint32, U32P, U32P, U32P, U32P, U32P]),
    "mk_save_keys": (ctypes.c_int, [VP, ctypes.c_int, VP, ctypes.c_size_t,
                                    ctypes.POINTER(ctypes.c_size_t)]),
    "mk_load_keys": (ctypes.c_int, [VP, VP, ctypes.c_size_t]),
    "mk_encrypt": (ctypes.c_int, [VP, ctypes.c_uint32, U8P, ctypes.c_size_t, ctypes.c_uint64, U32P]),
    "mk_encrypt_joint": (ctypes.c_int, [VP, U8P, ctypes.c_size_t, ctypes.c_uint64, U32P]),
    "mk_trivial": (ctypes.c_int, [VP, U8P, ctypes.c_size_t, U32P]),
    "mk_decrypt": (ctypes.c_int, [VP, VP, ctypes.c_size_t, ctypes.c_int, U8P]),
    "mk_phase": (ctypes.c_int, [VP, VP, ctypes.c_size_t, ctypes.c_int, U32P]),
    "mk_gate": (ctypes.c_int, [VP, ctypes.c_int, VP, VP, VP, ctypes.c_size_t]),
    "mk_gates": (ctypes.c_int, [VP, VP, VP, VP, VP, ctypes.c_size_t]),
    "mk_gates_lin": (ctypes.c_int, [VP, VP, VP, VP, VP, ctypes.c_size_t]),
    "mk_gate_lin": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, VP]),
    "mk_debug_fault": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64]),
    "mk_ctx_set_circuit_exec": (ctypes.c_int, [VP, ctypes.c_int]),
    "mk_not": (ctypes.c_int, [VP, VP, VP, ctypes.c_size_t]),
    "mk_gates_noalloc": (ctypes.c_int, [VP, VP, VP, VP, VP, ctypes.c_size_t]),
    "mk_stage_modswitch": (ctypes.c_int, [VP, VP, VP, VP, VP, ctypes.c_size_t]),
    "mk_stage_blind_rotate": (ctypes.c_int, [VP, VP, ctypes.c_size_t, ctypes.c_int64, VP]),
    "mk_stage_bootstrap": (ctypes.c_int, [VP, VP, VP, VP, VP, ctypes.c_size_t]),
    "mk_stage_keyswitch": (ctypes.c_int, [VP, VP, VP, ctypes.c_size_t]),
    "mk_ctx_set_variant": (ctypes.c_int, [VP, ctypes.c_int]),
    "mk_ctx_get_variant": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int)]),
    "mk_autotune": (ctypes.c_int, [VP, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_float)]),
    "mk_ctx_set_graphs": (ctypes.c_int, [VP, ctypes.c_int]),
    "mk_ctx_set_circuit_style": (ctypes.c_int, [VP, ctypes.c_int]),
    "mk_ctx_get_circuit_style": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int)]),
    "mk_ctx_set_cluster": (ctypes.c_int, [VP, ctypes.c_int]),
    "mk_autotune_form": (ctypes.c_int, [VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_float)]),
    "mk_add_kbit": (ctypes.c_int, [VP, ctypes.c_uint32, VP, VP, VP, ctypes.c_size_t]),
    "mk_sub_kbit": (ctypes.c_int, [VP, ctypes.c_uint32, VP, VP, VP, ctypes.c_size_t]),
    "mk_mul_kbit": (ctypes.c_int, [VP, ctypes.c_uint32, VP, VP, VP, ctypes.c_size_t]),
    "mk_div_kbit": (ctypes.c_int, [VP, ctypes.c_uint32, VP, VP, VP, VP, ctypes.c_size_t]),
    "mk_circuit_netlist": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, ctypes.c_int, VP, ctypes.c_uint32,
                                          ctypes.POINTER(ctypes.c_uint32), VP, ctypes.c_uint32,
                                          ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
    "mk_server_create": (ctypes.c_int, [VP, ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(VP)]),
    "mk_server_destroy": (ctypes.c_int, [VP]),
    "mk_server_submit": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_uint32, VP, VP, VP, VP, ctypes.c_uint32,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "mk_server_step": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_uint32)]),
    "mk_server_poll": (ctypes.c_int, [VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    "mk_server_stats": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
    "mk_timing_enable": (ctypes.c_int, [VP, ctypes.c_int]),
    "mk_timing_reset": (ctypes.c_int, [VP]),
    "mk_timing_read": (ctypes.c_int, [VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "mk_measure_butterfly_rate": (ctypes.c_int, [ctypes.c_int, VP, ctypes.c_int, ctypes.c_uint32,
                                                 ctypes.POINTER(ctypes.c_double)]),
    "mk_tc_negacyclic": (ctypes.c_int, [ctypes.c_int, VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        VP, VP, VP, ctypes.c_int]),
}

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load the CUDA library; raise if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise MkError("libmktfhe.so is not built (%s); run __graft_entry__.build()" % path)
        _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def preset(name, k):
    p = MkParams()
    rc = load().mk_params_preset(PRESETS[name], k, ctypes.byref(p))
    if rc != MK_OK:
        raise MkError("mk_params_preset: %s" % ERRORS.get(rc, rc))
    return p.as_dict()


def _np_u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(U32P)


def _dptr(t):
    """Device pointer of a CUDA tensor (marshalling only)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise MkError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def key_shapes(params):
    n, N, k, d, t = params["n"], params["N"], params["k"], params["d"], params["t"]
    nb = (1 << params["ks_bit"]) - 1
    return dict(crs=(d, N), s=(n,), z=(N,), pk=(d, N), bk=(n, 3, d, N), ks=(N, t, nb, n + 1))


class Context:
    """One mk_ctx: parameters, keys, device and stream."""

    def __init__(self, params, crs_seed, device=0, stream=None):
        self.L = load()
        self.params = dict(params)
        self._p = MkParams.from_dict(params)
        h = VP()
        if stream is None and device >= 0:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        rc = self.L.mk_ctx_create(ctypes.byref(self._p), crs_seed, device,
                                  ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if rc != MK_OK:
            raise MkError("mk_ctx_create: %s" % ERRORS.get(rc, rc))
        self.h = h
        self.device = device
        self.W = params["k"] * params["n"] + 1
        self.E = params["k"] * params["N"] + 1

    def close(self):
        if self.h:
            self.L.mk_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != MK_OK:
            msg = self.L.mk_last_error(self.h).decode()
            raise MkError("%s: %s (%s)" % (what, ERRORS.get(rc, rc), msg))

    # ---------------------------------------------------------------- settings
    def set_stream(self, stream):
        self._check(self.L.mk_ctx_set_stream(self.h, ctypes.c_void_p(stream or 0)), "mk_ctx_set_stream")

    def set_batch(self, n):
        self._check(self.L.mk_ctx_set_batch(self.h, n), "mk_ctx_set_batch")

    def set_form(self, form):
        self._check(self.L.mk_ctx_set_form(self.h, FORMS.get(form, form)), "mk_ctx_set_form")

    def get_form(self):
        f = ctypes.c_int()
        self._check(self.L.mk_ctx_get_form(self.h, ctypes.byref(f)), "mk_ctx_get_form")
        return f.value

    def set_variant(self, v):
        self._check(self.L.mk_ctx_set_variant(self.h, v), "mk_ctx_set_variant")

    def get_variant(self):
        v = ctypes.c_int()
        self._check(self.L.mk_ctx_get_variant(self.h, ctypes.byref(v)), "mk_ctx_get_variant")
        return v.value

    def autotune(self, sample_gates):
        """Time every blind-rotation variant; keep the fastest. -> (best, [ms per variant])."""
        best = ctypes.c_int()
        ms = (ctypes.c_float * NUM_VARIANTS)()
        self._check(self.L.mk_autotune(self.h, sample_gates, ctypes.byref(best), ms), "mk_autotune")
        return best.value, list(ms)

    def set_cluster(self, mode):
        """Latency (cluster) kernel: "auto" (small launches), "on" or "off"."""
        self._check(self.L.mk_ctx_set_cluster(self.h, CLUSTER_MODES[mode]), "mk_ctx_set_cluster")

    FAULTS = {"none": 0, "skip_key_step": 1, "skip_digit_tile": 2, "skip_wire_ready": 3}
    CIRCUIT_EXEC = {"auto": 0, "levels": 1, "persistent": 2}

    def set_circuit_exec(self, mode):
        """Operators: "levels" (a launch pair per netlist level), "persistent"
        (one launch over every gate and pair) or "auto"."""
        self._check(self.L.mk_ctx_set_circuit_exec(self.h, self.CIRCUIT_EXEC[mode]), "mk_ctx_set_circuit_exec")

    def debug_fault(self, kind="none", arg=0, wait_ns=0):
        """Test hook of the bounded waits (mk_debug_fault): skip one key copy
        of the staged kernel or one digit tile of the tcgen05 engine."""
        self._check(self.L.mk_debug_fault(self.h, self.FAULTS[kind], int(arg), int(wait_ns)), "mk_debug_fault")

    def set_graphs(self, on):
        """Replay each operator's level loop as a captured CUDA graph (default on)."""
        self._check(self.L.mk_ctx_set_graphs(self.h, 1 if on else 0), "mk_ctx_set_graphs")

    def set_circuit_style(self, style):
        """Netlist family of the operators: "array" (default) or "shallow"."""
        st = CIRCUIT_STYLES[style] if isinstance(style, str) else int(style)
        self._check(self.L.mk_ctx_set_circuit_style(self.h, st), "mk_ctx_set_circuit_style")

    def get_circuit_style(self):
        v = ctypes.c_int()
        self._check(self.L.mk_ctx_get_circuit_style(self.h, ctypes.byref(v)), "mk_ctx_get_circuit_style")
        return {b: a for a, b in CIRCUIT_STYLES.items()}[v.value]

    def autotune_form(self, sample_gates, forms=("ntt", "ntt2", "tc")):
        """Time each product form (with its best variant); keep the fastest.
        -> (best form name, {form name: ms})."""
        mask = 0
        for f in forms:
            mask |= 1 << FORMS[f]
        best = ctypes.c_int()
        ms = (ctypes.c_float * len(FORMS))()
        self._check(self.L.mk_autotune_form(self.h, sample_gates, mask, ctypes.byref(best), ms), "mk_autotune_form")
        names = {v: k for k, v in FORMS.items()}
        return names[best.value], {names[i]: ms[i] for i in range(len(FORMS)) if ms[i] > 0}

    def sync(self):
        self._check(self.L.mk_sync(self.h), "mk_sync")

    # ---------------------------------------------------------------- keys
    def keygen(self, party, seed):
        self._check(self.L.mk_keygen(self.h, party, seed), "mk_keygen")

    def import_crs(self, crs):
        a, p = _np_u32(crs)
        self._check(self.L.mk_import_crs(self.h, p), "mk_import_crs")

    def import_party(self, party, s, z, pk, bk, ks):
        arrs = [(_np_u32(x) if x is not None else (None, None)) for x in (s, z, pk, bk, ks)]
        self._check(self.L.mk_import_party(self.h, party, *[a[1] for a in arrs]), "mk_import_party")

    def import_oracle_keys(self, keys, with_secrets=True):
        """Copy a key set (numpy arrays, layouts of include/mk_tfhe.h) in."""
        self.import_crs(keys.crs)
        for i in range(self.params["k"]):
            self.import_party(i, keys.s[i] if with_secrets else None, keys.z[i] if with_secrets else None,
                              keys.pk[i], keys.bk[i], keys.ks[i])

    def export_crs(self):
        out = np.zeros(key_shapes(self.params)["crs"], np.uint32)
        self._check(self.L.mk_export_crs(self.h, out.ctypes.data_as(U32P)), "mk_export_crs")
        return out

    def export_party(self, party, parts=("s", "z", "pk", "bk", "ks")):
        sh = key_shapes(self.params)
        outs = {nm: np.zeros(sh[nm], np.uint32) for nm in parts}
        ptrs = [outs[nm].ctypes.data_as(U32P) if nm in outs else None for nm in ("s", "z", "pk", "bk", "ks")]
        self._check(self.L.mk_export_party(self.h, party, *ptrs), "mk_export_party")
        return outs

    def save_keys(self, include_secrets=True):
        n = ctypes.c_size_t()
        self._check(self.L.mk_save_keys(self.h, int(include_secrets), None, 0, ctypes.byref(n)), "mk_save_keys")
        buf = np.zeros(n.value, np.uint8)
        self._check(self.L.mk_save_keys(self.h, int(include_secrets), buf.ctypes.data_as(VP), n.value,
                                        ctypes.byref(n)), "mk_save_keys")
        return buf

    def load_keys(self, blob):
        blob = np.ascontiguousarray(blob, np.uint8)
        self._check(self.L.mk_load_keys(self.h, blob.ctypes.data_as(VP), blob.size), "mk_load_keys")

    # ---------------------------------------------------------------- enc / dec
    def encrypt(self, party, bits, seed):
        bits = np.ascontiguousarray(bits, np.uint8)
        out = np.zeros((len(bits), self.W), np.uint32)
        self._check(self.L.mk_encrypt(self.h, party, bits.ctypes.data_as(U8P), len(bits), seed,
                                      out.ctypes.data_as(U32P)), "mk_encrypt")
        return out

    def encrypt_joint(self, bits, seed):
        bits = np.ascontiguousarray(bits, np.uint8)
        out = np.zeros((len(bits), self.W), np.uint32)
        self._check(self.L.mk_encrypt_joint(self.h, bits.ctypes.data_as(U8P), len(bits), seed,
                                            out.ctypes.data_as(U32P)), "mk_encrypt_joint")
        return out

    def trivial(self, bits):
        """Noiseless ciphertexts of public bits (mk_trivial): [count][W] uint32."""
        bits = np.ascontiguousarray(bits, np.uint8)
        out = np.zeros((len(bits), self.W), np.uint32)
        self._check(self.L.mk_trivial(self.h, bits.ctypes.data_as(U8P), len(bits), out.ctypes.data_as(U32P)),
                    "mk_trivial")
        return out

    def _ct_arg(self, ct):
        if isinstance(ct, np.ndarray):
            ct = np.ascontiguousarray(ct, np.uint32)
            return ct, ct.ctypes.data_as(VP), ct.size // self.W, 0
        return ct, _dptr(ct), ct.numel() // self.W, 1

    def decrypt(self, ct):
        keep, ptr, count, dev = self._ct_arg(ct)
        out = np.zeros(count, np.uint8)
        self._check(self.L.mk_decrypt(self.h, ptr, count, dev, out.ctypes.data_as(U8P)), "mk_decrypt")
        return out

    def phase(self, ct):
        keep, ptr, count, dev = self._ct_arg(ct)
        out = np.zeros(count, np.uint32)
        self._check(self.L.mk_phase(self.h, ptr, count, dev, out.ctypes.data_as(U32P)), "mk_phase")
        return out

    # ---------------------------------------------------------------- gates (device tensors)
    def gate(self, gate, a, b, out):
        ty = GATES[gate] if isinstance(gate, str) else int(gate)
        self._check(self.L.mk_gate(self.h, ty, _dptr(a), _dptr(b), _dptr(out), a.numel() // self.W), "mk_gate")
        return out

    def gates(self, types, a, b, out):
        self._check(self.L.mk_gates(self.h, _dptr(types), _dptr(a), _dptr(b), _dptr(out), types.numel()),
                    "mk_gates")
        return out

    def gates_noalloc(self, types, a, b, out):
        """mk_gates without any device allocation (fixed scratch; see mk_tfhe.h)."""
        self._check(self.L.mk_gates_noalloc(self.h, _dptr(types), _dptr(a), _dptr(b), _dptr(out), types.numel()),
                    "mk_gates_noalloc")
        return out

    def gates_lin(self, lin, a, b, out):
        """lin: CUDA int32 tensor [count, 3] of (cst, s1, s2)."""
        self._check(self.L.mk_gates_lin(self.h, _dptr(lin), _dptr(a), _dptr(b), _dptr(out), lin.shape[0]),
                    "mk_gates_lin")
        return out

    def mk_not(self, a, out):
        self._check(self.L.mk_not(self.h, _dptr(a), _dptr(out), a.numel() // self.W), "mk_not")
        return out

    # ---------------------------------------------------------------- operators (device tensors)
    def add_kbit(self, kbits, a, b, out):
        pairs = a.numel() // (kbits * self.W)
        self._check(self.L.mk_add_kbit(self.h, kbits, _dptr(a), _dptr(b), _dptr(out), pairs), "mk_add_kbit")
        return out

    def sub_kbit(self, kbits, a, b, out):
        pairs = a.numel() // (kbits * self.W)
        self._check(self.L.mk_sub_kbit(self.h, kbits, _dptr(a), _dptr(b), _dptr(out), pairs), "mk_sub_kbit")
        return out

    def mul_kbit(self, kbits, a, b, out):
        pairs = a.numel() // (kbits * self.W)
        self._check(self.L.mk_mul_kbit(self.h, kbits, _dptr(a), _dptr(b), _dptr(out), pairs), "mk_mul_kbit")
        return out

    def div_kbit(self, kbits, a, b, q, r):
        pairs = a.numel() // (kbits * self.W)
        self._check(self.L.mk_div_kbit(self.h, kbits, _dptr(a), _dptr(b), _dptr(q), _dptr(r), pairs),
                    "mk_div_kbit")
        return q, r

    # ---------------------------------------------------------------- measurement
    def timing_enable(self, on=True):
        self._check(self.L.mk_timing_enable(self.h, int(on)), "mk_timing_enable")

    def timing_reset(self):
        self._check(self.L.mk_timing_reset(self.h), "mk_timing_reset")

    def timing_read(self, kernel):
        """kernel: 0 = blind rotation (bootstrap), 1 = key switch -> (ms_total, launches)."""
        ms, n = ctypes.c_double(), ctypes.c_uint64()
        self._check(self.L.mk_timing_read(self.h, kernel, ctypes.byref(ms), ctypes.byref(n)), "mk_timing_read")
        return ms.value, n.value

    # ---------------------------------------------------------------- stages
    def stage_modswitch(self, lin, a, b, abar):
        self._check(self.L.mk_stage_modswitch(self.h, _dptr(lin), _dptr(a), _dptr(b), _dptr(abar), lin.shape[0]),
                    "mk_stage_modswitch")
        return abar

    def stage_blind_rotate(self, abar, max_steps, acc):
        self._check(self.L.mk_stage_blind_rotate(self.h, _dptr(abar), abar.numel() // self.W, max_steps,
                                                 _dptr(acc)), "mk_stage_blind_rotate")
        return acc

    def stage_bootstrap(self, lin, a, b, ext):
        self._check(self.L.mk_stage_bootstrap(self.h, _dptr(lin), _dptr(a), _dptr(b), _dptr(ext), lin.shape[0]),
                    "mk_stage_bootstrap")
        return ext

    def stage_keyswitch(self, ext, out):
        self._check(self.L.mk_stage_keyswitch(self.h, _dptr(ext), _dptr(out), ext.numel() // self.E),
                    "mk_stage_keyswitch")
        return out


class MkLin(ctypes.Structure):
    _fields_ = [("cst", ctypes.c_uint32), ("s1", ctypes.c_int32), ("s2", ctypes.c_int32)]


def gate_lin(gate_type, neg_a=False, neg_b=False):
    """(cst, s1, s2) of a bootstrapped gate type, from the library (mk_gate_lin)."""
    r = MkLin()
    rc = load().mk_gate_lin(int(gate_type), 1 if neg_a else 0, 1 if neg_b else 0, ctypes.byref(r))
    if rc != MK_OK:
        raise MkError("mk_gate_lin: %s" % ERRORS.get(rc, rc))
    return r.cst, r.s1, r.s2


def lin_records(types):
    """numpy int32 [count, 3] of (cst, s1, s2) for gate types (int array)."""
    table = {t: gate_lin(t) for t in set(int(t) for t in types)}
    out = np.zeros((len(types), 3), np.int32)
    for g, t in enumerate(types):
        cst, s1, s2 = table[int(t)]
        out[g] = (np.uint32(cst).view(np.int32), s1, s2)
    return out


def measure_butterfly_rate(device=0, stream=None, iters=4096, form="ntt"):
    """Butterflies per second on every SM: Goldilocks (form "ntt"), Harvey
    butterflies modulo a 28-bit prime ("ntt2"), complex FP64 butterflies
    ("fft") -- the pipe ceiling of each form; for "tc", multiply-accumulates
    per second of bf16 m16n8k16 MMAs."""
    r = ctypes.c_double()
    rc = load().mk_measure_butterfly_rate(device, ctypes.c_void_p(stream or 0), FORMS.get(form, form), iters,
                                          ctypes.byref(r))
    if rc != MK_OK:
        raise MkError("mk_measure_butterfly_rate: %s" % ERRORS.get(rc, rc))
    return r.value


def tc_negacyclic(keys, digits, out, device=0, stream=None, engine=0):
    """out[g] = sum_c keys[c] * digits[c][g] (negacyclic, mod 2^32) by the
    tensor-form product kernel (engine 0: mma.sync, 1: tcgen05).  keys:
    device uint32/int32 [nchunks][N]; digits: device int8 [nchunks][G][N];
    out: device int32 [G][N]."""
    nch, N = int(keys.shape[0]), int(keys.shape[1])
    G = int(digits.shape[1])
    rc = load().mk_tc_negacyclic(device, ctypes.c_void_p(stream or 0), N, G, nch, _dptr(keys), _dptr(digits),
                                 _dptr(out), engine)
    if rc != MK_OK:
        raise MkError("mk_tc_negacyclic: %s" % ERRORS.get(rc, rc))


OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3}


class MkGateRec(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint8), ("neg_a", ctypes.c_uint8), ("neg_b", ctypes.c_uint8),
                ("reserved", ctypes.c_uint8), ("a", ctypes.c_int32), ("b", ctypes.c_int32)]


def circuit_netlist(op, kbits, style="array"):
    """The library's netlist of an operator in a construction family as a
    dict (same shape as the oracle's): ka, kb, gates [(op, a, neg_a, b,
    neg_b)], outputs [(wire, neg)], levels."""
    L = load()
    ng, no, nl = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    opi = OPS[op] if isinstance(op, str) else int(op)
    st = CIRCUIT_STYLES[style] if isinstance(style, str) else int(style)
    rc = L.mk_circuit_netlist(opi, kbits, st, None, 0, ctypes.byref(ng), None, 0, ctypes.byref(no),
                              ctypes.byref(nl))
    if rc != MK_OK:
        raise MkError("mk_circuit_netlist: %s" % ERRORS.get(rc, rc))
    gates = (MkGateRec * max(ng.value, 1))()
    outs = (ctypes.c_int32 * max(no.value, 1))()
    rc = L.mk_circuit_netlist(opi, kbits, st, gates, ng.value, ctypes.byref(ng), outs, no.value,
                              ctypes.byref(no), ctypes.byref(nl))
    if rc != MK_OK:
        raise MkError("mk_circuit_netlist: %s" % ERRORS.get(rc, rc))
    return dict(ka=kbits, kb=kbits, gates=[(g.op, g.a, g.neg_a, g.b, g.neg_b) for g in gates[:ng.value]],
                outputs=[(o >> 1, o & 1) for o in outs[:no.value]], levels=nl.value)


class Server:
    """mk_server: continuous batching of operator requests on one context."""

    def __init__(self, ctx, wave_gates=4096, pool_rows=1 << 18):
        self.ctx = ctx
        h = VP()
        ctx._check(ctx.L.mk_server_create(ctx.h, wave_gates, pool_rows, ctypes.byref(h)), "mk_server_create")
        self.h = h
        self._keep = {}

    def close(self):
        if self.h:
            self.ctx.L.mk_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, op, kbits, a, b, out, out2=None):
        """a, b: CUDA tensors [pairs][kbits][W]; out (and out2 for div) receive the result."""
        t = ctypes.c_uint64()
        pairs = a.numel() // (kbits * self.ctx.W)
        opi = OPS[op] if isinstance(op, str) else int(op)
        self.ctx._check(self.ctx.L.mk_server_submit(self.h, opi, kbits, _dptr(a), _dptr(b), _dptr(out),
                                                    _dptr(out2) if out2 is not None else None, pairs,
                                                    ctypes.byref(t)), "mk_server_submit")
        self._keep[t.value] = (a, b, out, out2)
        return t.value

    def step(self):
        n = ctypes.c_uint32()
        self.ctx._check(self.ctx.L.mk_server_step(self.h, ctypes.byref(n)), "mk_server_step")
        return n.value

    def poll(self, ticket):
        st = ctypes.c_int()
        self.ctx._check(self.ctx.L.mk_server_poll(self.h, ticket, ctypes.byref(st)), "mk_server_poll")
        return st.value

    def stats(self):
        w, g = ctypes.c_uint64(), ctypes.c_uint64()
        r, q = ctypes.c_uint32(), ctypes.c_uint32()
        self.ctx._check(self.ctx.L.mk_server_stats(self.h, ctypes.byref(w), ctypes.byref(g), ctypes.byref(r),
                                                   ctypes.byref(q)), "mk_server_stats")
        return dict(waves=w.value, gates=g.value, running=r.value, queued=q.value)

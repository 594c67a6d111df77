"""Benchmark: multi-key bootstrapped gates per second on one GB300.

Workload (full-size, 2 parties): n = 560, N = 1024, gadget base 2^8 with
d = 3, key-switching base 2^2 with t = 8, LWE sigma 2^-15; 4096 independent
gates per step, gate type and input bits uniform (seeded); c1 encrypted by
party 0 and c2 by party 1, so every CMux step of the blind rotation is active.
One step = the whole hot path over the batch: linear part, modulus switch,
blind rotation (exact NTT form), SampleExtract, key switch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain schoolbook implementation)
on the host cores over a bounded sample of the same workload.  Under torchrun
every rank runs its own 4096-gate batch on its own GPU (weak scaling, no
collective on the data path); rank 0 prints one JSON line.

Besides the timed k = 2 steps the line carries, measured after them: the
four-party half of the metric ("k4": batched gates/s over several batches,
p50/p99, the one-gate-per-launch rate and the blind rotation's roofline) and
bounded summaries of the other configurations -- the precision sweep
(512 joint-key gates per party count and product form), the regression
application (shallow netlists), the k-bit operators (8-bit throughput,
16-bit single-pair latency, both netlist families), Table 2's gates (each
gate directly and composed of bootstrapped NANDs) and the serving loop
(k = 4, 16-bit requests, a closed batch and Poisson arrivals at 0.5 and 0.9
of its capacity, with the array and the shallow netlists).  --sweep,
--regression and --operators run the full versions; --no-extras leaves the
summaries out.  The end-to-end figure ("e2e") times the same K steps through
the public API with the inputs copied from pinned host memory and the
outputs read back inside the timed region.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MK bootstrapped gates/sec (2 and 4 parties, N=1024); p50/p99 gate latency"
UNIT = "gates/s"
WORKLOAD = "full-size MK gate bootstrap, k=2 parties, n=560, N=1024, 4096 random gates per step"


# ----------------------------------------------------------------------------- distributed helpers
def dist_env():
    """(rank, world size, local rank): the library's replica helper."""
    from paper_2205_05825_gb300.replicas import dist_env as env
    return env()


def shard_seed(config_id, rank):
    """Each rank draws its own batch of gates (independent units, weak scaling)."""
    return config_id * 100 + rank


def reduce_max(value, world):
    """Max over ranks (time of the slowest rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            return None
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- roofline bookkeeping
def work_per_cmux(P, form="ntt"):
    """Algorithmic work of one CMux step, in the unit of the form's ceiling.
    Tensor form: FLOPs of the dense products -- (2k+4) d Toeplitz products
    per step, each 4 byte planes x N^2 multiply-accumulates.
    NTT forms: modular multiplies -- (k+2)(d+1) length-N transforms of
    (N/2) log2 N butterflies plus (2k+4) d N pointwise products (hybrid
    product, phase A and B), once per prime.  FFT form: FP64 instructions
    (an FMA counts one) -- 8 per complex butterfly, 4 per complex twist of
    each transformed point and 4 per pointwise complex multiply-add, on
    M = N/2 folded points."""
    k, d, N = P["k"], P["d"], P["N"]
    logn = N.bit_length() - 1
    if form == "tc":  # FLOPs (2 per multiply-accumulate) of the dense Toeplitz products, 4 byte planes
        return 2 * (2 * (k + 1) * d + 2 * d) * 4 * N * N
    if form == "fft":
        M = N // 2
        return (k + 2) * (d + 1) * ((M // 2) * (logn - 1) * 8 + M * 4) + (2 * k + 4) * d * M * 4
    per_prime = (k + 2) * (d + 1) * (N // 2) * logn + (2 * k + 4) * d * N
    return per_prime * (2 if form == "ntt2" else 1)


# Work units per measured butterfly of the ceiling microbenchmark.
UNITS_PER_BUTTERFLY = {"ntt": 1, "ntt2": 1, "fft": 8, "tc": 2}
UNIT_NAME = {"ntt": "G modmul/s", "ntt2": "G modmul/s", "fft": "G FP64 instr/s", "tc": "TFLOP/s"}
FORM_DESC = {"ntt": "ntt64 (exact, Goldilocks prime)",
             "ntt2": "ntt2x28 (exact, two 28-bit primes + CRT)",
             "fft": "fft64 (FP64, rounded; approximate)",
             "tc": "tc-bf16 (exact, tensor-core Toeplitz products of key byte planes)"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def kernel_source_hash():
    """Hash of the blind-rotation kernel's code with comments and whitespace
    removed, so that an edit of its comments keeps a capture valid."""
    h = hashlib.sha256()
    for f in ("mk_bootstrap.cuh", "mk_br.cu"):
        src = open(os.path.join(ROOT, "paper_2205_05825_gb300", "csrc", f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic_per_gate():
    """DRAM bytes per gate of the blind-rotation kernel from the committed ncu
    summary, or None when the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "bootstrap_ntt_k2_n1024_traffic.txt")
    try:
        kv = dict(line.split(":", 1) for line in open(path) if ":" in line)
    except OSError:
        return None
    if kv.get("kernel_source_sha256_16", "").strip() != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_gate"].strip())
    except (KeyError, ValueError):
        return None


# ----------------------------------------------------------------------------- regression application
def run_regression(dev_index, styles=("array", "shallow")):
    """Training and evaluation times of the encrypted linear regression at
    the full parameter set, k = 2: x encrypted by party 0, y by party 1, m = 8
    points on y = 2x + 1 (Sec. 5.5, Table 8), with each operator netlist
    family (MK_CIRCUIT_ARRAY, MK_CIRCUIT_SHALLOW).  Algorithm 7 at 8 bits
    trains from scratch; Algorithm 8 at 16 bits (zoom 100, learning rate
    1/16) times one iteration started at the exact zoomed solution, where
    both updates are zero.  The exact data make the expected models known
    without the oracle: (omega, b) = (2, 1), (W, B) unchanged, losses 0.
    Wall-clock seconds with the device synchronised on both sides of each
    phase."""
    import torch

    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import regression as G
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(2)
    ctx = B.Context(P, W.CRS_SEED, device=dev_index)
    for i, s_ in enumerate(W.party_seeds(2)):
        ctx.keygen(i, s_)
    xs = [-3, -2, -1, 0, 1, 2, 3, 0]          # sum 0: the mean is exact; nothing wraps at 8 bits
    ys = [2 * x + 1 for x in xs]
    dev = "cuda:%d" % dev_index

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    dec = lambda ct: int(G.decrypt_integers(ctx, ct)[0])  # noqa: E731
    out = {"parties": 2, "m": len(xs)}
    for style in styles:
        ctx.set_circuit_style(style)
        cx = G.encrypt_integers(ctx, xs, 8, 0, W.encryption_seed(70, 0), device=dev)
        cy = G.encrypt_integers(ctx, ys, 8, 1, W.encryption_seed(70, 1), device=dev)
        (om, b, calls), t_train = timed(lambda: G.closed_form(ctx, 8, cx, cy))
        (loss, _), t_eval = timed(lambda: G.loss_closed_form(ctx, 8, cx, cy, om, b))
        cf = {"kbits": 8, "train_s": t_train, "eval_s": t_eval, "operator_calls": calls,
              "model": [dec(om), dec(b)], "loss": dec(loss)}
        cf["ok"] = cf["model"] == [2, 1] and cf["loss"] == 0
        n = 100
        cx = G.encrypt_integers(ctx, xs, 16, 0, W.encryption_seed(71, 0), device=dev)
        cy = G.encrypt_integers(ctx, ys, 16, 1, W.encryption_seed(71, 1), device=dev)
        (Wc, Bc, calls), t_iter = timed(lambda: G.gradient_descent(ctx, 16, cx, cy, n, 1, 16, 1, w0=2 * n, b0=n))
        (loss, _), t_eval = timed(lambda: G.loss_gradient_descent(ctx, 16, cx, cy, Wc, Bc, n))
        gd = {"kbits": 16, "zoom": n, "learning_rate": "1/16", "train_s_per_iter": t_iter, "eval_s": t_eval,
              "operator_calls": calls, "model": [dec(Wc), dec(Bc)], "loss": dec(loss)}
        gd["ok"] = gd["model"] == [2 * n, n] and gd["loss"] == 0
        out[style] = {"closed_form": cf, "gradient_descent": gd}
    ctx.close()
    out["paper_table8_k2"] = {"formula_train_s": 227.467, "formula_eval_s": 37.131, "gd_train_s_per_iter": 1133.33,
                              "gd_eval_s": 190.644, "note": "Xeon Gold 5220 CPU; the paper does not state its data size"}
    return out


# ----------------------------------------------------------------------------- operators (config 3)
def run_operators(dev_index, full=False):
    """k-bit operators (Alg. 3-6) at the full parameter set, k = 2 (and k = 4
    with full=True).  Default (bounded): throughput of 8-bit add and multiply
    over 64 pairs (array netlists), and the latency of one pair of each
    16-bit operator with both netlist families.  full=True: the config-3
    table, every operator at 8 and 16 bits over 256 pairs: k = 2 with both
    families, k = 4 with the array family.  Wall-clock seconds with the device synchronised on both sides;
    every output decrypted against native two's-complement arithmetic."""
    import torch

    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    dev = "cuda:%d" % dev_index
    if full:
        cases = [(k, style, op, bits, 256) for k, style in ((2, "array"), (2, "shallow"), (4, "array"))
                 for bits in (8, 16) for op in ("add", "sub", "mul", "div")]
    else:
        cases = ([(2, "array", op, 8, 64) for op in ("add", "mul")] +
                 [(2, style, op, 16, 1) for style in ("array", "shallow") for op in ("add", "sub", "mul", "div")])
    out = []
    ctxs = {}
    for k, style, op, bits, pairs in cases:
        if k not in ctxs:
            for c_ in ctxs.values():
                c_.close()
            ctxs = {}
            P = W.full_params(k)
            ctx = B.Context(P, W.CRS_SEED, device=dev_index)
            for i, s_ in enumerate(W.party_seeds(k)):
                ctx.keygen(i, s_)
            ctx.autotune(1024)
            ctxs[k] = ctx
        ctx = ctxs[k]
        ctx.set_circuit_style(style)
        a, b = W.random_operands(bits, pairs, config_id=3)
        if op == "div":
            b = np.where(b == 0, 1, b)
        ca = ctx.encrypt(0, W.int_to_bits(a, bits).ravel(), W.encryption_seed(80, 0)).reshape(pairs, bits, -1)
        cb = ctx.encrypt(1, W.int_to_bits(b, bits).ravel(), W.encryption_seed(80, 1)).reshape(pairs, bits, -1)
        da = torch.from_numpy(ca.view(np.int32)).to(dev)
        db = torch.from_numpy(cb.view(np.int32)).to(dev)
        nout = 2 * bits if op == "mul" else bits
        o1 = torch.zeros((pairs, nout, ctx.W), dtype=torch.int32, device=dev)
        o2 = torch.zeros((pairs, bits, ctx.W), dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if op == "div":
            ctx.div_kbit(bits, da, db, o1, o2)
        else:
            getattr(ctx, op + "_kbit")(bits, da, db, o1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        got = W.bits_to_int(ctx.decrypt(o1).reshape(pairs, -1))
        if op == "div":
            r = W.bits_to_int(ctx.decrypt(o2).reshape(pairs, -1))
            exp = [W.expected_result(op, int(x), int(y), bits) for x, y in zip(a, b)]
            ok = all((int(q), int(rr)) == e for q, rr, e, x, y in zip(got, r, exp, a, b)
                     if not (x == -(1 << (bits - 1)) and y == -1))
        else:
            ok = all(int(g) == W.expected_result(op, int(x), int(y), bits) for g, x, y in zip(got, a, b))
        net = B.circuit_netlist(op, bits, style)
        gates = len(net["gates"]) * pairs
        out.append({"parties": k, "style": style, "op": op, "bits": bits, "pairs": pairs, "netlist_gates":
                    len(net["gates"]), "levels": net["levels"], "seconds": dt, "gates_per_s": gates / dt,
                    "s_per_level": dt / max(net["levels"], 1), "decrypt_ok": bool(ok)})
        ctx.set_circuit_style("array")
    for c_ in ctxs.values():
        c_.close()
    return out


def run_sweep(dev_index, gates, forms, parties=(2, 4, 8), autotune=True):
    """Precision sweep (config 4): gates/s of each product form at 2, 4 and 8
    parties, joint-key inputs (all k n CMux steps run), every output
    decrypted."""
    import torch

    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    out = []
    for kk in parties:
        Pk = W.full_params(kk)
        ck = B.Context(Pk, W.CRS_SEED, device=dev_index)
        for i, s_ in enumerate(W.party_seeds(kk)):
            ck.keygen(i, s_)
        ts, x1, x2 = W.random_gates(gates, config_id=40 + kk)
        e1 = ck.encrypt_joint(x1, W.encryption_seed(40 + kk, 0))
        e2 = ck.encrypt_joint(x2, W.encryption_seed(40 + kk, 1))
        tr = np.array([[a & b, a | b, 1 - (a & b), 1 - (a | b), a ^ b, 1 - (a ^ b)][t]
                       for t, a, b in zip(ts, x1.astype(int), x2.astype(int))], np.uint8)
        cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32  # noqa: E731
                                          else np.ascontiguousarray(a)).cuda()
        dt_, d1, d2 = cuda(ts.astype(np.uint8)), cuda(e1), cuda(e2)
        do = torch.zeros((gates, ck.W), dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        for form in forms:
            Gf = gates if form != "tc" else min(gates, 2048)  # the O(N^2) form: at most one 2048-gate wave
            ck.set_form(form)
            if autotune:
                ck.autotune(1024)
            else:
                ck.set_variant(1 if form == "tc" else 2)
            ck.gates(dt_[:Gf], d1[:Gf], d2[:Gf], do[:Gf])
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            ck.gates(dt_[:Gf], d1[:Gf], d2[:Gf], do[:Gf])
            s1.record(stream)
            torch.cuda.synchronize()
            ms = s0.elapsed_time(s1)
            out.append({"parties": kk, "form": form, "gates": Gf, "gates_per_s": Gf / (ms * 1e-3),
                        "decrypt_ok": bool(np.array_equal(ck.decrypt(do[:Gf]), tr[:Gf])),
                        "active_cmux_steps_per_gate": kk * Pk["n"]})
        ck.close()
    return out


def run_table2(dev_index, batch=4096):
    """Table 2's comparison on the GPU (full size, k = 2): each gate evaluated
    directly (one bootstrap; NOT is linear) and as the naive scheme composes
    it from bootstrapped NANDs alone (NOT = NAND(x, x); AND 2, OR 3, NOR 4,
    XOR 4, XNOR 5 NANDs, in 2-4 dependent steps).  Per gate type: the
    latency of one gate and the time per gate in a batch of `batch` gates
    (each NAND step one batched launch), CUDA events on the stream; every
    output decrypted against the truth table."""
    import torch

    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(2)
    ctx = B.Context(P, W.CRS_SEED, device=dev_index)
    for i, s_ in enumerate(W.party_seeds(2)):
        ctx.keygen(i, s_)
    ctx.autotune(1024)
    dev = "cuda:%d" % dev_index
    _, b1, b2 = W.random_gates(batch, config_id=77)
    A = torch.from_numpy(ctx.encrypt(0, b1, W.encryption_seed(77, 0)).view(np.int32)).to(dev)
    Bc = torch.from_numpy(ctx.encrypt(1, b2, W.encryption_seed(77, 1)).view(np.int32)).to(dev)
    names = ["AND", "OR", "NAND", "NOR", "XOR", "XNOR", "NOT"]
    truth = {"AND": b1 & b2, "OR": b1 | b2, "NAND": 1 - (b1 & b2), "NOR": 1 - (b1 | b2), "XOR": b1 ^ b2,
             "XNOR": 1 - (b1 ^ b2), "NOT": 1 - b1}
    # NAND steps of the naive scheme: (destination, first input, second input)
    recipe = {"AND": [("n", "a", "b"), ("r", "n", "n")],
              "OR": [("x", "a", "a"), ("y", "b", "b"), ("r", "x", "y")],
              "NAND": [("r", "a", "b")],
              "NOR": [("x", "a", "a"), ("y", "b", "b"), ("o", "x", "y"), ("r", "o", "o")],
              "XOR": [("n", "a", "b"), ("x", "a", "n"), ("y", "b", "n"), ("r", "x", "y")],
              "XNOR": [("n", "a", "b"), ("x", "a", "n"), ("y", "b", "n"), ("o", "x", "y"), ("r", "o", "o")],
              "NOT": [("r", "a", "a")]}
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()  # warm-up (plans, scratch)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) * 1e-3

    rows = []
    for name in names:
        t = names.index(name)
        res = {"gate": name, "nand_gates": len(recipe[name])}
        for g in (1, batch):
            a, b = A[:g].contiguous(), Bc[:g].contiguous()

            def direct():
                o = torch.zeros_like(a)
                if name == "NOT":
                    ctx.mk_not(a, o)
                else:
                    ctx.gate(t, a, b, o)
                return o

            def naive():
                w = {"a": a, "b": b}
                for dst, x, y in recipe[name]:
                    w[dst] = torch.zeros_like(a)
                    ctx.gate(2, w[x], w[y], w[dst])
                return w["r"]

            od, td = timed(direct)
            on, tn = timed(naive)
            ok = (np.array_equal(ctx.decrypt(od), truth[name][:g]) and
                  np.array_equal(ctx.decrypt(on), truth[name][:g]))
            key = "latency_s" if g == 1 else "s_per_gate_in_batch"
            res[key] = {"ours": td / g, "naive": tn / g}
            res.setdefault("decrypt_ok", True)
            res["decrypt_ok"] = res["decrypt_ok"] and bool(ok)
        rows.append(res)
    ctx.close()
    paper = {"AND": (0.238671, 0.238008), "OR": (0.584701, 0.23558), "NOT": (0.236541, 2e-06),
             "NAND": (0.235327, 0.239638), "NOR": (0.470561, 0.236153), "XOR": (0.71246, 0.2354),
             "XNOR": (0.710777, 0.23588)}
    for r in rows:
        r["paper_table2_s"] = {"naive": paper[r["gate"]][0], "ours": paper[r["gate"]][1],
                               "note": "one gate at a time, MKTFHE on a Xeon Gold 5220, k = 2"}
    return {"parties": 2, "batch": batch, "gates": rows}


def guarded(fn):
    """Run an optional part of the report; its failure is recorded, not fatal."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001
        return {"error": "%s: %s" % (type(e).__name__, e)}


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    B.load(build_if_missing=True)

    def setup(k, G):
        """k = 2: c1 by party 0, c2 by party 1 (every CMux step active).  k > 2:
        joint-key inputs (every party block non-zero, as for the outputs of
        earlier gates inside a circuit), so all k*n CMux steps run."""
        P = W.full_params(k)
        ctx = B.Context(P, W.CRS_SEED, device=dev_index)
        for i, s in enumerate(W.party_seeds(k)):
            ctx.keygen(i, s)
        cfg = shard_seed(2, rank)
        types, b1, b2 = W.random_gates(G, config_id=cfg)
        if k == 2:
            c1 = ctx.encrypt(0, b1, W.encryption_seed(cfg, 0))
            c2 = ctx.encrypt(1, b2, W.encryption_seed(cfg, 1))
        else:
            c1 = ctx.encrypt_joint(b1, W.encryption_seed(cfg, 0))
            c2 = ctx.encrypt_joint(b2, W.encryption_seed(cfg, 1))
        truth = np.array([[a & b, a | b, 1 - (a & b), 1 - (a | b), a ^ b, 1 - (a ^ b)][t]
                          for t, a, b in zip(types, b1.astype(int), b2.astype(int))], np.uint8)
        return P, ctx, types, c1, c2, truth

    G = args.gates
    P, ctx, types, c1, c2, truth = setup(2, G)
    tdev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32) if a.dtype == np.uint32
                                      else np.ascontiguousarray(a)).cuda()
    d_types, d_c1, d_c2 = tdev(types.astype(np.uint8)), tdev(c1), tdev(c2)
    d_out = torch.zeros((G, ctx.W), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    # product form, then autotune the blind-rotation variant on a sample of random ciphertexts
    form_ms = None
    if args.form == "auto":  # the product-form autotuner over the exact forms
        args.form, form_ms = ctx.autotune_form(min(args.autotune_gates, G), forms=("ntt", "ntt2", "tc"))
    ctx.set_form(args.form)
    if args.variant >= 0:
        ctx.set_variant(args.variant)
        variant, variant_ms = args.variant, None
    else:
        variant, variant_ms = ctx.autotune(min(args.autotune_gates, G))

    # warm-up (also uploads the keys)
    for _ in range(args.warmup):
        ctx.gates(d_types, d_c1, d_c2, d_out)
    torch.cuda.synchronize()
    ok = np.array_equal(ctx.decrypt(d_out), truth)

    # timed region: exactly K steps, barrier + sync on both sides
    clocks = ClockSampler(dev_index)
    clocks.start()
    ctx.timing_enable(True)
    ctx.timing_reset()
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(args.steps):
        step_ev[s][0].record(stream)
        ctx.gates(d_types, d_c1, d_c2, d_out)
        step_ev[s][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    br_ms, br_n = ctx.timing_read(0)
    ks_ms, ks_n = ctx.timing_read(1)
    ctx.timing_enable(False)
    clk = clocks.stop()
    total_ms = sum(step_ms)
    total_ms_max = reduce_max(total_ms, world)
    value = G * args.steps * world / (total_ms_max * 1e-3)
    launches_per_step = 3 * ((G + 4095) // 4096)

    # end to end through the public API with host buffers (pinned), copies inside
    h_types = torch.from_numpy(types.astype(np.uint8)).pin_memory()
    h_c1 = torch.from_numpy(c1.view(np.int32)).pin_memory()
    h_c2 = torch.from_numpy(c2.view(np.int32)).pin_memory()
    h_out = torch.empty((G, ctx.W), dtype=torch.int32).pin_memory()
    e2e_steps = args.steps  # the same K steps as the device-timed value
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        d_types.copy_(h_types, non_blocking=True)
        d_c1.copy_(h_c1, non_blocking=True)
        d_c2.copy_(h_c2, non_blocking=True)
        ctx.gates(d_types, d_c1, d_c2, d_out)
        h_out.copy_(d_out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1), world)
    e2e_value = G * e2e_steps * world / (e2e_ms * 1e-3)
    ok = ok and np.array_equal(ctx.decrypt(h_out.numpy().view(np.uint32)), truth)

    # one-gate-per-launch form (the plain denominator), a few gates
    plain_g = args.plain_gates
    ctx.set_batch(1)
    ctx.gates(d_types[:1], d_c1[:1], d_c2[:1], d_out[:1])
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    ctx.gates(d_types[:plain_g].contiguous(), d_c1[:plain_g].contiguous(), d_c2[:plain_g].contiguous(),
              d_out[:plain_g])
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    plain_rate = plain_g / (plain_ms * 1e-3)
    ctx.set_batch(4096)

    scale = 1e12 if args.form == "tc" else 1e9
    ceiling = (B.measure_butterfly_rate(dev_index, stream.cuda_stream, iters=2048, form=args.form) / scale
               * UNITS_PER_BUTTERFLY[args.form])

    # k = 4 parties (second half of the metric): several timed batches, the
    # blind rotation's roofline, and the one-gate-per-launch form
    k4 = None
    if args.k4_gates > 0:
        G4 = args.k4_gates
        P4, ctx4, t4, a4, b4, tr4 = setup(4, G4)
        ctx4.set_form(args.form)
        v4, _ = ctx4.autotune(min(args.autotune_gates, G4))
        dt4, da4, db4 = tdev(t4.astype(np.uint8)), tdev(a4), tdev(b4)
        do4 = torch.zeros((G4, ctx4.W), dtype=torch.int32, device="cuda")
        ctx4.gates(dt4, da4, db4, do4)
        torch.cuda.synchronize()
        k4_steps = max(3, min(args.steps, 5))
        ev4 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k4_steps)]
        ctx4.timing_enable(True)
        ctx4.timing_reset()
        for e_a, e_b in ev4:
            e_a.record(stream)
            ctx4.gates(dt4, da4, db4, do4)
            e_b.record(stream)
        torch.cuda.synchronize()
        ms4 = sorted(a_.elapsed_time(b_) for a_, b_ in ev4)
        br4_ms, br4_n = ctx4.timing_read(0)
        ctx4.timing_enable(False)
        k4_ok = bool(np.array_equal(ctx4.decrypt(do4), tr4))
        rate4 = G4 * len(ms4) / (sum(ms4) * 1e-3)
        ctx4.set_batch(1)
        ctx4.gates(dt4[:1], da4[:1], db4[:1], do4[:1])
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        ctx4.gates(dt4[:plain_g].contiguous(), da4[:plain_g].contiguous(), db4[:plain_g].contiguous(),
                   do4[:plain_g])
        p1.record(stream)
        torch.cuda.synchronize()
        plain4_ms = p0.elapsed_time(p1)
        plain4 = plain_g / (plain4_ms * 1e-3)
        ctx4.set_batch(4096)
        work4 = work_per_cmux(P4, args.form) * P4["k"] * P4["n"]
        ach4 = G4 * work4 / (br4_ms / max(br4_n, 1) * 1e-3) / scale
        k4 = {"gates_per_s": rate4, "gates": G4, "steps": len(ms4), "ms_per_batch": float(np.mean(ms4)),
              "latency_ms": {"p50": float(np.percentile(ms4, 50)), "p99": float(np.percentile(ms4, 99))},
              "decrypt_ok": k4_ok, "active_cmux_steps_per_gate": 4 * P4["n"], "inputs": "joint-key",
              "sigma_rlwe": P4["sigma_rlwe"], "variant": v4,
              "plain_one_gate_per_launch": {"gates_per_s": plain4, "gates": plain_g,
                                            "latency_ms": plain4_ms / plain_g, "batched_over_plain": rate4 / plain4},
              "roofline": {"bound": "tensor" if args.form == "tc" else "alu", "achieved": ach4, "peak": ceiling,
                           "unit": UNIT_NAME[args.form], "frac": ach4 / ceiling,
                           "algorithmic_work_per_gate": work4, "br_share_of_step": br4_ms / sum(ms4)}}
        ctx4.close()

    # Bounded summaries of the other configurations, outside the timed region
    # (--no-extras leaves them out; --sweep / --regression / --operators run
    # the full versions).
    extras = not args.no_extras
    sweep = None
    if args.sweep:
        sweep = guarded(lambda: run_sweep(dev_index, 8192, args.sweep_forms.split(",")))
    elif extras:
        sweep = guarded(lambda: run_sweep(dev_index, 512, ("ntt2", "tc", "fft"), autotune=False))
    regression = None
    if args.regression:
        regression = guarded(lambda: run_regression(dev_index))
    elif extras:
        regression = guarded(lambda: run_regression(dev_index, styles=("shallow",)))
    operators = None
    if args.operators or extras:
        operators = guarded(lambda: run_operators(dev_index, full=args.operators))
    table2 = guarded(lambda: run_table2(dev_index)) if extras else None
    serving = None
    if extras:
        from paper_2205_05825_gb300.serving import run_serving
        serving = {style: guarded(lambda style=style: run_serving(
                       parties=4, bits=16, capacity_requests=48, requests=24, loads=(0.5, 0.9), device=dev_index,
                       circuit_style=style)) for style in ("array", "shallow")}

    # roofline of the dominant kernel (blind rotation), live from the timed region
    avg_br_ms = br_ms / max(br_n, 1)
    mm_per_gate = work_per_cmux(P, args.form) * P["k"] * P["n"]
    achieved = G * mm_per_gate / (avg_br_ms * 1e-3) / scale
    traffic_pg = ncu_traffic_per_gate() if args.form == "ntt2" else None
    if args.form == "tc":
        mp = measured_peaks()
        peak = mp["bf16_tflops_sustained"] if mp else 1700.0
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "blind rotation, tensor form (tc_products_kernel + digit kernels)",
                    "algorithmic_work_per_gate": mm_per_gate,
                    "peak_source": ("measured bf16 dense GEMM, sustained (MEASURED_PEAKS.json)" if mp
                                    else "fallback 1.7 PFLOP/s sustained"),
                    "mma_sync_ceiling_tflops": ceiling,
                    "frac_of_mma_sync_ceiling": achieved / ceiling,
                    "br_share_of_step": br_ms / total_ms if total_ms else None}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": ceiling, "unit": UNIT_NAME[args.form],
                    "frac": achieved / ceiling, "traffic": (traffic_pg * G if traffic_pg is not None else None),
                    "kernel": "bootstrap_ntt_kernel<%s, 10, variant %d>" % (args.form, variant),
                    "algorithmic_work_per_gate": mm_per_gate,
                    "peak_source": ("measured: register-resident butterfly loop of the same arithmetic on every "
                                    "SM (mk_measure_butterfly_rate, %s)"
                                    % {"ntt": "Goldilocks 64-bit, one modmul per butterfly",
                                       "ntt2": "Harvey/Shoup mod a 28-bit prime, one modmul per butterfly",
                                       "fft": "complex FP64, 8 FP64 instructions per butterfly"}[args.form]),
                    "br_share_of_step": br_ms / total_ms if total_ms else None}

    ctx.close()
    if rank != 0:
        return
    sm = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parties": 2, "gates_per_step": G, "n": P["n"], "N": P["N"],
                   "bg_bit": P["bg_bit"], "d": P["d"], "ks_bit": P["ks_bit"], "t": P["t"],
                   "sigma_lwe": P["sigma_lwe"], "sigma_rlwe": P["sigma_rlwe"],
                   "form": FORM_DESC[args.form],
                   "variant": variant, "autotune_ms": variant_ms, "form_autotune_ms": form_ms,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "no flush: per-step working set (BK 82 MB NTT domain + KS 110 MB + 37 MB "
                         "ciphertexts) exceeds the 129 MB L2"},
        "latency_ms": {"p50": float(np.percentile(sm, 50)), "p99": float(np.percentile(sm, 99)),
                       "note": "every gate of a batched launch completes with its batch"},
        "plain_one_gate_per_launch": {"gates_per_s": plain_rate, "gates": plain_g,
                                      "latency_ms": plain_ms / plain_g,
                                      "batched_over_plain": value / world / plain_rate},
        "negacyclic_products_per_s": {
            "value": value * P["k"] * P["n"] * (2 * P["k"] + 4) * P["d"],
            "per_gate": P["k"] * P["n"] * (2 * P["k"] + 4) * P["d"],
            "note": "form-independent rate: k n (2k+4) d length-N negacyclic products per gate"},
        "k4": k4,
        "precision_sweep": sweep,
        "regression": regression,
        "operators": operators,
        "table2_gates": table2,
        "serving": serving,
        "decrypt_ok": bool(ok),
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(G + 2 * G * ctx.W * 4),
                "d2h_bytes_per_step": int(G * ctx.W * 4), "steps": e2e_steps},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline,
        "wall_s": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- oracle (CPU)
def _oracle_setup():
    from oracle import oracle as o
    from paper_2205_05825_gb300 import workloads as W
    P = W.full_params(2)
    return o, W, P, o.keygen(P, W.CRS_SEED, W.party_seeds(2))


def _oracle_step(o, W, P, keys, sample, cores):
    types, b1, b2 = W.random_gates(sample, config_id=shard_seed(2, 0))
    c1 = o.encrypt(P, keys, 0, b1, W.encryption_seed(2, 0))
    c2 = o.encrypt(P, keys, 1, b2, W.encryption_seed(2, 1))
    t0 = time.perf_counter()
    out = o.gates(P, keys, types, c1, c2, nthreads=cores)
    dt = time.perf_counter() - t0
    truth = np.array([[a & b, a | b, 1 - (a & b), 1 - (a | b), a ^ b, 1 - (a ^ b)][t]
                      for t, a, b in zip(types, b1.astype(int), b2.astype(int))], np.uint8)
    return dt, bool(np.array_equal(o.decrypt(P, keys, out), truth))


def cpu_baseline(args):
    """The oracle as it stands, OpenMP across gates on the host cores, over a
    bounded sample of the workload (gates/s extrapolated from the sample)."""
    o, W, P, keys = _oracle_setup()
    cores = o.default_threads()
    sample = max(cores, args.cpu_sample)
    dt, ok = _oracle_step(o, W, P, keys, sample, cores)
    return {"value": sample / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d gates of the same workload (k=2, n=560, N=1024), schoolbook products, "
                      "OpenMP across gates, %.1f s" % (sample, dt), "decrypt_ok": ok}


def run_reference(args):
    """Reference arm: the oracle timed on the host cores; each step is a bounded
    sample (one gate per core) of the 4096-gate workload."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    o, W, P, keys = _oracle_setup()
    cores = o.default_threads()
    sample = cores
    for _ in range(args.warmup):
        _oracle_step(o, W, P, keys, 1, 1)
    times, oks = [], []
    for _ in range(args.steps):
        dt, ok = _oracle_step(o, W, P, keys, sample, cores)
        times.append(dt)
        oks.append(ok)
    value = sample * len(times) / sum(times)
    desc = ("%d gates per step (one per core) of the same workload (k=2, n=560, N=1024), schoolbook "
            "products, OpenMP across gates" % sample)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parties": 2, "n": 560, "N": 1024, "form": "schoolbook (oracle)",
                       "gates_per_step": sample},
            "impl": "reference", "decrypt_ok": all(oks),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--gates", type=int, default=4096)
    ap.add_argument("--plain-gates", type=int, default=4)
    ap.add_argument("--k4-gates", type=int, default=4096)
    ap.add_argument("--cpu-sample", type=int, default=16)
    ap.add_argument("--autotune-gates", type=int, default=2048)
    ap.add_argument("--form", default="auto", choices=["auto", "ntt", "ntt2", "fft", "tc"],
                    help="product form; auto = the library's form autotuner over the exact forms")
    ap.add_argument("--variant", type=int, default=-1,
                    help="blind-rotation variant to use instead of autotuning (-1: autotune)")
    ap.add_argument("--sweep", action="store_true",
                    help="also time every product form at 2, 4 and 8 parties (8192 joint-key gates each)")
    ap.add_argument("--sweep-forms", default="ntt,ntt2,fft,tc",
                    help="comma-separated product forms the sweep times")
    ap.add_argument("--regression", action="store_true",
                    help="also time the encrypted linear regression (Algorithms 7 and 8) at k = 2, full size")
    ap.add_argument("--operators", action="store_true",
                    help="also time the config-3 operator table (every operator, 8 and 16 bits, 256 pairs; "
                         "k = 2 with both netlist families, k = 4 with the array family)")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the bounded sweep, regression, operator and serving summaries")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

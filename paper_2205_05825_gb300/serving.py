"""Serving driver: encrypted operator requests from several clients through
the library's continuous-batching server (mk_server_*), with Poisson
arrivals.  Reports throughput and p50/p99 request latency.

  python -m paper_2205_05825_gb300.serving [--parties 4] [--bits 16] ...

Every request is one k-bit operation on one operand pair, its operands
encrypted by two of the parties; results are checked by decryption against
native two's-complement arithmetic.
"""
import argparse
import json
import time

import numpy as np

from . import binding as B
from . import workloads as W


class Client:
    """Encrypts request operands (as their owning parties would) and keeps
    the device buffers of each request."""

    def __init__(self, ctx, bits):
        import torch
        self.ctx, self.bits, self.torch = ctx, bits, torch
        self.k = ctx.params["k"]

    def prepare(self, idx, op, a, b):
        torch = self.torch
        bits = self.bits
        pa, pb = idx % self.k, (idx + 1) % self.k
        ca = self.ctx.encrypt(pa, W.int_to_bits([a], bits).ravel(), W.encryption_seed(5, pa, idx % 4096))
        cb = self.ctx.encrypt(pb, W.int_to_bits([b], bits).ravel(), W.encryption_seed(5, pb, 4096 + idx % 4096))
        dev = lambda x: torch.from_numpy(x.reshape(1, bits, -1).view(np.int32)).cuda()
        nout = 2 * bits if op == "mul" else bits
        out = torch.zeros((1, nout, self.ctx.W), dtype=torch.int32, device="cuda")
        out2 = torch.zeros((1, bits, self.ctx.W), dtype=torch.int32, device="cuda") if op == "div" else None
        return dict(op=op, a=a, b=b, da=dev(ca), db=dev(cb), out=out, out2=out2)

    def result(self, req):
        bits = self.ctx.decrypt(req["out"]).reshape(1, -1)
        v = int(W.bits_to_int(bits)[0])
        if req["op"] != "div":
            return v
        r = int(W.bits_to_int(self.ctx.decrypt(req["out2"]).reshape(1, -1))[0])
        return v, r


def run_stream(server, client, reqs, arrivals=None):
    """Submit requests as their arrival times pass (all at once if arrivals is
    None) and step the server until all are done.  Returns per-request
    latency (s) and the wall time."""
    t0 = time.perf_counter()
    n = len(reqs)
    arrivals = np.zeros(n) if arrivals is None else np.asarray(arrivals)
    tickets, submit_t, done_t = [None] * n, np.zeros(n), np.full(n, np.nan)
    nxt = 0
    while True:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            r = reqs[nxt]
            tickets[nxt] = server.submit(r["op"], client.bits, r["da"], r["db"], r["out"], r["out2"])
            submit_t[nxt] = max(arrivals[nxt], now)
            nxt += 1
        st = server.stats()
        if st["running"] == 0 and st["queued"] == 0:
            if nxt == n:
                break
            time.sleep(max(0.0, min(arrivals[nxt] - now, 0.05)))
            continue
        server.step()
        now = time.perf_counter() - t0
        for i in range(nxt):
            if np.isnan(done_t[i]) and server.poll(tickets[i]) == 2:
                done_t[i] = now
    return done_t - submit_t, time.perf_counter() - t0


def run_serving(parties=4, bits=16, capacity_requests=96, requests=96, loads=(0.5, 0.9), wave_gates=4096,
                toy=False, cluster="auto", circuit_style="array", device=0, autotune_gates=1024):
    """Capacity (everything submitted at once) and Poisson runs at the given
    fractions of that capacity; returns a dict of throughput, p50/p99 latency
    (overall and per operator) and decryption checks."""
    P = W.toy_params(parties) if toy else W.full_params(parties)
    ctx = B.Context(P, W.CRS_SEED, device=device)
    for i, s in enumerate(W.party_seeds(parties)):
        ctx.keygen(i, s)
    if autotune_gates:
        ctx.autotune(autotune_gates)
    ctx.set_cluster(cluster)
    ctx.set_circuit_style(circuit_style)
    server = B.Server(ctx, wave_gates=wave_gates, pool_rows=1 << 20)
    client = Client(ctx, bits)
    stream = W.gd_request_stream(max(capacity_requests, requests), bits=bits)
    mix = {op: sum(1 for r in stream if r[0] == op) for op in ("add", "sub", "mul", "div")}

    def build(n, offset=0):
        return [client.prepare(offset + i, *stream[i]) for i in range(n)]

    # sustained capacity: everything submitted at t = 0 (closed batch)
    reqs = build(capacity_requests)
    lat, wall = run_stream(server, client, reqs)
    capacity = len(reqs) / wall
    ok = all(client.result(r) == W.expected_result(r["op"], r["a"], r["b"], bits) for r in reqs)
    out = {"parties": parties, "bits": bits, "n": P["n"], "N": P["N"], "mix": mix, "cluster": cluster,
           "circuit_style": circuit_style, "capacity_requests": capacity_requests,
           "capacity_requests_per_s": capacity, "capacity_wall_s": wall, "decrypt_ok": ok, "loads": []}
    for load in loads:
        reqs = build(requests, offset=10000)
        arr = W.poisson_arrivals(len(reqs), load * capacity)
        lat, wall = run_stream(server, client, reqs, arr)
        ok = all(client.result(r) == W.expected_result(r["op"], r["a"], r["b"], bits) for r in reqs)
        per_op = {}
        for op in ("add", "sub", "mul", "div"):
            l_op = [lat[i] for i in range(len(reqs)) if reqs[i]["op"] == op]
            if l_op:
                per_op[op] = {"p50_s": float(np.percentile(l_op, 50)), "p99_s": float(np.percentile(l_op, 99)),
                              "n": len(l_op)}
        out["loads"].append({"load": load, "requests": len(reqs), "rate_requests_per_s": load * capacity,
                             "throughput_requests_per_s": len(reqs) / wall,
                             "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                             "per_op": per_op, "decrypt_ok": ok, "wall_s": wall})
    out["server"] = server.stats()
    server.close()
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--parties", type=int, default=4)
    ap.add_argument("--bits", type=int, default=16)
    ap.add_argument("--capacity-requests", type=int, default=96)
    ap.add_argument("--requests", type=int, default=96)
    ap.add_argument("--loads", default="0.5,0.9")
    ap.add_argument("--wave-gates", type=int, default=4096)
    ap.add_argument("--toy", action="store_true")
    ap.add_argument("--cluster", default="auto", choices=["auto", "on", "off"],
                    help="latency (cluster) blind rotation for small waves")
    ap.add_argument("--circuit-style", default="array", choices=["array", "shallow"],
                    help="operator netlist family: fewest gates (array) or fewest levels (shallow)")
    args = ap.parse_args()
    B.load(build_if_missing=True)
    out = run_serving(args.parties, args.bits, args.capacity_requests, args.requests,
                      [float(x) for x in args.loads.split(",") if x], args.wave_gates, args.toy, args.cluster,
                      args.circuit_style)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

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


def main():
    import torch
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
    P = W.toy_params(args.parties) if args.toy else W.full_params(args.parties)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    for i, s in enumerate(W.party_seeds(args.parties)):
        ctx.keygen(i, s)
    ctx.autotune(1024)
    ctx.set_cluster(args.cluster)
    ctx.set_circuit_style(args.circuit_style)
    server = B.Server(ctx, wave_gates=args.wave_gates, pool_rows=1 << 20)
    client = Client(ctx, args.bits)
    stream = W.gd_request_stream(max(args.capacity_requests, args.requests), bits=args.bits)
    mix = {op: sum(1 for r in stream if r[0] == op) for op in ("add", "sub", "mul", "div")}

    def build(n, offset=0):
        return [client.prepare(offset + i, *stream[i]) for i in range(n)]

    # sustained capacity: everything submitted at t = 0 (closed batch)
    reqs = build(args.capacity_requests)
    lat, wall = run_stream(server, client, reqs)
    capacity = len(reqs) / wall
    ok = all(client.result(r) == W.expected_result(r["op"], r["a"], r["b"], args.bits) for r in reqs)
    out = {"parties": args.parties, "bits": args.bits, "n": P["n"], "N": P["N"], "mix": mix, "cluster": args.cluster,
           "capacity_requests_per_s": capacity, "capacity_wall_s": wall, "decrypt_ok": ok, "loads": []}
    for load in [float(x) for x in args.loads.split(",") if x]:
        reqs = build(args.requests, offset=10000)
        arr = W.poisson_arrivals(len(reqs), load * capacity)
        lat, wall = run_stream(server, client, reqs, arr)
        ok = all(client.result(r) == W.expected_result(r["op"], r["a"], r["b"], args.bits) for r in reqs)
        per_op = {}
        for op in ("add", "sub", "mul", "div"):
            l_op = [lat[i] for i in range(len(reqs)) if reqs[i]["op"] == op]
            if l_op:
                per_op[op] = {"p50_s": float(np.percentile(l_op, 50)), "p99_s": float(np.percentile(l_op, 99)),
                              "n": len(l_op)}
        out["loads"].append({"load": load, "rate_requests_per_s": load * capacity,
                             "throughput_requests_per_s": len(reqs) / wall,
                             "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                             "per_op": per_op, "decrypt_ok": ok, "wall_s": wall})
    out["server"] = server.stats()
    server.close()
    ctx.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

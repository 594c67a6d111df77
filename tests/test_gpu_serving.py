"""Continuous batching: requests of different operators, submitted at
different waves, share launches; each result is identical (word for word)
to the same request run alone through the ordinary operator entry points,
and decrypts to the native two's-complement result."""
import numpy as np
import pytest

from conftest import from_dev, oracle_keys

pytestmark = pytest.mark.gpu


def test_server_mix_equals_alone(gpu_ready):
    import torch
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    from paper_2205_05825_gb300.serving import Client
    P = W.toy_params(3)
    keys = oracle_keys(P)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    client = Client(ctx, 8)
    stream = W.gd_request_stream(10, bits=8, config_id=6)
    stream += [("div", -100, 7), ("mul", -128, 127), ("add", 127, 1), ("sub", -128, 1)]
    reqs = [client.prepare(i, *r) for i, r in enumerate(stream)]
    # alone: the ordinary entry points, one request at a time
    alone = []
    for r in reqs:
        o = torch.zeros_like(r["out"])
        if r["op"] == "div":
            o2 = torch.zeros_like(r["out2"])
            ctx.div_kbit(8, r["da"], r["db"], o, o2)
            alone.append((from_dev(o), from_dev(o2)))
        else:
            getattr(ctx, r["op"] + "_kbit")(8, r["da"], r["db"], o)
            alone.append((from_dev(o), None))
    # mixed: staggered submission, small waves so levels split and requests overlap
    server = B.Server(ctx, wave_gates=48, pool_rows=1 << 16)
    tickets = {}
    waves_with_several = 0
    step = 0
    while len(tickets) < len(reqs) or any(server.poll(t) != 2 for t in tickets.values()):
        for i in range(len(reqs)):
            if i not in tickets and i <= 2 * step:
                r = reqs[i]
                tickets[i] = server.submit(r["op"], 8, r["da"], r["db"], r["out"], r["out2"])
        if server.stats()["running"] + server.stats()["queued"] > 1:
            waves_with_several += 1
        server.step()
        step += 1
        assert step < 5000
    assert waves_with_several > 10
    for i, r in enumerate(reqs):
        assert np.array_equal(from_dev(r["out"]), alone[i][0]), i
        if r["op"] == "div":
            assert np.array_equal(from_dev(r["out2"]), alone[i][1]), i
        assert client.result(r) == W.expected_result(r["op"], r["a"], r["b"], 8), (i, r["op"], r["a"], r["b"])
    server.close()
    ctx.close()


def test_server_full_k4_mix_equals_alone(gpu_ready):
    """Full size (n = 560, N = 1024), four parties, 16-bit requests of all
    four operators (shallow netlist family, so the divider is 223 levels
    deep): submitted together, every result equals the same request run
    alone word for word, and decrypts to the native result."""
    import torch
    from paper_2205_05825_gb300 import binding as B
    from paper_2205_05825_gb300 import workloads as W
    from paper_2205_05825_gb300.serving import Client
    P = W.full_params(4)
    keys = oracle_keys(P)
    ctx = B.Context(P, W.CRS_SEED, device=0)
    ctx.import_oracle_keys(keys)
    ctx.set_circuit_style("shallow")
    client = Client(ctx, 16)
    stream = [("add", 1234, -567), ("sub", -32768, 1), ("mul", -181, 181), ("div", -30000, 7), ("mul", 255, -2)]
    reqs = [client.prepare(i, *r) for i, r in enumerate(stream)]
    alone = []
    for r in reqs:
        o = torch.zeros_like(r["out"])
        if r["op"] == "div":
            o2 = torch.zeros_like(r["out2"])
            ctx.div_kbit(16, r["da"], r["db"], o, o2)
            alone.append((from_dev(o), from_dev(o2)))
        else:
            getattr(ctx, r["op"] + "_kbit")(16, r["da"], r["db"], o)
            alone.append((from_dev(o), None))
    server = B.Server(ctx, wave_gates=4096, pool_rows=1 << 18)
    tickets = [server.submit(r["op"], 16, r["da"], r["db"], r["out"], r["out2"]) for r in reqs]
    steps = 0
    while any(server.poll(t) != 2 for t in tickets):
        server.step()
        steps += 1
        assert steps < 2000
    for i, r in enumerate(reqs):
        assert np.array_equal(from_dev(r["out"]), alone[i][0]), i
        if r["op"] == "div":
            assert np.array_equal(from_dev(r["out2"]), alone[i][1]), i
        assert client.result(r) == W.expected_result(r["op"], r["a"], r["b"], 16), (i, r["op"], r["a"], r["b"])
    server.close()
    ctx.close()

"""Parity at the full shape of the batched and the served workloads.

The batched workload: 4096 independent buffers with lognormal sizes (sigma
2) from 1 KiB to 64 MiB, about 2 GiB in all, packed in one allocation with
every start alignment modulo 16, parsed by one persistent launch replayed
from a CUDA graph (twice), then packed in buffer order on the device.  Every
buffer's count and every field's value and status must equal the oracle's.

The served workload: CSV requests (8 comma-separated columns, newline rows)
with lognormal sizes from 4 KiB to 256 MiB (at least one above 64 MiB),
submitted to the request server with Poisson-staggered arrivals under a
device-memory budget.  Every request's results must be the same in the mix
as alone, and equal to the oracle's.
"""
import random
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_batched_workload_at_full_shape_matches_the_oracle():
    texts = workloads.batch_buffers()  # 4096 buffers, about 2 GiB
    assert len(texts) == 4096
    lens = [len(t) for t in texts]
    assert sum(lens) > (1 << 31) * 0.9 and max(lens) > (32 << 20) and min(lens) >= 512
    arr, starts = workloads.pack_buffers(texts)
    d = torch.from_numpy(arr).cuda()
    views = [d[s:s + n] for s, n in zip(starts, lens)]
    offs = [0]
    for n in lens:
        offs.append(offs[-1] + n)
    out = torch.full((offs[-1],), -3.0, dtype=torch.float64, device="cuda")
    st = torch.full((offs[-1],), 0xEE, dtype=torch.uint8, device="cuda")
    cnt = torch.full((len(texts),), -1, dtype=torch.int64, device="cuda")
    # the oracle on all buffers at once: every buffer ends with a complete
    # field and no separator, so joining them with '\n' gives their fields
    # one after the other
    assert all(not t.endswith(b"\n") for t in texts)
    want_counts = [oracle.count_fields(t) for t in texts]
    rb, rs = oracle.parse_buffer(b"\n".join(texts))
    assert rb.size == sum(want_counts)
    plan = fp.BatchPlan(views, out, st, offs, cnt, graph=True)
    try:
        packed_v = torch.empty(rb.size, dtype=torch.float64, device="cuda")
        packed_s = torch.empty(rb.size, dtype=torch.uint8, device="cuda")
        tot = torch.empty(1, dtype=torch.int64, device="cuda")
        for rep in range(2):
            packed_v.fill_(-9.0)
            packed_s.fill_(0xAB)
            plan.launch()
            plan.gather(packed_v, packed_s, tot)
            torch.cuda.synchronize()
            assert fp.get_error() == 0
            assert cnt.cpu().tolist() == want_counts, "replay %d: per-buffer counts" % rep
            assert int(tot.item()) == rb.size
            got_v = packed_v.cpu().numpy().view(np.uint64)
            bad = np.nonzero(got_v != rb)[0]
            assert bad.size == 0, "replay %d: %d values differ, first at field %d" % (
                rep, bad.size, int(bad[0]))
            assert np.array_equal(packed_s.cpu().numpy(), rs), "replay %d: statuses" % rep
    finally:
        plan.close()
    del out, st, d, packed_v, packed_s
    torch.cuda.empty_cache()


def _serving_requests(count, seed):
    """count CSV request bodies, sizes clip(lognormal(ln 1 MiB, 1.85), 4 KiB,
    256 MiB), the largest forced above 64 MiB."""
    rng = np.random.default_rng(seed)
    sizes = np.clip(np.exp(np.log(1 << 20) + 1.85 * rng.standard_normal(count)), 4 << 10,
                    256 << 20).astype(np.int64)
    sizes[int(np.argmax(sizes))] = max(int(sizes.max()), 96 << 20)
    pool = workloads.csv_pool()
    return [workloads.csv_request(int(z), seed * 1000 + j, pool) for j, z in enumerate(sizes)]


def test_served_workload_at_full_shape_alone_equals_mix_and_oracle():
    texts = _serving_requests(48, 5151)
    assert max(len(t) for t in texts) > (64 << 20)
    # alone: one request at a time through the plain host entry point
    alone = []
    for t in texts:
        v, s = fp.parse_f64_host(t, b",")
        alone.append((v.view(np.uint64).copy(), s.copy()))
    # the mix: Poisson-staggered submissions to the server, so that requests
    # arrive while others are on the GPU
    rnd = random.Random(77)
    bufs = []
    for t in texts:  # pinned before the arrivals start
        n = max(len(t), 1)
        bufs.append((torch.frombuffer(bytearray(t), dtype=torch.uint8).pin_memory(),
                     torch.full((n,), -5.0, dtype=torch.float64).pin_memory(),
                     torch.full((n,), 0xEE, dtype=torch.uint8).pin_memory()))
    gaps = [rnd.expovariate(1.0 / 0.0002) for _ in texts]  # mean 0.2 ms between arrivals
    with fp.Server(device_budget=40_000_000_000, max_batch=1024, max_inflight=4,
                   delim=b",") as srv:
        rids = []
        t_next = time.perf_counter()
        for h, gap in zip(bufs, gaps):
            while time.perf_counter() < t_next:
                pass
            rids.append(srv.submit(*h))
            t_next += gap
        infos = [srv.wait(r, timeout_s=300) for r in rids]
        stats = srv.stats()
    assert stats["completed"] == len(texts)
    assert stats["max_batch_seen"] > 1  # requests shared launches
    for i, (t, info, h) in enumerate(zip(texts, infos, bufs)):
        assert info is not None and info["error"] == 0, (i, info)
        rb, rs = oracle.parse_buffer(t, b",")
        k = info["count"]
        assert k == rb.size == alone[i][0].size, "request %d: counts" % i
        got_v = h[1][:k].numpy().view(np.uint64)
        got_s = h[2][:k].numpy()
        assert np.array_equal(got_v, alone[i][0]) and np.array_equal(got_s, alone[i][1]), \
            "request %d: mix differs from alone" % i
        assert np.array_equal(got_v, rb) and np.array_equal(got_s, rs), \
            "request %d: differs from the oracle" % i

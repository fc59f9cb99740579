"""The request server (fp_server_*): continuous batching of host-memory
requests under a device-memory budget.  Each request's result must be the
same, bit for bit, alone (fp_parse_f64_host) and in any mix of requests
that share launches; the oracle pins a sample of them.
"""
import random
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


def request_texts(count, seed):
    """CSV blocks (the serving workload), plus other shapes: hard cases that
    take the fallback, empty and tiny texts, invalid fields."""
    rnd = random.Random(seed)
    pool = workloads.csv_pool(8 << 20, workloads.SEED_BASE + 55)
    texts = []
    for i in range(count):
        k = rnd.randrange(10)
        if k < 6:
            size = int(min(4 << 20, max(64, rnd.lognormvariate(10.0, 1.6))))
            texts.append(workloads.csv_request(size, seed * 1000 + i, pool))
        elif k == 6:
            texts.append(workloads.hard_case_text(rnd.randrange(1, 300), seed * 1000 + i)
                         .replace(b"\n", b","))
        elif k == 7:
            texts.append(b"")
        elif k == 8:
            texts.append(b"1,-2.5e-3,,x,1e400\n0x1p3,+.5,-0")
        else:
            texts.append(workloads.bulk_mixed_text(rnd.randrange(1, 20000), seed * 1000 + i))
    return texts


def host_arrays(text):
    n = max(len(text), 1)
    t = torch.frombuffer(bytearray(text), dtype=torch.uint8) if text else \
        torch.empty(0, dtype=torch.uint8)
    return (t.pin_memory(), torch.full((n,), -5.0, dtype=torch.float64).pin_memory(),
            torch.full((n,), 0xEE, dtype=torch.uint8).pin_memory())


def alone(texts):
    res = []
    for t in texts:
        v, s = fp.parse_f64_host(t, b",")
        res.append((v.view(np.uint64).copy(), s.copy()))
    return res


def serve(texts, server, stagger_s=0.0, seed=0):
    rnd = random.Random(seed)
    arrays = [host_arrays(t) for t in texts]  # pinned before the submissions start
    reqs = []
    for h in arrays:
        reqs.append((server.submit(*h), h))
        if stagger_s:
            time.sleep(rnd.random() * stagger_s)
    out = []
    for rid, (_, v, s) in reqs:
        info = server.wait(rid, timeout_s=120)
        assert info is not None and info["error"] == 0, info
        k = info["count"]
        out.append((v[:k].numpy().view(np.uint64).copy(), s[:k].numpy().copy(), info))
    return out


def assert_same(ref, got):
    for i, ((rv, rs), (gv, gs, info)) in enumerate(zip(ref, got)):
        assert gv.size == rv.size, "request %d: %d fields alone, %d in the mix" % (i, rv.size,
                                                                                  gv.size)
        assert np.array_equal(gv, rv), "request %d values differ" % i
        assert np.array_equal(gs, rs), "request %d statuses differ" % i


@pytest.fixture(scope="module")
def texts():
    return request_texts(240, 7)


@pytest.fixture(scope="module")
def ref(texts):
    return alone(texts)


def test_alone_results_match_the_oracle(texts, ref):
    for i in range(0, len(texts), 7):
        rb, rs = oracle.parse_buffer(texts[i], b",")
        assert np.array_equal(ref[i][0], rb) and np.array_equal(ref[i][1], rs)


def test_burst_mix_equals_alone(texts, ref):
    # a budget that holds only part of the burst, so admission has to wait
    total = sum(len(t) for t in texts)
    with fp.Server(device_budget=10 * (total // 4 + (8 << 20)), max_batch=16, max_inflight=3,
                   delim=b",") as srv:
        got = serve(texts, srv)
        st = srv.stats()
    assert_same(ref, got)
    assert st["completed"] == len(texts) and st["submitted"] == len(texts)
    assert st["max_batch_seen"] <= 16
    assert max(g[2]["batch_size"] for g in got) > 1  # requests did share launches
    assert st["launches"] >= (len(texts) + 15) // 16
    assert st["fields"] == sum(r[0].size for r in ref)


def test_launches_overlap_and_admission_follows_the_budget(texts, ref):
    total = sum(len(t) for t in texts)
    budget = 10 * (total // 6 + (8 << 20))
    with fp.Server(device_budget=budget, max_batch=8, max_inflight=3, delim=b",") as srv:
        got = serve(texts, srv)
        st = srv.stats()
    assert_same(ref, got)
    infos = [g[2] for g in got]
    # held units never exceeded the arena (units = budget / 10)
    assert st["peak_units"] <= budget // 10
    # some later launch began while an earlier one was still in flight
    ends = {}
    for i in infos:  # launch time -> when its last request completed
        ends[i["launch_ns"]] = max(ends.get(i["launch_ns"], 0), i["done_ns"])
    launches = sorted(ends.items())
    assert len(launches) > 2
    assert any(b[0] < a[1] for a, b in zip(launches, launches[1:]))
    # arrival order is admission order (first come, first served)
    admits = [i["admit_ns"] for i in infos]
    assert admits == sorted(admits)
    for i in infos:
        assert i["submit_ns"] <= i["admit_ns"] <= i["launch_ns"] <= i["done_ns"]


def test_staggered_arrivals_equal_alone(texts, ref):
    with fp.Server(device_budget=4 << 30, max_batch=64, max_inflight=2, delim=b",") as srv:
        got = serve(texts, srv, stagger_s=0.002, seed=3)
    assert_same(ref, got)


def test_budget_limits():
    text = workloads.csv_request(100_000, 1)
    with fp.Server(device_budget=10 * 65536, max_batch=4, max_inflight=1, delim=b",") as srv:
        h = host_arrays(text)
        with pytest.raises(_lib.FpError) as e:
            srv.submit(*h)  # needs more units than the whole arena
        assert e.value.code == _lib.FP_ERR_BUDGET
        small = workloads.csv_request(60_000, 2)
        hs = host_arrays(small)
        info = srv.wait(srv.submit(*hs), timeout_s=60)  # fits: 60,000 -> 60,160 units
        assert info["error"] == 0
        rb, rs = oracle.parse_buffer(small, b",")
        assert info["count"] == rb.size
        assert np.array_equal(hs[1][:rb.size].numpy().view(np.uint64), rb)
        with pytest.raises(_lib.FpError):
            srv.wait(123456, timeout_s=0)  # unknown id


def test_bad_configurations_are_refused():
    for kw in (dict(device_budget=100), dict(max_batch=0), dict(max_batch=70000),
               dict(max_inflight=0), dict(max_inflight=9)):
        with pytest.raises(_lib.FpError):
            fp.Server(**kw)


def test_output_capacity_bounds_the_copy():
    text = workloads.csv_request(20_000, 9)
    rb, rs = oracle.parse_buffer(text, b",")
    t = torch.frombuffer(bytearray(text), dtype=torch.uint8).pin_memory()
    v = torch.full((10,), -5.0, dtype=torch.float64).pin_memory()
    s = torch.full((10,), 0xEE, dtype=torch.uint8).pin_memory()
    with fp.Server(device_budget=1 << 26, max_batch=4, max_inflight=1, delim=b",") as srv:
        info = srv.wait(srv.submit(t, v, s[:7]), timeout_s=60)
    assert info["error"] == 0 and info["count"] == rb.size > 10
    assert np.array_equal(v[:7].numpy().view(np.uint64), rb[:7])
    assert (v[7:] == -5.0).all() and np.array_equal(s[:7].numpy(), rs[:7])


def test_pageable_host_memory_takes_the_copy_path(texts, ref):
    """Texts and result arrays that are not pinned are moved by copy calls
    instead of the gather / scatter kernels; results are the same."""
    with fp.Server(device_budget=1 << 30, max_batch=32, max_inflight=2, delim=b",") as srv:
        reqs = []
        for i, t in enumerate(texts[:60]):
            n = max(len(t), 1)
            ht = torch.frombuffer(bytearray(t), dtype=torch.uint8) if t else \
                torch.empty(0, dtype=torch.uint8)
            hv = torch.full((n,), -5.0, dtype=torch.float64)
            hs = torch.full((n,), 0xEE, dtype=torch.uint8)
            if i % 3 == 1:
                ht = ht.pin_memory()          # pinned text, pageable results
            elif i % 3 == 2:
                hv, hs = hv.pin_memory(), hs.pin_memory()  # pageable text, pinned results
            reqs.append((srv.submit(ht, hv, hs), hv, hs))
        got = []
        for rid, hv, hs in reqs:
            info = srv.wait(rid, timeout_s=120)
            assert info["error"] == 0
            k = info["count"]
            got.append((hv[:k].numpy().view(np.uint64).copy(), hs[:k].numpy().copy(), info))
    assert_same(ref[:60], got)


def test_large_requests_in_overlapping_segments():
    """Requests of 32 MB and more with pinned host arrays launch alone and
    are parsed in segments cut at separators, whose copies in, parses and
    copies out overlap: results equal the oracle's (hard cases at both ends
    of a segmented request included) while small requests are served beside
    them; a segmented request whose result array is shorter than its field
    count gets the full count and exactly the first out_cap results."""
    pool = workloads.csv_pool()
    hard_a = workloads.hard_case_text(2000, 143).replace(b"\n", b",")
    hard_b = workloads.hard_case_text(2000, 145).replace(b"\n", b",")
    big = [hard_a + b"\n" + workloads.csv_request(90 << 20, 144, pool) + b"\n" + hard_b,
           workloads.csv_request(40 << 20, 146, pool)]
    small = [workloads.csv_request(200_000, 147 + i, pool) for i in range(6)]
    texts = [big[0], small[0], small[1], big[1]] + small[2:]
    with fp.Server(device_budget=8_000_000_000, max_batch=64, max_inflight=4, delim=b",") as srv:
        got = serve(texts, srv)
        st = srv.stats()
    for i, (t, (gv, gs, info)) in enumerate(zip(texts, got)):
        rb, rs = oracle.parse_buffer(t, b",")
        assert gv.size == rb.size, i
        assert np.array_equal(gv, rb) and np.array_equal(gs, rs), i
    # 5 + 4 segment launches for the two large requests, at least one for the rest
    assert st["launches"] >= 10, st
    t = big[1]
    rb, rs = oracle.parse_buffer(t, b",")
    cap = rb.size // 2 + 3
    ht, hv, hs = host_arrays(t)
    with fp.Server(device_budget=2_000_000_000, max_batch=4, max_inflight=2, delim=b",") as srv:
        info = srv.wait(srv.submit(ht, hv[:cap], hs[:cap]), timeout_s=120)
    assert info["error"] == 0 and info["count"] == rb.size
    assert np.array_equal(hv[:cap].numpy().view(np.uint64), rb[:cap])
    assert np.array_equal(hs[:cap].numpy(), rs[:cap])
    assert (hv[cap:] == -5.0).all() and (hs[cap:].numpy() == 0xEE).all()

"""Batch plans (fp_batch_plan_*): many device buffers parsed by one
persistent launch that is set up once and replayed, directly or from a CUDA
graph.  Their results must equal the per-buffer entry point's and the
oracle's, bit for bit, on every replay and after the buffers' contents
change between replays.
"""
import random

import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import workloads

pytestmark = pytest.mark.gpu


def mixed_texts(count, seed):
    rnd = random.Random(seed)
    texts = []
    for i in range(count):
        k = rnd.randrange(5)
        if k == 0:
            texts.append(b"")
        elif k == 1:
            texts.append(workloads.uniform_text(rnd.randrange(1, 3000), seed * 1000 + i))
        elif k == 2:
            texts.append(workloads.bulk_mixed_text(rnd.randrange(1, 30000), seed * 1000 + i))
        elif k == 3:
            texts.append(workloads.hard_case_text(rnd.randrange(1, 400), seed * 1000 + i))
        else:
            texts.append(b"1.5,,2e5\n-0\n.25e-400\nx\n")
    return texts


def pack_to_device(texts):
    arr, starts = workloads.pack_buffers(texts)
    d = torch.from_numpy(arr).cuda()
    return d, [d[s:s + len(t)] for s, t in zip(starts, texts)]


def outputs(texts):
    offs = [0]
    for t in texts:
        offs.append(offs[-1] + len(t))
    cap = max(offs[-1], 1)
    out = torch.full((cap,), -3.0, dtype=torch.float64, device="cuda")
    st = torch.full((cap,), 0xEE, dtype=torch.uint8, device="cuda")
    cnt = torch.full((len(texts),), -1, dtype=torch.int64, device="cuda")
    return offs, out, st, cnt


def check_against_oracle(texts, offs, out, st, cnt, delim=b"\n"):
    counts = cnt.cpu().tolist()
    allv = out.cpu().numpy().view(np.uint64)
    alls = st.cpu().numpy()
    for b, t in enumerate(texts):
        rb, rs = oracle.parse_buffer(t, delim)
        assert counts[b] == rb.size, "buffer %d: %d fields, oracle %d" % (b, counts[b], rb.size)
        assert np.array_equal(allv[offs[b]:offs[b] + counts[b]], rb), "buffer %d values" % b
        assert np.array_equal(alls[offs[b]:offs[b] + counts[b]], rs), "buffer %d statuses" % b


@pytest.mark.parametrize("graph", [False, True])
def test_plan_matches_oracle_on_every_replay(graph):
    texts = mixed_texts(80, 11)
    _, views = pack_to_device(texts)
    offs, out, st, cnt = outputs(texts)
    plan = fp.BatchPlan(views, out, st, offs, cnt, delim=b",", graph=graph)
    try:
        for _ in range(3):
            out.fill_(-3.0)
            st.fill_(0xEE)
            cnt.fill_(-1)
            plan.launch()
            torch.cuda.synchronize()
            check_against_oracle(texts, offs, out, st, cnt, b",")
    finally:
        plan.close()


@pytest.mark.parametrize("graph", [False, True])
def test_replay_reads_the_buffers_current_contents(graph):
    a = [workloads.bulk_mixed_text(5000, 21), workloads.hard_case_text(300, 22)]
    b = [workloads.uniform_text(5000, 23), workloads.bulk_mixed_text(300, 24)]
    n = max(len(x) for x in a + b) + 64
    # same buffers, same lengths: pad each pair to a common length with a
    # run of newlines (empty trailing fields are INVALID, on both sides)
    a = [x + b"\n" * (n - len(x)) for x in a]
    b = [x + b"\n" * (n - len(x)) for x in b]
    d, views = pack_to_device(a)
    offs, out, st, cnt = outputs(a)
    plan = fp.BatchPlan(views, out, st, offs, cnt, graph=graph)
    try:
        plan.launch()
        torch.cuda.synchronize()
        check_against_oracle(a, offs, out, st, cnt)
        for v, x in zip(views, b):
            v.copy_(torch.frombuffer(bytearray(x), dtype=torch.uint8))
        plan.launch()
        torch.cuda.synchronize()
        check_against_oracle(b, offs, out, st, cnt)
    finally:
        plan.close()


def test_plan_equals_batch_call_and_per_buffer_calls():
    texts = mixed_texts(300, 31)
    _, views = pack_to_device(texts)
    offs, out, st, cnt = outputs(texts)
    plan = fp.BatchPlan(views, out, st, offs, cnt, graph=True)
    plan.launch()
    offs2, out2, st2, cnt2 = outputs(texts)
    fp.parse_f64_batch_into(views, out2, st2, offs2, cnt2)
    torch.cuda.synchronize()
    assert torch.equal(cnt, cnt2)
    counts = cnt.cpu().tolist()
    for b, v in enumerate(views):
        vals, s = fp.parse_f64(v)
        k = counts[b]
        assert vals.numel() == k
        assert torch.equal(out[offs[b]:offs[b] + k].view(torch.int64), vals.view(torch.int64))
        assert torch.equal(out2[offs[b]:offs[b] + k].view(torch.int64), vals.view(torch.int64))
        assert torch.equal(st[offs[b]:offs[b] + k], s)
    plan.close()


def test_single_buffer_plan_and_capacity_limit():
    text = workloads.uniform_text(1000, 41)
    _, views = pack_to_device([text])
    out = torch.full((400,), -1.0, dtype=torch.float64, device="cuda")
    st = torch.full((400,), 9, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    plan = fp.BatchPlan(views, out, st, [100, 300], cnt, graph=True)
    plan.launch()
    torch.cuda.synchronize()
    rb, _ = oracle.parse_buffer(text)
    assert int(cnt.item()) == 1000
    got = out.cpu().numpy().view(np.uint64)
    assert np.array_equal(got[100:300], rb[:200])
    assert (out[:100].cpu() == -1.0).all() and (out[300:].cpu() == -1.0).all()
    assert (st[:100].cpu() == 9).all() and (st[300:].cpu() == 9).all()
    plan.close()


def test_plan_on_the_batched_workload_sample():
    """A 64 MiB slice of the 4096-buffer workload's size law (lognormal,
    sigma 2), every buffer checked against the oracle."""
    texts = workloads.batch_buffers(512, 64 << 20, hi=8 << 20, seed=workloads.SEED_BASE + 44)
    _, views = pack_to_device(texts)
    offs, out, st, cnt = outputs(texts)
    plan = fp.BatchPlan(views, out, st, offs, cnt, graph=True)
    plan.launch()
    plan.launch()
    torch.cuda.synchronize()
    check_against_oracle(texts, offs, out, st, cnt)
    plan.close()


@pytest.mark.parametrize("graph", [False, True])
def test_gather_packs_the_results_in_buffer_order(graph):
    """fp_batch_plan_gather: every buffer's results, exactly its count of
    them, in buffer order and nothing after the total -- equal to the
    oracle's results of the buffers one after the other; empty buffers and
    buffers larger than one packing piece (8192 fields) included."""
    texts = mixed_texts(60, 21) + [workloads.uniform_text(20000, 22), b"",
                                   workloads.bulk_mixed_text(30000, 23)]
    _, views = pack_to_device(texts)
    offs, out, st, cnt = outputs(texts)
    plan = fp.BatchPlan(views, out, st, offs, cnt, graph=graph)
    try:
        cap = max(offs[-1], 1)
        dst = torch.full((cap + 16,), -7.0, dtype=torch.float64, device="cuda")
        dst_st = torch.full((cap + 16,), 0xAB, dtype=torch.uint8, device="cuda")
        tot = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        want_v, want_s = [], []
        for t in texts:
            rb, rs = oracle.parse_buffer(t)
            want_v.append(rb)
            want_s.append(rs)
        want_v = np.concatenate(want_v)
        want_s = np.concatenate(want_s)
        for _ in range(2):
            plan.launch()
            plan.gather(dst, dst_st, tot)
            torch.cuda.synchronize()
            n = int(tot.item())
            assert n == want_v.size
            assert np.array_equal(dst[:n].cpu().numpy().view(np.uint64), want_v)
            assert np.array_equal(dst_st[:n].cpu().numpy(), want_s)
            assert (dst[n:].cpu().numpy() == -7.0).all() and (dst_st[n:].cpu().numpy() == 0xAB).all()
    finally:
        plan.close()


def test_gather_keeps_what_each_buffer_holds():
    """A buffer with more fields than output room keeps its first ones and
    reports all of them; the packing takes min(count, room) of each buffer,
    the last one's included, so nothing past the plan's outputs is read and
    the total fits the room the offsets reserve."""
    texts = [workloads.uniform_text(20000, 31), workloads.bulk_mixed_text(3000, 32), b"",
             workloads.uniform_text(700, 33)]
    want = [oracle.parse_buffer(t) for t in texts]
    rooms = [10000, want[1][0].size + 5, 0, 5]  # first and last below their counts
    offs = [0]
    for r in rooms:
        offs.append(offs[-1] + r)
    _, views = pack_to_device(texts)
    out = torch.full((offs[-1],), -3.0, dtype=torch.float64, device="cuda")
    st = torch.full((offs[-1],), 0xEE, dtype=torch.uint8, device="cuda")
    cnt = torch.full((len(texts),), -1, dtype=torch.int64, device="cuda")
    plan = fp.BatchPlan(views, out, st, offs, cnt)
    try:
        plan.launch()
        total = sum(min(w[0].size, r) for w, r in zip(want, rooms))
        dst = torch.full((total + 16,), -7.0, dtype=torch.float64, device="cuda")
        dst_st = torch.full((total + 16,), 0xAB, dtype=torch.uint8, device="cuda")
        tot = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        plan.gather(dst, dst_st, tot)
        torch.cuda.synchronize()
        assert cnt.cpu().tolist() == [w[0].size for w in want]
        assert int(tot.item()) == total
        want_v = np.concatenate([w[0][:r] for w, r in zip(want, rooms)])
        want_s = np.concatenate([w[1][:r] for w, r in zip(want, rooms)])
        assert np.array_equal(dst[:total].cpu().numpy().view(np.uint64), want_v)
        assert np.array_equal(dst_st[:total].cpu().numpy(), want_s)
        assert (dst[total:].cpu().numpy() == -7.0).all()
        assert (dst_st[total:].cpu().numpy() == 0xAB).all()
    finally:
        plan.close()


def test_binding_refuses_misplaced_outputs():
    """Outputs the kernels would write through a wrong address are refused
    before any call: host tensors, another dtype, too few entries, counts of
    the wrong width."""
    text = torch.frombuffer(bytearray(b"1.5\n2\n"), dtype=torch.uint8).cuda()
    good = dict(out_f64=torch.empty(6, dtype=torch.float64, device="cuda"),
                out_status=torch.empty(6, dtype=torch.uint8, device="cuda"),
                out_count=torch.zeros(1, dtype=torch.int64, device="cuda"))
    bad = [("out_f64", torch.empty(6, dtype=torch.float64)),
           ("out_f64", torch.empty(6, dtype=torch.float32, device="cuda")),
           ("out_f64", torch.empty(5, dtype=torch.float64, device="cuda")),
           ("out_status", torch.empty(6, dtype=torch.uint8)),
           ("out_count", torch.zeros(1, dtype=torch.int32, device="cuda")),
           ("out_count", torch.zeros(1, dtype=torch.int64))]
    for name, t in bad:
        args = dict(good, **{name: t})
        with pytest.raises((TypeError, ValueError)):
            fp.parse_f64_into(text, args["out_f64"], args["out_status"], args["out_count"])
    fp.parse_f64_into(text, good["out_f64"], good["out_status"], good["out_count"])
    torch.cuda.synchronize()
    assert int(good["out_count"].item()) == 2

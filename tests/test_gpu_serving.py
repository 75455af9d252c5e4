"""Serving loop (continuous batching, admission by footprint, graph
replay) through the C ABI: every result equals the same frame denoised
alone, per-stream delivery order, refusals and bounded waits."""
import threading

import numpy as np
import pytest

import synth
from tests._util import args, stack_frames, to_dev

pytestmark = pytest.mark.gpu

OK, EBUSY, ETIMEOUT = 0, 5, 6


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _frames(sizes, seed0):
    return [to_dev(stack_frames([synth.make_frame(h, w, seed0 + i)])) for i, (h, w) in enumerate(sizes)]


def test_mixed_sizes_equal_solo_results(torch):
    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300.serving import Server
    wb = synth.make_weights(seed=11)
    sizes = [(72, 128), (90, 160), (72, 128), (45, 67), (90, 160), (72, 128)] * 3
    frames = _frames(sizes, 500)
    srv = Server(wb, "bf16", max_hw=(96, 176), n_workers=3, max_batch=3, batch_window_us=500)
    outs = [torch.full((1, 3, h, w), float("nan"), device="cuda") for (h, w) in sizes]
    tickets = [None] * len(sizes)

    def client(sid):  # three client streams submitting concurrently
        for i in range(sid, len(sizes), 3):
            tickets[i] = srv.submit(sid, *args(frames[i]), outs[i])

    th = [threading.Thread(target=client, args=(s,)) for s in range(3)]
    [t.start() for t in th]
    [t.join() for t in th]
    for t in tickets:
        assert srv.wait(t, 20000) == OK
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(sizes) and st["failed"] == 0
    assert st["graph_launches"] > 0 and st["p99_ms"] >= st["p50_ms"] > 0
    solo = {}
    for i, (h, w) in enumerate(sizes):
        if (h, w) not in solo:
            solo[(h, w)] = wk.Denoiser(wb, "bf16", max_hw=(h, w))
        ref = solo[(h, w)].denoise(*args(frames[i]))
        assert torch.equal(outs[i], ref), i


def test_delivery_in_order_per_stream_and_bounded_wait(torch):
    from paper_2202_05977_b300.serving import Server
    wb = synth.make_weights(seed=12)
    big, small = _frames([(96, 176)], 600)[0], _frames([(16, 16)], 601)[0]
    srv = Server(wb, "bf16", max_hw=(96, 176), n_workers=2, max_batch=1, batch_window_us=0)
    srv.pause(True)
    o1 = torch.empty((1, 3, 96, 176), device="cuda")
    o2 = torch.empty((1, 3, 16, 16), device="cuda")
    t1 = srv.submit(7, *args(big), o1)
    t2 = srv.submit(7, *args(small), o2)
    assert srv.wait(t2, 50) == ETIMEOUT      # paused: nothing runs, the wait gives up
    srv.pause(False)
    assert srv.wait(t2, 20000) == OK          # t2 is delivered only after t1 (same stream)
    assert srv.wait(t1, 0) == OK
    srv.stop()


def test_admission_refusals(torch):
    from paper_2202_05977_b300.serving import Server
    wb = synth.make_weights(seed=13)
    fr = _frames([(64, 64)], 700)[0]
    out = torch.empty((1, 3, 64, 64), device="cuda")
    # footprint of one 64x64 request is far above a 1 KiB budget
    srv = Server(wb, "bf16", max_hw=(64, 64), n_workers=1, max_batch=1, mem_budget=1024)
    st, _ = srv.try_submit(0, *args(fr), out)
    assert st == EBUSY
    srv.stop()
    # queue limit
    srv = Server(wb, "bf16", max_hw=(64, 64), n_workers=1, max_batch=1, max_queue=2)
    srv.pause(True)
    outs = [torch.empty((1, 3, 64, 64), device="cuda") for _ in range(3)]
    t = [srv.try_submit(0, *args(fr), outs[i]) for i in range(3)]
    assert [s for s, _ in t] == [OK, OK, EBUSY]
    srv.pause(False)
    assert all(srv.wait(tk, 20000) == OK for s, tk in t if s == OK)
    assert srv.stats()["rejected"] == 1
    srv.stop()


def test_budget_limits_concurrency_but_everything_completes(torch):
    from paper_2202_05977_b300.serving import Server
    wb = synth.make_weights(seed=14)
    frames = _frames([(64, 96)] * 6, 800)
    # budget fits about two requests at a time
    probe = Server(wb, "bf16", max_hw=(64, 96), n_workers=1, max_batch=1)
    probe.stop()
    per_req = 64 * 96 * 600
    srv = Server(wb, "bf16", max_hw=(64, 96), n_workers=4, max_batch=1, mem_budget=2 * per_req, batch_window_us=0)
    outs = [torch.empty((1, 3, 64, 96), device="cuda") for _ in frames]
    tk = [srv.submit(i, *args(f), o) for i, (f, o) in enumerate(zip(frames, outs))]
    assert all(srv.wait(t, 20000) == OK for t in tk)
    st = srv.stats()
    assert st["mem_peak"] <= 2 * per_req and st["completed"] == 6
    srv.stop()


def test_temporal_streams_equal_sequential_library_calls(torch):
    # per-stream temporal histories in the server: frames of three streams
    # (two sizes) submitted together batch across streams, run one at a time
    # per stream, and equal TemporalAccumulator + Denoiser called in order
    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300.serving import Server
    from paper_2202_05977_b300.temporal import TemporalAccumulator
    wb = synth.make_weights(seed=13)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    streams = {0: synth.make_sequence(40, 56, 4, seed=21), 1: synth.make_sequence(48, 64, 4, seed=22),
               2: synth.make_sequence(40, 56, 4, seed=23)}
    data = {s: [{k: dev(f[k]) for k in ("radiance", "albedo", "normal", "depth", "position", "motion")}
                for f in seq] for s, seq in streams.items()}
    srv = Server(wb, "bf16", max_hw=(48, 64), n_workers=3, max_batch=4, batch_window_us=500)
    srv.pause(True)
    outs, tickets = {}, []
    for t in range(4):
        for s in streams:
            f = data[s][t]
            o = torch.full((1, 3, *f["radiance"].shape[1:]), float("nan"), device="cuda")
            outs[(s, t)] = o
            tickets.append(srv.submit_temporal(s, f["radiance"], f["albedo"], f["normal"], f["depth"],
                                               f["position"], f["motion"], o, reset=(s == 2 and t == 2)))
    srv.pause(False)
    for tk in tickets:
        assert srv.wait(tk, 20000) == OK
    st = srv.stats()
    srv.stop()
    assert st["temporal_frames"] == 12 and st["temporal_streams"] == 3 and st["failed"] == 0
    for s, seq in data.items():
        h, w = seq[0]["radiance"].shape[1:]
        ta = TemporalAccumulator(h, w)
        d = wk.Denoiser(wb, "bf16", max_hw=(h, w))
        for t, f in enumerate(seq):
            if s == 2 and t == 2:
                ta.reset()
            acc = ta.step(f["radiance"], f["position"], f["normal"], f["motion"])
            ref = d.denoise(acc[None], f["albedo"][None], f["normal"][None], f["depth"][None])
            assert torch.equal(outs[(s, t)], ref), (s, t)


def test_temporal_stream_restarts_when_its_size_changes(torch):
    # a stream whose frames change size gets a fresh history at the new size
    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300.serving import Server
    from paper_2202_05977_b300.temporal import TemporalAccumulator
    wb = synth.make_weights(seed=14)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    small = synth.make_sequence(40, 56, 2, seed=31)
    large = synth.make_sequence(48, 64, 2, seed=32)
    seq = [{k: dev(f[k]) for k in ("radiance", "albedo", "normal", "depth", "position", "motion")}
           for f in small + large]
    srv = Server(wb, "bf16", max_hw=(48, 64), n_workers=2, max_batch=2)
    outs = []
    for f in seq:
        o = torch.empty((1, 3, *f["radiance"].shape[1:]), device="cuda")
        t = srv.submit_temporal(5, f["radiance"], f["albedo"], f["normal"], f["depth"], f["position"], f["motion"], o)
        assert srv.wait(t, 20000) == OK
        outs.append(o)
    srv.stop()
    for part, frames in ((outs[:2], seq[:2]), (outs[2:], seq[2:])):
        h, w = frames[0]["radiance"].shape[1:]
        ta, d = TemporalAccumulator(h, w), wk.Denoiser(wb, "bf16", max_hw=(h, w))
        for o, f in zip(part, frames):
            acc = ta.step(f["radiance"], f["position"], f["normal"], f["motion"])
            assert torch.equal(o, d.denoise(acc[None], f["albedo"][None], f["normal"][None], f["depth"][None]))


def test_saturating_burst_batches_overlaps_and_matches_solo(torch):
    """Saturating load: 60 requests of three sizes queued at once (admission
    paused while they arrive, then resumed) on two workers.  The scheduler
    forms batches of several frames, the two workers' batches are in flight
    on the GPU at the same time (their dispatch-to-done intervals overlap),
    and every result is bit-identical to the same frame denoised alone."""
    import paper_2202_05977_b300 as wk
    from paper_2202_05977_b300.serving import Server
    wb = synth.make_weights(seed=14)
    shapes = [(96, 160), (72, 128), (120, 200)]
    sizes = [shapes[i % 3] for i in range(60)]
    frames = _frames(sizes, 800)
    srv = Server(wb, "bf16", max_hw=(120, 200), n_workers=2, max_batch=4, batch_window_us=0)
    # graphs captured before the measured burst
    warm = [torch.empty((1, 3, h, w), device="cuda") for (h, w) in shapes]
    for (h, w), o, f in zip(shapes, warm, frames[:3]):
        assert srv.wait(srv.submit(0, *args(f), o), 20000) == OK
    srv.pause(True)
    outs = [torch.full((1, 3, h, w), float("nan"), device="cuda") for (h, w) in sizes]
    tickets = [srv.submit(i % 6, *args(frames[i]), outs[i]) for i in range(len(sizes))]
    srv.pause(False)
    infos = []
    for t in tickets:
        s, info = srv.wait_info(t, 30000)
        assert s == OK
        infos.append(info)
    st = srv.stats()
    srv.stop()
    assert st["failed"] == 0
    batches = [x["batch"] for x in infos]
    assert max(batches) > 1 and sum(batches) / len(batches) > 1.5, batches
    by_worker = {}
    for x in infos:
        by_worker.setdefault(x["worker"], set()).add((x["dispatch_ms"], x["done_ms"]))
    assert set(by_worker) == {0, 1}, by_worker.keys()
    overlap = any(a0 < b1 and a1 < b0 for (a0, b0) in by_worker[0] for (a1, b1) in by_worker[1])
    assert overlap, by_worker
    solo = {}
    for i, (h, w) in enumerate(sizes):
        if (h, w) not in solo:
            solo[(h, w)] = wk.Denoiser(wb, "bf16", max_hw=(h, w))
        assert torch.equal(outs[i], solo[(h, w)].denoise(*args(frames[i]))), i

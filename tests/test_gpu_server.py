"""Continuous-batching server (fse_server_*) on the GPU: results equal the
same jobs run alone, new requests join the running executor, cancellation,
errors."""
import numpy as np
import pytest

import paper_2207_00238_gb300 as fse
from paper_2207_00238_gb300 import synth
from tests.gpu_util import run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    fse.build()
    c = fse.Context(0, arena_bytes=1 << 30)
    yield c
    c.close()


def _mix(n, seed=synth.SEED_BASE + 50):
    rng = synth.Rng(seed)
    jobs = []
    for i in range(n):
        W = int(rng.randint(1, 40, 300)[0])
        H = int(rng.randint(1, 40, 220)[0])
        small = i % 3 == 0
        b, B, F, K = (4, 14, 32, 60) if small else (8, 16, 64, int(rng.randint(1, 20, 120)[0]))
        sub = synth.Rng(seed * 7 + i)
        img = synth.image(W, H, sub, structure=True)
        nb = ((W + b - 1) // b) * ((H + b - 1) // b)
        mask, _ = synth.block_mask(W, H, b, max(1, int(0.2 * nb)), sub)
        n_tiles = 1 + i % 3
        jobs.append(dict(image=img, mask=mask, params=synth.params(b, B, F, K, n_tiles=n_tiles, overlap=8)))
    return jobs


def test_results_same_alone_and_in_the_mix(ctx):
    jobs = _mix(18)
    srv = fse.Server(ctx, arena_bytes=512 << 20, max_queue=64, max_resident=8, max_batch=4)
    try:
        outs = [np.zeros_like(j["image"]) for j in jobs]
        gs = [np.zeros(j["image"].shape, np.float32) for j in jobs]
        tickets = [srv.submit(j["image"], j["mask"], o, j["params"], out_f32=g)
                   for j, o, g in zip(jobs, outs, gs)]
        for t in tickets:
            srv.wait(t, timeout_ms=60000)
        lat = srv.latencies()
        assert len(lat) == len(jobs) and (lat > 0).all()
    finally:
        srv.close()
    for j, o, g in zip(jobs, outs, gs):
        alone, _ = run_gpu(ctx, [j])
        assert (alone[0]["out"] == o).all()
        assert (alone[0]["g"] == g).all()


def test_server_errors(ctx):
    srv = fse.Server(ctx, arena_bytes=64 << 20, max_queue=2, max_resident=1, max_batch=1)
    try:
        with pytest.raises(fse.FseError) as e:
            srv.wait(12345, timeout_ms=10)
        assert e.value.code == fse.ENOTFOUND
        big = np.zeros((4096, 4096), np.uint8)
        with pytest.raises(fse.FseError) as e:
            srv.submit(big, big, big, synth.params(8, 16, 64, 10))
        assert e.value.code == fse.ENOMEM
        with pytest.raises(fse.FseError) as e:
            srv.submit(big[:16, :16], big[:16, :16], big[:16, :16], synth.params(8, 16, 16, 10))
        assert e.value.code == fse.EINVAL
        # a long request occupies the only resident slot; the queue fills up
        job = synth.tiled_1024(W=512, H=512, K=200, n_tiles=1)[0]
        outs = [np.zeros_like(job["image"]) for _ in range(6)]
        got_busy = False
        tickets, taken = [], []
        for o in outs:
            try:
                tickets.append(srv.submit(job["image"], job["mask"], o, job["params"]))
                taken.append(o)
            except fse.FseError as ex:
                assert ex.code == fse.EBUSY
                got_busy = True
        assert got_busy
        for t in tickets:
            srv.wait(t, timeout_ms=60000)
        for o in taken:  # the requests the server took, one after the other in one slot
            assert (o == taken[0]).all()
    finally:
        srv.close()


def test_short_request_overtakes_a_long_one(ctx):
    """A short request submitted after a long one finishes first: it joins the
    resident executor beside the long one instead of waiting for it."""
    long_job = synth.tiled_1024(W=2048, H=2048, K=200, n_tiles=4)[0]
    short_job = _mix(1)[0]
    srv = fse.Server(ctx, arena_bytes=2 << 30, max_queue=8, max_resident=8)
    try:
        lo = np.zeros_like(long_job["image"])
        so = np.zeros_like(short_job["image"])
        t_long = srv.submit(long_job["image"], long_job["mask"], lo, long_job["params"])
        t_short = srv.submit(short_job["image"], short_job["mask"], so, short_job["params"])
        srv.wait(t_short, timeout_ms=60000)
        assert srv.poll(t_long) != fse.REQ_DONE
        srv.wait(t_long, timeout_ms=120000)
    finally:
        srv.close()
    for j, o in ((long_job, lo), (short_job, so)):
        alone, _ = run_gpu(ctx, [j])
        assert (alone[0]["out"] == o).all()


def test_cancel_queued_and_running(ctx):
    long_job = synth.tiled_1024(W=2048, H=2048, K=200, n_tiles=4)[0]
    job = _mix(2)[1]
    srv = fse.Server(ctx, arena_bytes=2 << 30, max_queue=8, max_resident=1)
    try:
        outs = [np.zeros_like(long_job["image"]), np.zeros_like(job["image"]), np.zeros_like(job["image"])]
        t_run = srv.submit(long_job["image"], long_job["mask"], outs[0], long_job["params"])
        t_q = srv.submit(job["image"], job["mask"], outs[1], job["params"])  # behind the only slot
        srv.cancel(t_q)
        with pytest.raises(fse.FseError) as e:
            srv.wait(t_q, timeout_ms=10000)
        assert e.value.code == fse.ECANCELLED
        srv.cancel(t_run)
        with pytest.raises(fse.FseError) as e:
            srv.wait(t_run, timeout_ms=60000)
        assert e.value.code == fse.ECANCELLED
        with pytest.raises(fse.FseError) as e:
            srv.cancel(987654)
        assert e.value.code == fse.ENOTFOUND
        # the server goes on serving correctly
        t = srv.submit(job["image"], job["mask"], outs[2], job["params"])
        srv.wait(t, timeout_ms=60000)
    finally:
        srv.close()
    alone, _ = run_gpu(ctx, [job])
    assert (alone[0]["out"] == outs[2]).all()


def test_single_class_server(ctx):
    """A server that runs only the F = 64 class (the serving workload's) at full
    occupancy; F = 32 requests are refused; results equal the jobs run alone."""
    jobs = [j for j in _mix(9) if j["params"]["fft"] == 64]
    ctx.set_option(fse.OPT_SERVER_CLASSES, 2)
    try:
        srv = fse.Server(ctx, arena_bytes=512 << 20, max_queue=64, max_resident=8)
    finally:
        ctx.set_option(fse.OPT_SERVER_CLASSES, 3)
    try:
        small = _mix(1)[0]
        with pytest.raises(fse.FseError) as e:
            srv.submit(small["image"], small["mask"], np.zeros_like(small["image"]), small["params"])
        assert e.value.code == fse.EINVAL
        outs = [np.zeros_like(j["image"]) for j in jobs]
        tickets = [srv.submit(j["image"], j["mask"], o, j["params"]) for j, o in zip(jobs, outs)]
        for t in tickets:
            srv.wait(t, timeout_ms=60000)
    finally:
        srv.close()
    for j, o in zip(jobs, outs):
        alone, _ = run_gpu(ctx, [j])
        assert (alone[0]["out"] == o).all()

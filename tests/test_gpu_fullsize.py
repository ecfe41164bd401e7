"""Full-size workloads in the benchmark's launch configuration (needs a GPU).

The oracle cannot extrapolate a whole 1024^2 or 3840x2160 image inside a
test, but every block of PHASED phase 0 sees no earlier reconstruction, so
its result depends on the input alone; the oracle computes a seeded sample of
those blocks one by one.  Properties that hold at any size are checked on the
whole output: known pixels unchanged, every lost pixel modelled, the number of
lost blocks equal to an independent count from the mask and the tiling.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import paper_2207_00238_gb300 as fse
from paper_2207_00238_gb300 import synth
from tests.gpu_util import run_gpu

pytestmark = pytest.mark.gpu

TOL = 1.0  # FP32 path: grey levels


@pytest.fixture(scope="module")
def ctx():
    fse.build()
    c = fse.Context(0, arena_bytes=4 << 30)
    yield c
    c.close()


def _count_and_sample(oracle_lib, job, n_sample, seed):
    """Lost-block count of all extended tiles and a sample of phase-0 blocks
    that own lost core pixels: (tile, I, J)."""
    img, mask, p = job["image"], job["mask"], job["params"]
    H, W = img.shape
    b, B = p["block"], p["border"]
    P = -(-B // b) + 1
    rc, tiles = oracle_lib.plan_tiles(W, H, p["n_tiles"], p["overlap"])
    assert rc == 0
    total, cand = 0, []
    for t, (x, y, w, h, ex, ey, ew, eh) in enumerate(tiles):
        nby, nbx = -(-eh // b), -(-ew // b)
        m = np.zeros((nby * b, nbx * b), np.uint8)
        m[:eh, :ew] = mask[ey:ey + eh, ex:ex + ew]
        lost = m.reshape(nby, b, nbx, b).max(axis=(1, 3)) > 0
        total += int(lost.sum())
        core = np.zeros_like(m)
        core[y - ey:y - ey + h, x - ex:x - ex + w] = 1
        owns = (m * core).reshape(nby, b, nbx, b).max(axis=(1, 3)) > 0
        for I, J in zip(*np.nonzero(lost & owns)):
            if I % P == 0 and J % P == 0:
                cand.append((t, int(I), int(J)))
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(cand), size=min(n_sample, len(cand)), replace=False)
    return total, tiles, [cand[i] for i in sorted(pick)]


def _check_job(oracle_lib, job, got, lost_blocks, n_sample=32, seed=0):
    img, mask, p = job["image"], job["mask"], job["params"]
    lost = mask > 0
    assert (got["out"][~lost] == img[~lost]).all()
    assert np.isfinite(got["g"][lost]).all()
    total, tiles, sample = _count_and_sample(oracle_lib, job, n_sample, seed)
    if lost_blocks is not None:
        assert lost_blocks == total
    b = p["block"]

    def one(s):
        t, I, J = s
        x, y, w, h, ex, ey, ew, eh = tiles[t]
        _, g = oracle_lib.fse_block_alone(img, mask, tiles[t], I, J, **p)
        errs = []
        for yy in range(b):
            for xx in range(b):
                gy, gx = ey + I * b + yy, ex + J * b + xx
                if (gy < ey + eh and gx < ex + ew and mask[gy, gx] and x <= gx < x + w
                        and y <= gy < y + h):
                    errs.append(abs(float(got["g"][gy, gx]) - g[yy, xx]))
                    u8 = int(np.rint(np.clip(g[yy, xx], 0, 255)))
                    errs.append(abs(int(got["out"][gy, gx]) - u8))
        return max(errs)

    with ThreadPoolExecutor(8) as ex:
        worst = max(ex.map(one, sample))
    assert len(sample) > 0
    assert worst <= TOL, f"worst sampled error {worst}"
    return worst


def test_tiled_1024_full_size(ctx, oracle_lib):
    job = synth.tiled_1024()[0]
    got, st = run_gpu(ctx, [job])
    assert st["tiles"] == 16
    _check_job(oracle_lib, job, got[0], st["lost_blocks"], n_sample=32, seed=1)


def test_defects_4k_full_size(ctx, oracle_lib):
    job = synth.defects_4k()[0]
    got, st = run_gpu(ctx, [job])
    _check_job(oracle_lib, job, got[0], st["lost_blocks"], n_sample=48, seed=2)


def test_batch_subset_16_images(ctx, oracle_lib):
    """The first 16 images of the 256-image batch (uneven sizes, mixed block
    and DFT sizes, truncated supports) in one call."""
    jobs = synth.batch_256(n_images=16)
    got, st = run_gpu(ctx, jobs)
    assert st["jobs"] == 16
    for k, (j, g) in enumerate(zip(jobs, got)):
        _check_job(oracle_lib, j, g, None, n_sample=6, seed=10 + k)


def test_served_requests(ctx, oracle_lib):
    """Requests of the serving workload through the server."""
    stream = synth.serving_stream(n_requests=3)
    jobs = [job for _, job in stream]
    srv = fse.Server(ctx, arena_bytes=8 << 30, max_queue=16, max_resident=8, max_batch=4)
    try:
        outs = [np.zeros_like(j["image"]) for j in jobs]
        gs = [np.zeros(j["image"].shape, np.float32) for j in jobs]
        tickets = [srv.submit(j["image"], j["mask"], o, j["params"], out_f32=g)
                   for j, o, g in zip(jobs, outs, gs)]
        for t in tickets:
            srv.wait(t, timeout_ms=120000)
    finally:
        srv.close()
    for k, (j, o, g) in enumerate(zip(jobs, outs, gs)):
        _check_job(oracle_lib, j, dict(out=o, g=g), None, n_sample=6, seed=20 + k)

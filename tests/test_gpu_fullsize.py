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
from tests.gpu_util import oracle_run, psnr, run_gpu

pytestmark = pytest.mark.gpu

TOL = 1.0  # FP32 path: grey levels
# At F = 64 with K = 200, late iterations select among residual bins whose
# FP32 values carry rounding accumulated from the early, large updates; near-tied
# selections then differ from FP64 and the extrapolated pixels move by a few grey
# levels (0.4 % of the lost pixels of the 1024^2 workload, PSNR change 5e-4 dB).
# The FP64 device path shows the arithmetic itself is exact (1e-9 gates below).
TOL_F64_K200 = 4.0
TOL_FP64 = 1e-9


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


def _check_job(oracle_lib, job, got, lost_blocks, n_sample=32, seed=0, tol=None):
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
    if tol is None:
        tol = TOL if p["fft"] == 32 else TOL_F64_K200
    assert worst <= tol, f"worst sampled error {worst}"
    return worst


def test_tiled_1024_full_size(ctx, oracle_lib):
    """The benchmark workload: FP64 device path equals the oracle on the whole
    image; FP32 meets the PSNR gate against the oracle's whole image."""
    job = synth.tiled_1024()[0]
    got, st = run_gpu(ctx, [job])
    got64, _ = run_gpu(ctx, [job], precision=64, f64=True)
    assert st["tiles"] == 16
    ref = oracle_run(oracle_lib, job, report=False)
    lost = job["mask"] > 0
    assert np.abs(got64[0]["g"][lost] - ref["g"][lost]).max() <= TOL_FP64
    assert (got64[0]["out"] == ref["out"]).all()
    err = np.abs(got[0]["out"].astype(int) - ref["out"].astype(int))[lost]
    dpsnr = psnr(got[0]["out"], job["image"], lost) - psnr(ref["out"], job["image"], lost)
    assert abs(dpsnr) <= 0.05
    assert err.max() <= TOL_F64_K200 and (err > 1).mean() < 0.01
    _check_job(oracle_lib, job, got[0], st["lost_blocks"], n_sample=32, seed=1)


def test_defects_4k_full_size(ctx, oracle_lib):
    job = synth.defects_4k()[0]
    got, st = run_gpu(ctx, [job])
    _check_job(oracle_lib, job, got[0], st["lost_blocks"], n_sample=48, seed=2)
    got64, st64 = run_gpu(ctx, [job], precision=64, f64=True)
    _check_job(oracle_lib, job, got64[0], st64["lost_blocks"], n_sample=24, seed=3, tol=TOL_FP64)


def test_batch_subset_16_images(ctx, oracle_lib):
    """The first 16 images of the 256-image batch (uneven sizes, mixed block
    and DFT sizes, truncated supports) in one call."""
    jobs = synth.batch_256(n_images=16)
    got, st = run_gpu(ctx, jobs)
    assert st["jobs"] == 16
    for k, (j, g) in enumerate(zip(jobs, got)):
        _check_job(oracle_lib, j, g, None, n_sample=6, seed=10 + k)
    got64, _ = run_gpu(ctx, jobs, precision=64, f64=True)
    for k, (j, g) in enumerate(zip(jobs, got64)):
        _check_job(oracle_lib, j, g, None, n_sample=3, seed=30 + k, tol=TOL_FP64)


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

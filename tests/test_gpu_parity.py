"""CUDA path vs the FP64 oracle, through the C ABI (needs a GPU).

FP32 path: per-config max |err| <= 1.0 grey level and |delta PSNR| <= 0.05 dB
against the oracle's reconstruction.  FP64 device path: the same selected
bin sequence per block as the oracle and model values within 1e-9.
"""
import json
import os

import numpy as np
import pytest

import paper_2207_00238_gb300 as fse
from paper_2207_00238_gb300 import synth
from tests.gpu_util import oracle_run, psnr, run_gpu

pytestmark = pytest.mark.gpu

TOL_ERR = 1.0
TOL_DPSNR = 0.05
TOL_F64 = 1e-9


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    fse.build()
    c = fse.Context(0, arena_bytes=1 << 30)
    yield c
    c.close()


def _small_tiled(W=128, H=96, K=60, n_tiles=4, seed=synth.SEED_BASE + 20):
    return synth.tiled_1024(seed=seed, W=W, H=H, K=K, n_tiles=n_tiles)[0]


def _defects(W=96, H=72, seed=synth.SEED_BASE + 30, cols=2):
    rng = synth.Rng(seed)
    img = synth.image(W, H, rng, structure=True)
    mask = synth.defect_mask(W, H, 0.01, cols, rng)
    return dict(image=img, mask=mask, params=synth.params(4, 14, 32, 100, n_tiles=2, overlap=16))


CASES = {
    "plain_64": lambda: synth.plain_64()[0],
    "tiled_small_f64": lambda: _small_tiled(),
    "defects_small": lambda: _defects(),
}


def _fp32_check(oracle_lib, job, got, tol_err=TOL_ERR, name=None):
    ref = oracle_run(oracle_lib, job, report=False)
    lost = job["mask"] > 0
    err = np.abs(got["out"].astype(int) - ref["out"].astype(int))[lost]
    p_gpu = psnr(got["out"], job["image"], lost)
    p_ref = psnr(ref["out"], job["image"], lost)
    report = os.environ.get("FSE_TEST_REPORT")  # optional JSON-lines record of the comparisons
    if report and name:
        p = job["params"]
        with open(report, "a") as f:
            f.write(json.dumps({"workload": name, "lost_pixels": int(lost.sum()), "fft": p["fft"], "K": p["K"],
                                "order": p.get("order", "phased"), "fp32_max_err": int(err.max()),
                                "fp32_pixels_over_1": int((err > 1).sum()),
                                "fp32_max_abs_g": float(np.abs(got["g"][lost] - ref["g"][lost]).max()),
                                "fp32_dpsnr_db": float(p_gpu - p_ref)}) + "\n")
    assert (got["out"][~lost] == job["image"][~lost]).all()
    assert err.max() <= tol_err, f"max |err| {err.max()}"
    assert abs(p_gpu - p_ref) <= TOL_DPSNR, f"PSNR gpu {p_gpu:.4f} oracle {p_ref:.4f}"
    return err.max(), p_gpu - p_ref


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp32_within_tolerance(ctx, oracle_lib, case):
    job = CASES[case]()
    got, st = run_gpu(ctx, [job])
    assert st["lost_blocks"] > 0
    _fp32_check(oracle_lib, job, got[0], name=case)


def _seq_check(oracle_lib, ctx, job, **over):
    job = dict(job)
    job["params"] = dict(job["params"], **over)
    ctx.set_option(fse.OPT_DEBUG_CAPTURE, 1)
    try:
        got, st = run_gpu(ctx, [job], precision=64, f64=True)
        rec, useq = ctx.debug_fetch(int(st["lost_blocks"]) + 8)
    finally:
        ctx.set_option(fse.OPT_DEBUG_CAPTURE, 0)
    ref = oracle_run(oracle_lib, job, report=True)
    assert len(rec) == len(ref["blocks"]) == st["lost_blocks"]
    want = {(int(t), int(i), int(j)): tuple(s) for (t, i, j, _), s in zip(ref["blocks"], ref["useq"])}
    have = {(int(r[1]), int(r[2]), int(r[3])): tuple(s) for r, s in zip(rec, useq)}
    assert have.keys() == want.keys()
    bad = [k for k in want if have[k] != want[k]]
    assert not bad, f"{len(bad)} of {len(want)} blocks differ, e.g. {bad[0]}"
    lost = job["mask"] > 0
    np.testing.assert_allclose(got[0]["g"][lost], ref["g"][lost], rtol=0, atol=TOL_F64)
    assert (got[0]["out"] == ref["out"]).all()


@pytest.mark.parametrize("layout", [1, 2, 3, 4])
@pytest.mark.parametrize("case", ["plain_64", "defects_small"])
def test_fp32_f32_executor_layouts(ctx, oracle_lib, layout, case):
    """Each layout of the F = 32 executor meets the FP32 gate."""
    job = CASES[case]()
    ctx.set_option(fse.OPT_F32_LAYOUT, layout)
    try:
        got, _ = run_gpu(ctx, [job])
    finally:
        ctx.set_option(fse.OPT_F32_LAYOUT, 0)
    _fp32_check(oracle_lib, job, got[0])


@pytest.mark.parametrize("layout64,layout32", [(6, 3), (4, 1), (5, 2)])
def test_tma_staging_matches_plain_loads(ctx, layout64, layout32):
    """Support staging by TMA tensor copies hands the executors the same
    weights and values as plain loads: identical bytes and model values."""
    jobs = [CASES["plain_64"](), CASES["defects_small"](), _small_tiled()]
    res = {}
    for tma in (0, 1):
        ctx.set_option(fse.OPT_TMA_STAGING, tma)
        ctx.set_option(fse.OPT_F64_WARPS, layout64)
        ctx.set_option(fse.OPT_F32_LAYOUT, layout32)
        try:
            res[tma], _ = run_gpu(ctx, jobs)
        finally:
            ctx.set_option(fse.OPT_TMA_STAGING, 2)
            ctx.set_option(fse.OPT_F64_WARPS, 0)
            ctx.set_option(fse.OPT_F32_LAYOUT, 0)
    for a, b in zip(res[0], res[1]):
        assert (a["out"] == b["out"]).all()
        np.testing.assert_array_equal(a["g"], b["g"])


@pytest.mark.parametrize("layout32", [3, 2])
def test_tma_staging_small_support(ctx, oracle_lib, layout32):
    """A support smaller than the DFT (b=4, B=8: S=20 in F=32) narrows the TMA
    boxes; TMA and plain loads agree bit for bit and meet the FP32 gate."""
    rng = synth.Rng(synth.SEED_BASE + 41)
    img = synth.image(96, 64, rng, structure=True)
    mask, _ = synth.block_mask(96, 64, 4, 60, rng)
    job = dict(image=img, mask=mask, params=synth.params(4, 8, 32, 60, n_tiles=2, overlap=12))
    res = {}
    for tma in (0, 1):
        ctx.set_option(fse.OPT_TMA_STAGING, tma)
        ctx.set_option(fse.OPT_F32_LAYOUT, layout32)
        try:
            res[tma], _ = run_gpu(ctx, [job])
        finally:
            ctx.set_option(fse.OPT_TMA_STAGING, 2)
            ctx.set_option(fse.OPT_F32_LAYOUT, 0)
    assert (res[0][0]["out"] == res[1][0]["out"]).all()
    np.testing.assert_array_equal(res[0][0]["g"], res[1][0]["g"])
    _fp32_check(oracle_lib, job, res[1][0])


def test_f32_run_layout_matches_column_layout(ctx):
    """The row-run layouts of the F = 32 executor (TMA-capable and compact) do
    the column layout's arithmetic in the same order: identical bytes and model
    values."""
    jobs = [CASES["plain_64"](), CASES["defects_small"]()]
    res = {}
    for layout in (1, 3, 4):
        ctx.set_option(fse.OPT_F32_LAYOUT, layout)
        try:
            res[layout], _ = run_gpu(ctx, jobs)
        finally:
            ctx.set_option(fse.OPT_F32_LAYOUT, 0)
    for other in (3, 4):
        for a, b in zip(res[1], res[other]):
            assert (a["out"] == b["out"]).all()
            np.testing.assert_array_equal(a["g"], b["g"])


@pytest.mark.parametrize("warps", [2, 4, 5, 6, 8])
def test_fp32_f64_executor_variants(ctx, oracle_lib, warps):
    """Each warps-per-block variant of the F = 64 executor meets the FP32 gate."""
    job = _small_tiled()
    ctx.set_option(fse.OPT_F64_WARPS, warps)
    try:
        got, _ = run_gpu(ctx, [job])
    finally:
        ctx.set_option(fse.OPT_F64_WARPS, 0)
    _fp32_check(oracle_lib, job, got[0])


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_selection_sequence(ctx, oracle_lib, case):
    _seq_check(oracle_lib, ctx, CASES[case]())


@pytest.mark.parametrize("order", ["raster", "independent"])
def test_fp64_orders(ctx, oracle_lib, order):
    _seq_check(oracle_lib, ctx, _defects(W=80, H=56, cols=1), order=order)
    _seq_check(oracle_lib, ctx, _small_tiled(W=96, H=80, K=30, n_tiles=2), order=order)


# RASTER chains feed each block's reconstruction into the next one down a
# defect column, so a selection that differs from FP64 in one block moves the
# supports of all later ones: the FP32 gate here checks the whole chain.
@pytest.mark.parametrize("order", ["raster", "independent"])
def test_fp32_orders(ctx, oracle_lib, order):
    job = _defects(W=80, H=56, cols=1)
    job["params"] = dict(job["params"], order=order)
    got, _ = run_gpu(ctx, [job])
    _fp32_check(oracle_lib, job, got[0])


def test_tma_staging_dense_burst_loss(ctx):
    """Many F = 32 blocks whose supports hold reconstructions of other
    blocks (45 % of the 4x4 blocks lost, half in bursts), staged by TMA while
    the blocks they read are written by other warps of the same launch: the
    bytes and model values equal those of plain loads."""
    rng = synth.Rng(synth.SEED_BASE + 42)
    W, H = 512, 384
    img = synth.image(W, H, rng, structure=True)
    nb = (W // 4) * (H // 4)
    mask, _ = synth.block_mask(W, H, 4, int(0.45 * nb), rng)
    job = dict(image=img, mask=mask, params=synth.params(4, 14, 32, 60, n_tiles=2, overlap=16))
    res = {}
    ctx.set_option(fse.OPT_F32_LAYOUT, 3)  # the row-run layout with TMA staging
    try:
        for tma in (0, 1):
            ctx.set_option(fse.OPT_TMA_STAGING, tma)
            try:
                res[tma], st = run_gpu(ctx, [job])
            finally:
                ctx.set_option(fse.OPT_TMA_STAGING, 2)
            assert st["lost_blocks"] > 5000
    finally:
        ctx.set_option(fse.OPT_F32_LAYOUT, 0)
    assert (res[0][0]["out"] == res[1][0]["out"]).all()
    np.testing.assert_array_equal(res[0][0]["g"], res[1][0]["g"])


def test_tma_wait_times_out_and_context_survives(ctx):
    """A TMA staging whose completion never arrives (test option): its bounded
    wait runs out, the call reports FSE_ETIMEOUT, and the next call on the same
    context is correct."""
    job = CASES["defects_small"]()
    ref, _ = run_gpu(ctx, [job])
    ctx.set_option(fse.OPT_F32_LAYOUT, 3)  # the row-run layout with TMA staging
    ctx.set_option(fse.OPT_TMA_STAGING, 1)
    ctx.set_option(fse.OPT_TIMEOUT_MS, 50)
    ctx.set_option(fse.OPT_DEBUG_TMA_STALL, 1)
    try:
        with pytest.raises(fse.FseError) as e:
            run_gpu(ctx, [job])
        assert e.value.code == fse.ETIMEOUT
    finally:
        ctx.set_option(fse.OPT_DEBUG_TMA_STALL, 0)
        ctx.set_option(fse.OPT_TIMEOUT_MS, 20000)
    try:
        got, _ = run_gpu(ctx, [job])
    finally:
        ctx.set_option(fse.OPT_TMA_STAGING, 2)
        ctx.set_option(fse.OPT_F32_LAYOUT, 0)
    assert (got[0]["out"] == ref[0]["out"]).all()
    np.testing.assert_array_equal(got[0]["g"], ref[0]["g"])


def test_exec_modes_bitwise_equal(ctx):
    jobs = [_defects(), _small_tiled()]
    outs = {}
    for mode in ["dag", "levels", "per_block"]:
        ctx.exec_mode(mode)
        try:
            got, st = run_gpu(ctx, jobs)
        finally:
            ctx.exec_mode("dag")
        outs[mode] = got
    for mode in ["levels", "per_block"]:
        for a, b in zip(outs["dag"], outs[mode]):
            assert (a["out"] == b["out"]).all() and (a["g"] == b["g"]).all()


def test_batch_equals_alone(ctx):
    jobs = [_defects(), _small_tiled(), synth.plain_64()[0], _small_tiled(W=70, H=50, n_tiles=1)]
    mixed, st = run_gpu(ctx, jobs)
    assert st["jobs"] == 4
    for j, m in zip(jobs, mixed):
        alone, _ = run_gpu(ctx, [j])
        assert (alone[0]["out"] == m["out"]).all() and (alone[0]["g"] == m["g"]).all()


def test_item_ids_contiguous_per_tile(ctx):
    """The ordered enumeration: within a work class, item ids follow the tile
    (and so the job) order, each tile's lost blocks one contiguous id range."""
    jobs = [_defects(), _small_tiled(), synth.plain_64()[0], _small_tiled(W=70, H=50, n_tiles=1),
            _defects(W=80, H=64)]
    ctx.set_option(fse.OPT_DEBUG_CAPTURE, 1)
    try:
        _, st = run_gpu(ctx, jobs)
        rec, _ = ctx.debug_fetch(int(st["lost_blocks"]) + 8)
    finally:
        ctx.set_option(fse.OPT_DEBUG_CAPTURE, 0)
    assert len(rec) == st["lost_blocks"]
    tiles = rec[:, 1]
    descents = int((np.diff(tiles) < 0).sum())
    assert descents <= 2  # one non-decreasing run of tiles per work class
    runs = tiles[np.r_[True, np.diff(tiles) != 0]]
    assert len(runs) == len(np.unique(runs))  # no tile split over two id ranges
    assert len({tuple(r) for r in rec}) == len(rec)


def test_root_window_does_not_change_results(ctx):
    """Fed roots (FSE_OPT_ROOT_WINDOW) only change when blocks without lost
    predecessors enter the queue; every block still waits for its
    predecessors, so outputs and model values are bitwise those of the
    all-at-once queue, for windows down to one root per consumer."""
    # one CTA per SM keeps the window (roots per consumer x consumers) below
    # the number of roots, so most roots are fed by finished blocks
    jobs = [_defects(W=400, H=300), _small_tiled(W=512, H=384, n_tiles=4), synth.plain_64()[0],
            _small_tiled(W=70, H=50, n_tiles=1)]
    jobs += [dict(j, params=dict(j["params"], order="raster")) for j in (_defects(W=80, H=64), _small_tiled(W=96))]
    ctx.set_option(fse.OPT_CTAS_PER_SM, 1)
    ctx.set_option(fse.OPT_ROOT_WINDOW, 0)
    try:
        ref, st0 = run_gpu(ctx, jobs)
        for w in (1, 2, 5):
            ctx.set_option(fse.OPT_ROOT_WINDOW, w)
            got, st = run_gpu(ctx, jobs)
            assert st["lost_blocks"] == st0["lost_blocks"]
            for r, g in zip(ref, got):
                assert (r["out"] == g["out"]).all() and (r["g"] == g["g"]).all(), w
    finally:
        ctx.set_option(fse.OPT_ROOT_WINDOW, 2)
        ctx.set_option(fse.OPT_CTAS_PER_SM, 0)


def test_host_path_equals_device_path(ctx):
    """The host-buffer entry point: rows that are a multiple of 16 bytes
    (plain copies), packed rows of other widths (packed copies and a device
    re-pitch both ways) and strided host rows (2-D copies) in one call."""
    jobs = [_small_tiled(), _small_tiled(W=70, H=50, n_tiles=1), _small_tiled(W=53, H=41, n_tiles=2)]
    dev, _ = run_gpu(ctx, jobs)
    hj, outs, gs = [], [], []
    for i, job in enumerate(jobs):
        img, msk = job["image"], job["mask"]
        H, W = img.shape
        if i == 2:  # strided host rows: views into wider arrays, pitch W + 11
            wide = [np.zeros((H, W + 11), np.uint8) for _ in range(3)]
            wide[0][:, :W] = img
            wide[1][:, :W] = msk
            img, msk, out = (w[:, :W] for w in wide)
        else:
            out = np.zeros_like(img)
        g = np.zeros((H, W), np.float32)
        hj.append(fse.make_job(img, msk, out, job["params"], out_f32=g))
        outs.append(out)
        gs.append(g)
    for call in range(2):  # twice: the second call reuses the packed area
        for o, g in zip(outs, gs):
            o[...] = 0
            g[...] = 0
        ctx.extrapolate_host(hj)
        for o, g, d in zip(outs, gs, dev):
            assert (o == d["out"]).all() and (g == d["g"]).all(), call


def test_graph_replay(ctx):
    import torch
    job = _defects()
    ref, _ = run_gpu(ctx, [job])
    dev = torch.device("cuda", 0)
    img = torch.from_numpy(job["image"]).to(dev)
    msk = torch.from_numpy(job["mask"]).to(dev)
    out = torch.zeros_like(img)
    cj = [fse.make_job(img, msk, out, job["params"])]
    ctx.set_option(fse.OPT_USE_GRAPH, 1)
    try:
        for _ in range(3):
            out.zero_()
            ctx.extrapolate(cj, stats=False)
            torch.cuda.synchronize()
            assert (out.cpu().numpy() == ref[0]["out"]).all()
    finally:
        ctx.set_option(fse.OPT_USE_GRAPH, 0)


def test_back_to_back_calls_without_synchronisation(ctx):
    """Calls return before their table upload has run.  Two different job
    sets alternate on one stream with no synchronisation in between, each call
    writing its own output buffers; then graph replays of one set alternate
    with direct calls of the other.  Every call must see its own tables: a
    staging buffer rewritten under a queued copy hands a call the other set's
    tables, and its own outputs stay unwritten."""
    import torch
    dev = torch.device("cuda", 0)
    R = 12
    sets = [[_defects()], [_small_tiled(), synth.plain_64()[0]]]
    refs = [run_gpu(ctx, js)[0] for js in sets]
    outs, cjobs = [], []
    for js in sets:
        o_set, c_set = [], []
        for j in js:
            img = torch.from_numpy(j["image"]).to(dev)
            msk = torch.from_numpy(j["mask"]).to(dev)
            o = [torch.zeros_like(img) for _ in range(R)]
            o_set.append((img, msk, o))
            c_set.append([fse.make_job(img, msk, x, j["params"]) for x in o])
        outs.append(o_set)
        cjobs.append(c_set)

    def call(si, r):
        ctx.extrapolate([c[r] for c in cjobs[si]], stats=False)

    def check(si, rs):
        for k, (_, _, o) in enumerate(outs[si]):
            for r in rs:
                assert (o[r].cpu().numpy() == refs[si][k]["out"]).all(), (si, k, r)

    torch.cuda.synchronize()
    for r in range(R):  # direct launches, alternating sets
        call(0, r)
        call(1, r)
    torch.cuda.synchronize()
    check(0, range(R))
    check(1, range(R))
    for _, _, o in outs[0] + outs[1]:
        for x in o:
            x.zero_()
    try:
        ctx.set_option(fse.OPT_USE_GRAPH, 1)
        call(0, 0)  # capture
        torch.cuda.synchronize()
        for r in range(R):  # replays of set 0 between direct calls of set 1
            for _, _, o in outs[0]:
                o[0].zero_()
            ctx.set_option(fse.OPT_USE_GRAPH, 1)
            call(0, 0)
            ctx.set_option(fse.OPT_USE_GRAPH, 0)
            call(1, r)
        torch.cuda.synchronize()
    finally:
        ctx.set_option(fse.OPT_USE_GRAPH, 0)
    check(0, [0])
    check(1, range(R))


def test_edge_cases(ctx, oracle_lib):
    rng = synth.Rng(synth.SEED_BASE + 40)
    img = synth.image(45, 37, rng)  # ragged: not a multiple of the block size
    # nothing lost: output == input, no blocks
    job = dict(image=img, mask=np.zeros_like(img), params=synth.params(4, 14, 32, 50, n_tiles=3, overlap=8))
    got, st = run_gpu(ctx, [job])
    assert st["lost_blocks"] == 0 and (got[0]["out"] == img).all()
    # everything lost: every support is empty, output 0
    job = dict(image=img, mask=np.ones_like(img), params=synth.params(4, 14, 32, 50))
    got, st = run_gpu(ctx, [job])
    assert st["empty_blocks"] == st["lost_blocks"] > 0 and (got[0]["out"] == 0).all()
    # image smaller than one support, portrait, ragged, several tiles
    img = synth.image(21, 53, rng)
    mask = np.zeros_like(img)
    mask[10:14, 3:9] = 1
    mask[40, 17] = 1
    job = dict(image=img, mask=mask, params=synth.params(8, 16, 64, 40, n_tiles=3, overlap=5))
    got, _ = run_gpu(ctx, [job])
    _fp32_check(oracle_lib, job, got[0])
    _seq_check(oracle_lib, ctx, job)


@pytest.mark.parametrize("block,border,fft,K,kw", [
    (2, 15, 32, 256, {}),                          # support fills the DFT, K at its maximum
    (16, 24, 64, 50, {}),                          # F = 64 support fills the DFT, 16x16 blocks
    (4, 14, 32, 1, dict(gamma=1.0)),               # one iteration, full step
    (8, 8, 32, 80, dict(rho=0.5, delta=1.0)),      # other weights, reconstructions at full weight
    (1, 8, 32, 60, dict(order="raster")),          # single-pixel blocks, raster chains
])
def test_parameter_extremes(ctx, oracle_lib, block, border, fft, K, kw):
    """Parameters at the ends of their ranges: the FP64 device path selects
    the oracle's bins on every block and the FP32 path meets the gate."""
    rng = synth.Rng(synth.SEED_BASE + 70 + block + K)
    W, H = 120, 88
    img = synth.image(W, H, rng, structure=True)
    nb = ((W + block - 1) // block) * ((H + block - 1) // block)
    mask, _ = synth.block_mask(W, H, block, max(1, int(0.12 * nb)), rng)
    job = dict(image=img, mask=mask, params=synth.params(block, border, fft, K, n_tiles=2, overlap=16, **kw))
    got, st = run_gpu(ctx, [job])
    assert st["lost_blocks"] > 0
    _fp32_check(oracle_lib, job, got[0])
    _seq_check(oracle_lib, ctx, job)


def test_contexts_keep_their_own_executor_choice(ctx):
    """Executor variants are a context's own setting: two contexts in one
    process, set to different variants that compute the same arithmetic (F = 32
    column and row-run layouts, K-loop unrolled or not) and used in turn, give
    the same bytes, and the first context's choice survives the second's."""
    jobs = [_defects(), _small_tiled()]
    a = fse.Context(0, arena_bytes=256 << 20)
    b = fse.Context(0, arena_bytes=256 << 20)
    try:
        a.set_option(fse.OPT_F32_LAYOUT, 1)
        a.set_option(fse.OPT_F64_WARPS, 6)
        b.set_option(fse.OPT_F32_LAYOUT, 3)
        b.set_option(fse.OPT_F32_UNROLL, 2)
        b.set_option(fse.OPT_F64_WARPS, 6)
        b.set_option(fse.OPT_F64_UNROLL, 2)
        ra, _ = run_gpu(a, jobs)
        rb, _ = run_gpu(b, jobs)
        ra2, _ = run_gpu(a, jobs)  # a's choice survives b's calls
        a.set_option(fse.OPT_KERNEL_TIMING, 1)
        b.set_option(fse.OPT_KERNEL_TIMING, 1)
        run_gpu(a, jobs)
        run_gpu(b, jobs)
        assert len(a.class_times()) == 1 and len(b.class_times()) == 1  # each records its own calls
        for x, y, z in zip(ra, rb, ra2):
            assert (x["out"] == y["out"]).all() and (x["g"] == y["g"]).all()
            assert (x["out"] == z["out"]).all() and (x["g"] == z["g"]).all()
    finally:
        a.close()
        b.close()


def test_invalid_jobs_rejected(ctx):
    import torch
    img = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    for bad in [dict(fft=16), dict(fft=32, border=16), dict(K=300), dict(rho=0.0), dict(gamma=2.0),
                dict(block=0), dict(precision=16)]:
        p = dict(synth.params(4, 14, 32, 10))
        p.update(bad)
        with pytest.raises(fse.FseError) as e:
            ctx.extrapolate([fse.make_job(img, img, img, p)])
        assert e.value.code == fse.EINVAL
    p = synth.params(4, 2, 32, 10, n_tiles=23)
    img = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(fse.FseError) as e:
        ctx.extrapolate([fse.make_job(img, img, img, p)])
    assert e.value.code == fse.EDEGENERATE


def test_bounded_wait_times_out_and_context_survives(ctx):
    assert ctx.wait_probe(20000) == fse.ETIMEOUT
    job = synth.plain_64()[0]
    got, st = run_gpu(ctx, [job])
    assert st["lost_blocks"] == 26


def test_autotune_picks_a_valid_configuration(ctx, oracle_lib, tmp_path):
    import torch
    jobs = [_small_tiled(), _defects()]
    dev = torch.device("cuda", 0)
    keep, cj, outs = [], [], []
    for j in jobs:
        img = torch.from_numpy(j["image"]).to(dev)
        msk = torch.from_numpy(j["mask"]).to(dev)
        out = torch.empty_like(img)
        keep += [img, msk]
        outs.append(out)
        cj.append(fse.make_job(img, msk, out, j["params"]))
    path = str(tmp_path / "tune.txt")
    c = fse.Context(0, arena_bytes=256 << 20, tune_cache=path)
    try:
        trace = c.autotune(cj, reps=2)
        assert len(trace) >= 3
        assert {int(t[0]) for t in trace} == {-1, 0, 1}  # both classes, then the class launch
        got, _ = run_gpu(c, jobs)
        for j, g in zip(jobs, got):
            _fp32_check(oracle_lib, j, g)
        with open(path) as f:
            lines = f.read().splitlines()
        assert len(lines) >= 3
    finally:
        c.close()
        ctx.set_option(fse.OPT_F64_WARPS, 0)
    c2 = fse.Context(0, arena_bytes=256 << 20, tune_cache=path)  # reads the cache back
    got, _ = run_gpu(c2, jobs)
    c2.close()
    ctx.set_option(fse.OPT_F64_WARPS, 0)
    for j, g in zip(jobs, got):
        _fp32_check(oracle_lib, j, g)


def test_vertical_tiling_fp64_sequence_and_fp32(ctx, oracle_lib):
    job = _small_tiled(W=128, H=64, K=40, n_tiles=3)
    job["params"] = dict(job["params"], tiling="vertical", overlap=12)
    _seq_check(oracle_lib, ctx, job)
    got, st = run_gpu(ctx, [job])
    assert st["tiles"] == 3
    _fp32_check(oracle_lib, job, got[0])

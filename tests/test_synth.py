"""The seeded input generator (CPU): SplitMix64 against its published
definition and first outputs, and each workload against its stated recipe
(shapes, exact loss counts, parameters, determinism)."""
import numpy as np

from paper_2207_00238_gb300 import synth

M64 = (1 << 64) - 1


def splitmix64_reference(seed, n):
    """SplitMix64 as published (Steele, Lea, Flood 2014): a stateful scalar
    loop, state += golden gamma, then the two xor-shift-multiply rounds."""
    s, out = seed, []
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_first_outputs():
    # the generator's well-known first outputs for seed 0
    got = [int(x) for x in synth.Rng(0).u64(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_form_equals_stateful_form():
    for seed in (1, synth.SEED_BASE + 2, M64):
        r = synth.Rng(seed)
        got = [int(x) for x in r.u64(5)] + [int(x) for x in r.u64(4)]  # two calls continue the stream
        assert got == splitmix64_reference(seed, 9)


def test_uniform_and_choice_distinct():
    r = synth.Rng(7)
    u = r.uniform(100000, -2.0, 3.0)
    assert u.min() >= -2.0 and u.max() < 3.0 and abs(u.mean() - 0.5) < 0.02
    pick = synth.Rng(8).choice_distinct(1000, 300)
    assert len(set(pick.tolist())) == 300 and pick.min() >= 0 and pick.max() < 1000


def test_plain_64():
    (j,) = synth.plain_64()
    assert j["image"].shape == (64, 64) and j["image"].dtype == np.uint8
    flags = j["mask"].reshape(16, 4, 16, 4)
    blocks = flags.max(axis=(1, 3))
    assert blocks.sum() == 26                                # round(0.10 * 256)
    assert (flags.min(axis=(1, 3)) == blocks).all()          # whole 4x4 blocks
    p = j["params"]
    assert (p["block"], p["border"], p["fft"], p["K"]) == (4, 14, 32, 100)


def test_tiled_1024():
    (j,) = synth.tiled_1024()
    assert j["image"].shape == (1024, 1024)
    blocks = j["mask"].reshape(128, 8, 128, 8).max(axis=(1, 3))
    assert blocks.sum() == 3277                              # round(0.20 * 16384)
    p = j["params"]
    assert (p["block"], p["border"], p["fft"], p["K"], p["n_tiles"], p["overlap"]) == (8, 16, 64, 200, 16, 32)


def test_block_mask_burst_share():
    rng = synth.Rng(11)
    mask, flags = synth.block_mask(256, 192, 8, 200, rng)
    assert flags.sum() == 200 and mask.shape == (192, 256)
    # half of the lost blocks come in runs along block rows: many horizontal neighbours
    horiz = (flags[:, 1:] & flags[:, :-1]).sum()
    assert horiz >= 60


def test_defects_4k():
    (j,) = synth.defects_4k()
    m = j["mask"]
    assert m.shape == (2160, 3840) and j["image"].shape == (2160, 3840)
    full_cols = np.flatnonzero(m.all(axis=0))
    assert len(full_cols) == 20                              # 20 column defects
    rest = m.copy()
    rest[:, full_cols] = 0
    # round(0.01 * W * H) isolated pixels, minus those that fell on a defect
    # column (about k * 20 / W = 432 of them)
    k = int(round(0.01 * 3840 * 2160))
    assert k - 3 * 432 <= rest.sum() <= k


def test_batch_recipe_small():
    jobs = synth.batch_256(n_images=6)
    assert len(jobs) == 6
    for j in jobs:
        H, W = j["image"].shape
        assert 256 <= W <= 2048 and 256 <= H <= 1536
        p = j["params"]
        assert (p["block"], p["border"], p["fft"], p["K"]) in ((4, 14, 32, 100), (8, 16, 64, 200))
        b = p["block"]
        nb = ((W + b - 1) // b) * ((H + b - 1) // b)
        lost = j["mask"][::b, ::b].sum()
        assert 0.05 * nb - 1 <= lost <= 0.50 * nb + 1


def test_serving_stream_small():
    items = list(synth.serving_stream(n_requests=5, max_area=512 * 512))
    ts = [t for t, _ in items]
    assert all(b > a for a, b in zip(ts, ts[1:]))
    for _, j in items:
        H, W = j["image"].shape
        assert W >= H and W * H >= 16 * 16
        assert 100 <= j["params"]["K"] <= 200 and j["params"]["fft"] == 64


def test_deterministic():
    a = synth.tiled_1024(W=128, H=96, K=20, n_tiles=4)[0]
    b = synth.tiled_1024(W=128, H=96, K=20, n_tiles=4)[0]
    assert (a["image"] == b["image"]).all() and (a["mask"] == b["mask"]).all()
    c = synth.tiled_1024(seed=synth.SEED_BASE + 9, W=128, H=96, K=20, n_tiles=4)[0]
    assert not (a["image"] == c["image"]).all()


def test_burst_flags_exact_count_and_runs():
    for (nbx, nby, n) in ((40, 30, 1), (40, 30, 300), (40, 30, 1200), (7, 3, 21), (960, 540, 50000)):
        f = synth.burst_flags(nbx, nby, n, synth.Rng(synth.SEED_BASE + nbx + n))
        assert f.shape == (nby, nbx) and f.dtype == bool
        assert int(f.sum()) == min(n, nbx * nby)
    # at 10 % loss about half the lost blocks sit in horizontal runs of >= 2
    f = synth.burst_flags(200, 100, 2000, synth.Rng(synth.SEED_BASE + 9))
    left = np.zeros_like(f)
    left[:, 1:] = f[:, :-1]
    right = np.zeros_like(f)
    right[:, :-1] = f[:, 1:]
    in_run = f & (left | right)
    assert 0.35 < in_run.sum() / f.sum() < 0.75


def test_serving_requests_are_fresh_and_follow_the_workload():
    tex = [synth.image(640, 480, synth.Rng(synth.SEED_BASE + 1), structure=True)]
    items = list(synth.serving_requests(tex, n_requests=50, max_area=640 * 480))
    t = np.array([a for a, _ in items])
    assert (np.diff(t) > 0).all()
    seen = set()
    for _, spec in items:
        job = synth.materialise(tex, spec)
        H, W = job["image"].shape
        assert job["mask"].shape == (H, W) and job["image"].flags["C_CONTIGUOUS"]
        assert 100 <= job["params"]["K"] <= 200 and job["params"]["fft"] == 64
        lost = job["mask"].reshape(-1).mean()
        assert 0.0 < lost <= 0.31 + 64.0 / (W * H)
        seen.add((spec["x0"], spec["y0"], W, H))
    assert len(seen) == len(items)

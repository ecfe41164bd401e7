"""Pins for the oracle's FSE arithmetic (Sec. II; greedy weighted model fit).

Each test checks the oracle against something other than itself: a closed
form, an exact energy identity, numpy's FFT, or an independent brute-force
pipeline on tiny inputs.
"""
import numpy as np
import pytest

from tests import brute_fse


def _iso(S, b, B, rho):
    m, n = np.mgrid[0:S, 0:S]
    mc = B + (b - 1) / 2
    return rho ** np.sqrt((m - mc) ** 2 + (n - mc) ** 2)


def _rand_support(rng, S, lost_frac=0.3):
    w = rng.uniform(0.05, 1.0, (S, S)) * (rng.uniform(size=(S, S)) > lost_frac)
    r = rng.uniform(0, 255, (S, S)) * (w > 0)
    return w, r


@pytest.mark.parametrize("S,F", [(8, 8), (6, 8), (12, 16), (10, 16)])
def test_projections_match_numpy_fft(oracle_lib, S, F):
    """K iterations against the numpy-FFT brute force: same selected bins,
    same coefficients (the separable direct sums equal fft2 of the zero-padded
    weighted residual)."""
    rng = np.random.default_rng(S * 100 + F)
    for _ in range(3):
        w, r = _rand_support(rng, S)
        res = oracle_lib.fse_fit(w, r, F, 25, 0.7)
        useq, c, rr = brute_fse.fit(w, r, F, 25, 0.7)
        assert list(res["useq"]) == useq
        np.testing.assert_allclose(res["c"], c, rtol=0, atol=1e-9 * np.abs(c).max())
        np.testing.assert_allclose(res["r"], rr, rtol=0, atol=1e-8 * np.abs(r).max())


def test_first_projection_is_argmax_of_fft(oracle_lib):
    rng = np.random.default_rng(3)
    S, F, gamma = 32, 32, 0.5
    w, r = _rand_support(rng, S, 0.1)
    res = oracle_lib.fse_fit(w, r, F, 1, gamma)
    p = np.fft.fft2(np.pad(w * r, ((0, F - S), (0, F - S))))
    E = np.abs(p) ** 2
    u = int(res["useq"][0])
    assert E.ravel()[u] >= (1 - 1e-9) * E.max()
    u1, u2 = divmod(u, F)
    assert abs(res["c"][u1, u2] - gamma * p[u1, u2] / w.sum()) < 1e-9 * abs(p[u1, u2])


@pytest.mark.parametrize("v", [(0, 0), (3, 5), (31, 1), (16, 16)])
def test_complex_exponential_recovered_in_one_iteration(oracle_lib, v):
    """r = A phi_v on a fully known support with gamma = 1: u = v, c_v = A and
    the residual vanishes (closed form of one weighted projection)."""
    S = F = 32
    w = _iso(S, 4, 14, 0.8)
    m, n = np.mgrid[0:S, 0:S]
    A = 37.5 - 12.25j
    r = A * np.exp(2j * np.pi * (v[0] * m + v[1] * n) / F)
    res = oracle_lib.fse_fit(w, r, F, 1, 1.0)
    assert res["useq"][0] == v[0] * F + v[1]
    assert abs(res["c"][v] - A) < 1e-12 * abs(A)
    assert np.abs(res["r"]).max() < 1e-11 * abs(A)


@pytest.mark.parametrize("gamma,K", [(0.5, 100), (0.3, 17), (1.5, 9)])
def test_constant_signal_closed_form(oracle_lib, gamma, K):
    """Constant A: bin 0 wins every iteration (|W(k)| < W(0) for k != 0) and
    the model is A (1 - (1 - gamma)^K)."""
    S, F = 40, 64
    w = _iso(S, 8, 16, 0.8)
    w[16:24, 16:24] = 0  # the lost block itself
    A = 117.0
    res = oracle_lib.fse_fit(w, np.full((S, S), A), F, K, gamma)
    assert (res["useq"] == 0).all()
    expect = A * (1 - (1 - gamma) ** K)
    assert abs(oracle_lib.fse_model(res["c"], 18, 19) - expect) < 1e-9 * A


def test_energy_decrease_identity(oracle_lib):
    """sum w |r|^2 drops by exactly gamma (2 - gamma) |p_u|^2 / W0 per iteration;
    one K-iteration call equals K chained one-iteration calls."""
    rng = np.random.default_rng(11)
    S, F, gamma, K = 20, 32, 0.6, 30
    w, r0 = _rand_support(rng, S)
    full = oracle_lib.fse_fit(w, r0, F, K, gamma)
    W0 = w.sum()
    r = r0.astype(complex)
    c_acc = np.zeros((F, F), complex)
    for it in range(K):
        step = oracle_lib.fse_fit(w, r, F, 1, gamma)
        u = int(step["useq"][0])
        assert u == full["useq"][it]
        dlt = step["c"].ravel()[u]
        p_u = dlt * W0 / gamma
        drop = step["energy"][0] - step["energy"][1]
        assert abs(drop - gamma * (2 - gamma) * abs(p_u) ** 2 / W0) <= 1e-9 * step["energy"][0]
        assert abs(step["energy"][0] - full["energy"][it]) <= 1e-9 * full["energy"][0]
        assert drop >= 0
        c_acc += step["c"]
        r = step["r"]
    np.testing.assert_allclose(c_acc, full["c"], atol=1e-9 * np.abs(full["c"]).max())


def test_real_sinusoid_recovered_in_lost_block(oracle_lib):
    """An on-grid real sinusoid (+ offset) with the central 4x4 block lost is
    recovered at the lost pixels to rounding after K = 200."""
    S = F = 32
    m, n = np.mgrid[0:S, 0:S]
    w = _iso(S, 4, 14, 0.8)
    lost = (m >= 14) & (m < 18) & (n >= 14) & (n < 18)
    w[lost] = 0
    f = 20 * np.cos(2 * np.pi * (3 * m + 5 * n) / F + 0.4) + 7
    res = oracle_lib.fse_fit(w, np.where(lost, 0, f), F, 200, 0.5)
    err = max(abs(oracle_lib.fse_model(res["c"], mm, nn) - f[mm, nn])
              for mm in range(14, 18) for nn in range(14, 18))
    assert err < 1e-6 * 20


def test_empty_support(oracle_lib):
    res = oracle_lib.fse_fit(np.zeros((8, 8)), np.ones((8, 8)), 8, 5, 0.5)
    assert res["W0"] == 0 and np.abs(res["c"]).max() == 0


def _tiny_case(seed, W, H, b, lost_frac):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    img = np.clip(128 + 40 * np.sin(x / 5.0) + 30 * np.cos(y / 7.0) + rng.normal(0, 3, (H, W)), 0, 255)
    img = np.rint(img).astype(np.uint8)
    nby, nbx = -(-H // b), -(-W // b)
    flags = rng.uniform(size=(nby, nbx)) < lost_frac
    mask = np.kron(flags, np.ones((b, b), np.uint8))[:H, :W].astype(np.uint8)
    # a few isolated defect pixels as well
    mask[rng.integers(0, H, 5), rng.integers(0, W, 5)] = 1
    return img, mask


@pytest.mark.parametrize("order", ["phased", "raster", "independent"])
@pytest.mark.parametrize("N,d", [(1, 0), (3, 4), (4, 6)])
def test_whole_pipeline_matches_brute_force(oracle_lib, order, N, d):
    """Tiling, block order, staging with rho / delta weights, model and merge
    against the independent sequential brute force on tiny images."""
    W, H, b, B, F, K = 30, 22, 4, 3, 16, 12
    img, mask = _tiny_case(N * 10 + d, W, H, b, 0.35)
    res = oracle_lib.fse_image(img, mask, block=b, border=B, fft=F, K=K, rho=0.7, delta=0.4,
                               gamma=0.6, order=order, n_tiles=N, overlap=d, report=True)
    assert res["rc"] == 0
    out, g, seqs = brute_fse.image(img, mask, b, B, F, K, 0.7, 0.4, 0.6, order, N, d)
    lost = mask > 0
    np.testing.assert_allclose(res["g"][lost], g[lost], rtol=0, atol=1e-9)
    assert (res["out"] == out).all()
    got = {(int(t), int(i), int(j)): list(s) for (t, i, j, _), s in zip(res["blocks"], res["useq"])}
    assert got == {k: list(v) for k, v in seqs.items()}


def test_all_known_is_identity(oracle_lib):
    img, _ = _tiny_case(1, 40, 30, 4, 0)
    res = oracle_lib.fse_image(img, np.zeros_like(img), block=4, border=6, fft=16, K=10,
                               n_tiles=3, overlap=4)
    assert res["rc"] == 0 and (res["out"] == img).all() and res["stats"]["processed"] == 0


def test_phased_parallel_equals_literal_sequential(oracle_lib):
    """Blocks of one PHASED phase never read each other's pixels, so running a
    phase concurrently and committing it at once equals the literal one-by-one
    sequence, bit for bit."""
    img, mask = _tiny_case(5, 96, 80, 8, 0.4)
    kw = dict(block=8, border=16, fft=64, K=20, n_tiles=2, overlap=16, order="phased")
    a = oracle_lib.fse_image(img, mask, threads=8, literal_seq=False, **kw)
    b = oracle_lib.fse_image(img, mask, threads=1, literal_seq=True, **kw)
    lost = mask > 0
    assert (a["g"][lost] == b["g"][lost]).all()
    assert (a["out"] == b["out"]).all()


def test_output_ownership(oracle_lib):
    """Every lost pixel of the image receives a value from exactly its owner
    tile (finite g), every known pixel is copied."""
    img, mask = _tiny_case(9, 70, 50, 4, 0.3)
    res = oracle_lib.fse_image(img, mask, block=4, border=6, fft=16, K=8, n_tiles=5, overlap=6)
    lost = mask > 0
    assert np.isfinite(res["g"][lost]).all()
    assert np.isnan(res["g"][~lost]).all()
    assert (res["out"][~lost] == img[~lost]).all()


def test_invalid_params(oracle_lib):
    img = np.zeros((16, 16), np.uint8)
    bad = [dict(fft=8), dict(rho=0.0), dict(rho=1.5), dict(gamma=2.0), dict(gamma=0.0), dict(block=0)]
    for b in bad:
        kw = dict(block=4, border=4, fft=16, K=4)
        kw.update(b)
        assert oracle_lib.fse_image(img, img, **kw)["rc"] == -1


def test_block_alone_equals_phase0_blocks_of_whole_image(oracle_lib):
    """The single-block routine reproduces the whole-image run on every block
    of phase 0 (no earlier reconstruction inside its support)."""
    img, mask = _tiny_case(21, 70, 54, 4, 0.3)
    kw = dict(block=4, border=6, fft=16, K=15, rho=0.75, gamma=0.6)
    res = oracle_lib.fse_image(img, mask, n_tiles=3, overlap=6, delta=0.5, report=True, **kw)
    _, tiles = oracle_lib.plan_tiles(70, 54, 3, 6)
    P = -(-6 // 4) + 1
    n = 0
    for t, I, J, _ in res["blocks"]:
        if (I % P) * P + (J % P) != 0:
            continue
        x, y, w, h, ex, ey, ew, eh = tiles[t]
        _, g = oracle_lib.fse_block_alone(img, mask, tiles[t], int(I), int(J), **kw)
        for yy in range(4):
            for xx in range(4):
                gy, gx = ey + I * 4 + yy, ex + J * 4 + xx
                if gy < ey + eh and gx < ex + ew and mask[gy, gx] and x <= gx < x + w and y <= gy < y + h:
                    assert abs(res["g"][gy, gx] - g[yy, xx]) < 1e-9
                    n += 1
    assert n > 20

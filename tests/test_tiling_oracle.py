"""Pins for the oracle's tiling (Algorithm 1, Eqs. 1-5, Sec. III)."""
import numpy as np
import pytest

from tests import brute_fse
from tests.golden.load import tiling_goldens


@pytest.mark.parametrize("key", sorted(tiling_goldens()))
def test_hand_goldens(oracle_lib, key):
    W, H, N = key
    rc, t = oracle_lib.plan_tiles(W, H, N, 0)
    assert rc == 0 and len(t) == N
    rows = tiling_goldens()[key]
    k = 0
    for (_, y, h, nc, widths) in rows:
        x = 0
        for wv in widths:
            assert tuple(t[k, :4]) == (x, y, wv, h)
            x += wv
            k += 1
        assert x == W and len(widths) == nc
    assert k == N


def test_exact_half_rounding(oracle_lib):
    # 64x25, N=16: sqrt(N*H/W) = 2.5 exactly, Eq. (2) rounds half up to 3 rows
    # (float half-even rounding would give 2).
    _, t = oracle_lib.plan_tiles(64, 25, 16, 0)
    assert len(set(t[:, 1].tolist())) == 3


def test_degenerate_last_row(oracle_lib):
    # 32x32, N=23: n_R = 5, heights 10,10,10,7 leave -5 for the last row.
    rc, _ = oracle_lib.plan_tiles(32, 32, 23, 0)
    assert rc == -2


def test_invalid(oracle_lib):
    for args in [(0, 10, 1, 0), (10, 0, 1, 0), (10, 10, 0, 0), (10, 10, 1, -1)]:
        assert oracle_lib.plan_tiles(*args)[0] == -1


def _check_partition(W, H, N, d, t):
    cover = np.zeros((H, W), np.int32)
    for x, y, w, h, ex, ey, ew, eh in t:
        assert w > 0 and h > 0
        cover[y:y + h, x:x + w] += 1
        # extended tile = core grown by d, clipped to the image
        assert ex == max(0, x - d) and ey == max(0, y - d)
        assert ex + ew == min(W, x + w + d) and ey + eh == min(H, y + h + d)
    assert (cover == 1).all()          # every pixel owned by exactly one core tile
    assert int((t[:, 2] * t[:, 3]).sum()) == W * H


def test_partition_sweep_matches_brute_force(oracle_lib):
    rng = np.random.default_rng(7)
    n_deg = 0
    for _ in range(400):
        W = int(rng.integers(1, 300))
        H = int(rng.integers(1, 300))
        N = int(rng.integers(1, 40))
        d = int(rng.integers(0, 40))
        rc, t = oracle_lib.plan_tiles(W, H, N, d)
        bf = brute_fse.tiles(W, H, N, d)
        if bf is None:
            assert rc == -2
            n_deg += 1
            continue
        assert rc == 0
        assert [tuple(map(int, r)) for r in t] == bf
        _check_partition(W, H, N, d, t)
    assert n_deg > 0  # the sweep does reach the degenerate case


def test_portrait_is_transposed_landscape(oracle_lib):
    _, a = oracle_lib.plan_tiles(480, 1024, 22, 32)
    _, b = oracle_lib.plan_tiles(1024, 480, 22, 32)
    assert (a[:, [1, 0, 3, 2, 5, 4, 7, 6]] == b).all()


def test_compact_equal_area(oracle_lib):
    # Sec. III goals 1-2: tiles of about equal size, compact
    for W, H, N in [(6024, 4024, 32), (1024, 480, 22), (3840, 2160, 16), (7680, 4320, 64)]:
        _, t = oracle_lib.plan_tiles(W, H, N, 0)
        a = t[:, 2] * t[:, 3]
        assert a.max() / a.min() < 1.1
        assert (np.maximum(t[:, 2], t[:, 3]) / np.minimum(t[:, 2], t[:, 3])).max() < 2.0


def test_vertical_stripes_hand_golden(oracle_lib):
    # 1024 = 22 * 46 + 12: the first 12 stripes are 47 wide, the other 10 are 46
    rc, t = oracle_lib.plan_tiles(1024, 480, 22, 0, "vertical")
    assert rc == 0
    assert t[:, 2].tolist() == [47] * 12 + [46] * 10
    assert (t[:, 1] == 0).all() and (t[:, 3] == 480).all()
    assert t[:, 0].tolist() == list(np.cumsum([0] + [47] * 12 + [46] * 9))


def test_vertical_overlap_exceeds_alg1(oracle_lib):
    """Sec. III: stripes have the longer boundary, so their overlap stripes
    add more processed pixels than the compact tiles of Algorithm 1."""
    for W, H, N, d in [(6024, 4024, 32, 32), (1024, 480, 22, 32), (3840, 2160, 16, 32)]:
        areas = {}
        for tiling in ["alg1", "vertical"]:
            _, t = oracle_lib.plan_tiles(W, H, N, d, tiling)
            areas[tiling] = int((t[:, 6] * t[:, 7]).sum())
        assert areas["vertical"] > areas["alg1"] > W * H

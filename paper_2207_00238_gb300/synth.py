"""Seeded synthetic inputs: 8-bit images and loss masks.

The paper evaluates on three 6024x4024 photographs with two masks (14 % and
62 % lost, Sec. IV); none of them is available here.  These generators stand in
for them with the shapes the paper's workloads have: 8-bit grey images with
smooth structure, edges and texture; isolated and connected lost blocks;
isolated defect pixels and column defects (defect-pixel compensation, Sec. I).

Randomness comes from SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), a
counter-based generator: output i of a stream with seed s is mix(s + (i+1)*G).
Gaussian noise uses the Box-Muller transform.  This module holds no part of
the extrapolation method; it only makes inputs, identically for the oracle and
for the CUDA path.
"""
import math

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

SEED_BASE = 0x5EED0000


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Rng:
    """SplitMix64 stream (counter-based, vectorised)."""

    def __init__(self, seed):
        self.seed = int(seed) & _MASK64
        self.count = 0

    def u64(self, n):
        idx = np.arange(self.count + 1, self.count + 1 + n, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            return _mix(np.uint64(self.seed) + idx * _G)

    def uniform(self, n, lo=0.0, hi=1.0):
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def randint(self, n, lo, hi):
        """Integers uniform in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + (self.u64(n) % np.uint64(span)).astype(np.int64)

    def normal(self, n):
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0, 1]
        z = np.concatenate([rad * np.cos(2 * math.pi * u2), rad * np.sin(2 * math.pi * u2)])
        return z[:n]

    def choice_distinct(self, n_pool, k):
        """k distinct integers from range(n_pool): partial Fisher-Yates."""
        k = min(k, n_pool)
        r = self.u64(k)
        perm = {}
        out = np.empty(k, np.int64)
        for i in range(k):
            j = i + int(r[i] % np.uint64(n_pool - i))
            vi, vj = perm.get(i, i), perm.get(j, j)
            perm[i], perm[j] = vj, vi
            out[i] = vj
        return out


def _to_u8(x):
    return np.rint(np.clip(x, 0.0, 255.0)).astype(np.uint8)


def image(W, H, rng, structure=False):
    """128 + linear gradient + 6 random 2-D sinusoids (+ 8 rectangles and 4 step
    edges when ``structure``) + Gaussian noise sigma=2, clipped and rounded."""
    xs = np.arange(W, dtype=np.float64)
    ys = np.arange(H, dtype=np.float64)
    gx = rng.uniform(1, -32, 32)[0] / W
    gy = rng.uniform(1, -32, 32)[0] / H
    img = 128.0 + gx * (xs[None, :] - W / 2) + gy * (ys[:, None] - H / 2)
    a = rng.uniform(6, 8, 24)
    fx = rng.uniform(6, -0.15, 0.15)
    fy = rng.uniform(6, -0.15, 0.15)
    ph = rng.uniform(6, 0, 2 * math.pi)
    for i in range(6):
        # a cos(2 pi (fx x + fy y) + ph), evaluated separably
        cx, sx = np.cos(2 * math.pi * fx[i] * xs), np.sin(2 * math.pi * fx[i] * xs)
        cy = np.cos(2 * math.pi * fy[i] * ys + ph[i])
        sy = np.sin(2 * math.pi * fy[i] * ys + ph[i])
        img += a[i] * (cy[:, None] * cx[None, :] - sy[:, None] * sx[None, :])
    y = ys[:, None]
    x = xs[None, :]
    if structure:
        for _ in range(8):
            rw = int(round(rng.uniform(1, 0.05, 0.30)[0] * W))
            rh = int(round(rng.uniform(1, 0.05, 0.30)[0] * H))
            x0 = int(rng.randint(1, 0, max(W - rw, 0))[0])
            y0 = int(rng.randint(1, 0, max(H - rh, 0))[0])
            img[y0:y0 + rh, x0:x0 + rw] += rng.uniform(1, -40, 40)[0]
        for _ in range(4):
            px, py = rng.uniform(1, 0, W)[0], rng.uniform(1, 0, H)[0]
            th = rng.uniform(1, 0, 2 * math.pi)[0]
            step = rng.uniform(1, -30, 30)[0]
            img += step * (((x - px) * math.cos(th) + (y - py) * math.sin(th)) > 0)
    img += 2.0 * rng.normal(W * H).reshape(H, W)
    return _to_u8(img)


def block_mask(W, H, b, n_lost, rng, burst_frac=0.5):
    """Exactly n_lost distinct b x b blocks of the image grid lost: a share
    ``burst_frac`` as bursts (runs of 2..8 consecutive blocks along a block
    row), the rest isolated uniform picks.  Returns (mask u8, lost block flags)."""
    nby, nbx = (H + b - 1) // b, (W + b - 1) // b
    nb = nbx * nby
    n_lost = min(n_lost, nb)
    lost = np.zeros(nb, bool)
    n_burst = int(round(n_lost * burst_frac))
    cnt = 0
    guard = 0
    while cnt < n_burst and guard < 100 * nb:
        guard += 1
        start = int(rng.randint(1, 0, nb - 1)[0])
        L = int(rng.randint(1, 2, 8)[0])
        r, c = divmod(start, nbx)
        for cc in range(c, min(c + L, nbx)):
            if cnt >= n_burst:
                break
            k = r * nbx + cc
            if not lost[k]:
                lost[k] = True
                cnt += 1
    free = np.flatnonzero(~lost)
    pick = rng.choice_distinct(len(free), n_lost - cnt)
    lost[free[pick]] = True
    flags = lost.reshape(nby, nbx)
    mask = np.kron(flags.astype(np.uint8), np.ones((b, b), np.uint8))[:H, :W]
    return np.ascontiguousarray(mask), flags


def defect_mask(W, H, frac_pixels, n_columns, rng):
    """round(frac*W*H) distinct isolated defect pixels + n_columns distinct
    full-height column defects."""
    mask = np.zeros(H * W, np.uint8)
    k = int(round(frac_pixels * W * H))
    mask[rng.choice_distinct(W * H, k)] = 1
    mask = mask.reshape(H, W)
    cols = rng.choice_distinct(W, n_columns)
    mask[:, cols] = 1
    return mask


# ---------------------------------------------------------------------------
# The five workloads.  Each job: dict(image, mask, params) with params named as
# in the C ABI (block, border, fft, K, rho, delta, gamma, order, n_tiles, overlap).
# ---------------------------------------------------------------------------

DEFAULTS = dict(rho=0.8, delta=0.5, gamma=0.5, order="phased")


def params(block, border, fft, K, n_tiles=1, overlap=32, **kw):
    p = dict(DEFAULTS, block=block, border=border, fft=fft, K=K, n_tiles=n_tiles, overlap=overlap)
    p.update(kw)
    return p


def plain_64(seed=SEED_BASE + 1):
    """64x64 image, exactly 26 (10 %) of the 4x4 blocks lost at random,
    b=4, B=14 (32x32 support), F=32, K=100."""
    rng = Rng(seed)
    img = image(64, 64, rng)
    nb = 16 * 16
    flags = np.zeros(nb, np.uint8)
    flags[rng.choice_distinct(nb, int(round(0.10 * nb)))] = 1
    mask = np.kron(flags.reshape(16, 16), np.ones((4, 4), np.uint8))
    return [dict(image=img, mask=np.ascontiguousarray(mask), params=params(4, 14, 32, 100))]


def tiled_1024(seed=SEED_BASE + 2, W=1024, H=1024, K=200, n_tiles=16):
    """1024x1024 image with edges and rectangles, 20 % of the 8x8 blocks lost
    (half bursts along block rows, half isolated), b=8, B=16, F=64, K=200,
    16 tiles of Algorithm 1 with overlap d=32."""
    rng = Rng(seed)
    img = image(W, H, rng, structure=True)
    nb = ((W + 7) // 8) * ((H + 7) // 8)
    mask, _ = block_mask(W, H, 8, int(round(0.20 * nb)), rng)
    return [dict(image=img, mask=mask, params=params(8, 16, 64, K, n_tiles=n_tiles, overlap=32))]


def defects_4k(seed=SEED_BASE + 3, W=3840, H=2160):
    """3840x2160 image, 1 % isolated defect pixels + 20 full-height column
    defects; b=4, B=14, F=32, K=100, one tile."""
    rng = Rng(seed)
    img = image(W, H, rng, structure=True)
    mask = defect_mask(W, H, 0.01, 20, rng)
    return [dict(image=img, mask=mask, params=params(4, 14, 32, 100))]


def batch_256(seed=SEED_BASE + 4, n_images=256, max_w=2048, max_h=1536):
    """n_images of uneven size (W in 256..max_w, H in 256..max_h), loss rate
    U(5 %, 50 %) of the blocks, block 4 (F=32, B=14, K=100) or 8 (F=64, B=16,
    K=200) with p=1/2, isolated/burst 50/50, truncated supports at borders."""
    rng = Rng(seed)
    jobs = []
    for i in range(n_images):
        W = int(rng.randint(1, 256, max_w)[0])
        H = int(rng.randint(1, 256, max_h)[0])
        rate = rng.uniform(1, 0.05, 0.50)[0]
        big = bool(rng.randint(1, 0, 1)[0])
        b, B, F, K = (8, 16, 64, 200) if big else (4, 14, 32, 100)
        sub = Rng(seed * 1000003 + i)
        img = image(W, H, sub, structure=True)
        nb = ((W + b - 1) // b) * ((H + b - 1) // b)
        mask, _ = block_mask(W, H, b, int(round(rate * nb)), sub)
        jobs.append(dict(image=img, mask=mask, params=params(b, B, F, K)))
    return jobs


def serving_stream(seed=SEED_BASE + 5, n_requests=2200, rate_hz=200.0,
                   min_area=128 * 128, max_area=7680 * 4320):
    """Poisson arrivals (exponential gaps, mean 1/rate_hz), area log-uniform in
    [min_area, max_area], landscape aspect U(1, 16/9), loss U(1 %, 30 %) of the
    8x8 blocks (isolated/burst 50/50), K uniform in 100..200, F=64, B=16.
    Yields (arrival_s, job) lazily so large streams stay cheap."""
    rng = Rng(seed)
    t = 0.0
    for k in range(n_requests):
        t += -math.log1p(-rng.uniform(1)[0]) / rate_hz
        area = math.exp(rng.uniform(1, math.log(min_area), math.log(max_area))[0])
        aspect = rng.uniform(1, 1.0, 16.0 / 9.0)[0]
        W = max(16, int(round(math.sqrt(area * aspect))))
        H = max(16, int(round(math.sqrt(area / aspect))))
        rate = rng.uniform(1, 0.01, 0.30)[0]
        K = int(rng.randint(1, 100, 200)[0])
        sub = Rng(seed * 1000003 + k)
        img = image(W, H, sub, structure=True)
        nb = ((W + 7) // 8) * ((H + 7) // 8)
        mask, _ = block_mask(W, H, 8, max(1, int(round(rate * nb))), sub)
        yield t, dict(image=img, mask=mask, params=params(8, 16, 64, K))



def burst_flags(nbx, nby, n_lost, rng, burst_frac=0.5):
    """Vectorised lost-block flags for large grids: about ``burst_frac`` of the
    n_lost blocks in runs of 2..8 along a block row (runs drawn at once, clipped
    at the row end, overlaps merged), the rest isolated uniform picks among the
    blocks still present.  Exactly min(n_lost, nbx*nby) flags are set."""
    nb = nbx * nby
    n_lost = min(int(n_lost), nb)
    lost = np.zeros(nb, bool)
    n_burst = int(round(n_lost * burst_frac))
    if n_burst > 0:
        runs = max(1, n_burst // 5)
        start = rng.randint(runs, 0, nb - 1)
        L = rng.randint(runs, 2, 8)
        r, c = np.divmod(start, nbx)
        off = np.arange(8)
        cc = c[:, None] + off[None, :]
        ok = (off[None, :] < L[:, None]) & (cc < nbx)
        k = np.unique((r[:, None] * nbx + cc)[ok])
        if len(k) > n_burst:  # drop a random excess, not the last rows
            k = k[np.argpartition(rng.u64(len(k)), n_burst - 1)[:n_burst]]
        lost[k] = True
    rest = n_lost - int(lost.sum())
    if rest > 0:
        free = np.flatnonzero(~lost)
        # distinct picks by sorting random keys (vectorised; no Python loop)
        pick = np.argpartition(rng.u64(len(free)), rest - 1)[:rest] if rest < len(free) else np.arange(len(free))
        lost[free[pick]] = True
    return lost.reshape(nby, nbx)


def expand_flags(flags, b, W, H):
    """Pixel mask (u8, 1 = lost) of a b x b block-flag grid, cropped to H x W."""
    return np.ascontiguousarray(np.repeat(np.repeat(flags.astype(np.uint8), b, 0), b, 1)[:H, :W])


def serving_textures(n=2, seed=SEED_BASE + 6, W=7680, H=4320):
    """Large seeded images from which fresh serving requests take their content."""
    return [image(W, H, Rng(seed * 1009 + i), structure=True) for i in range(n)]


def serving_requests(textures, n_requests=2000, seed=SEED_BASE + 7, rate_hz=200.0,
                     min_area=128 * 128, max_area=7680 * 4320):
    """Fresh requests of the serving workload, drawn per request like
    serving_stream (Poisson arrivals, log-uniform area, aspect U(1, 16/9), loss
    U(1 %, 30 %) of the 8x8 blocks, isolated/burst 50/50, K in 100..200, F=64,
    B=16).  The pixels of each request are a crop, at a position drawn per
    request, of one of ``textures`` (so generating a request costs a copy, not
    a synthesis); its block flags are drawn fresh.  Yields (arrival_s, spec)
    with spec = dict(tex, x0, y0, W, H, flags, K): materialise() turns it into
    a job."""
    rng = Rng(seed)
    t = 0.0
    TH, TW = textures[0].shape
    for k in range(n_requests):
        t += -math.log1p(-rng.uniform(1)[0]) / rate_hz
        area = math.exp(rng.uniform(1, math.log(min_area), math.log(max_area))[0])
        aspect = rng.uniform(1, 1.0, 16.0 / 9.0)[0]
        W = min(TW, max(16, int(round(math.sqrt(area * aspect)))))
        H = min(TH, max(16, int(round(math.sqrt(area / aspect)))))
        rate = rng.uniform(1, 0.01, 0.30)[0]
        K = int(rng.randint(1, 100, 200)[0])
        ti = int(rng.randint(1, 0, len(textures) - 1)[0])
        x0 = int(rng.randint(1, 0, TW - W)[0])
        y0 = int(rng.randint(1, 0, TH - H)[0])
        nbx, nby = (W + 7) // 8, (H + 7) // 8
        flags = burst_flags(nbx, nby, max(1, int(round(rate * nbx * nby))), Rng(seed * 1000003 + k))
        yield t, dict(tex=ti, x0=x0, y0=y0, W=W, H=H, flags=flags, K=K)


def materialise(textures, spec):
    """The job of a serving_requests spec: contiguous image crop, pixel mask."""
    W, H = spec["W"], spec["H"]
    img = np.ascontiguousarray(textures[spec["tex"]][spec["y0"]:spec["y0"] + H, spec["x0"]:spec["x0"] + W])
    return dict(image=img, mask=expand_flags(spec["flags"], 8, W, H), params=params(8, 16, 64, spec["K"]))

CONFIGS = {
    "plain_64": plain_64,
    "tiled_1024": tiled_1024,
    "defects_4k": defects_4k,
    "batch_256": batch_256,
}

"""Brute-force FSE for tiny inputs, written independently of the C oracle.

Used only to pin the oracle: projections come from numpy's FFT of the
zero-padded weighted residual (a library routine) instead of the oracle's
explicit direct sums; the tiling uses exact rational arithmetic; the
processing order, staging and merge are plain Python loops.
"""
from fractions import Fraction
import math

import numpy as np


def tiles(W, H, N, d):
    """Algorithm 1 (Sec. III) with exact rationals; returns list of
    (x, y, w, h, ex, ey, ew, eh) or None if a tile is degenerate."""
    swap = W < H
    if swap:
        W, H = H, W
    x2 = Fraction(N * H, W)                       # (sqrt(N/r))^2, r = W/H
    nR = 0
    while Fraction(2 * nR + 1, 2) ** 2 <= x2:     # round half up of sqrt(x2)
        nR += 1
    nR = max(1, nR)
    out, y = [], 0
    for i in range(1, nR + 1):
        nC = math.ceil(N / nR) if i <= N % nR else N // nR
        h = (H * nC) // N + ((H * nC) % N) // nR
        if i == nR:
            h = H - y
        x = 0
        for j in range(1, nC + 1):
            w = math.ceil(W / nC) if j <= W % nC else W // nC
            if w <= 0 or h <= 0:
                return None
            ex, ey = max(0, x - d), max(0, y - d)
            t = (x, y, w, h, ex, ey, min(W, x + w + d) - ex, min(H, y + h + d) - ey)
            if swap:
                t = (t[1], t[0], t[3], t[2], t[5], t[4], t[7], t[6])
            out.append(t)
            x += w
        y += h
    return out


def fit(w, r, F, K, gamma, tau=1e-9):
    """Greedy weighted fit; returns (useq, c[F,F], residual)."""
    S = w.shape[0]
    r = r.astype(complex).copy()
    W0 = w.sum()
    c = np.zeros((F, F), complex)
    useq = []
    m, n = np.mgrid[0:S, 0:S]
    if W0 <= 0:
        return useq, c, r
    for _ in range(K):
        pad = np.zeros((F, F), complex)
        pad[:S, :S] = w * r
        p = np.fft.fft2(pad)
        E = (p.real ** 2 + p.imag ** 2).ravel()
        u = int(np.flatnonzero(E >= (1 - tau) * E.max())[0])
        useq.append(u)
        u1, u2 = divmod(u, F)
        dlt = gamma * p[u1, u2] / W0
        c[u1, u2] += dlt
        r -= dlt * np.exp(2j * np.pi * (u1 * m + u2 * n) / F)
    return useq, c, r


def model(c, m, n):
    F = c.shape[0]
    k1, k2 = np.mgrid[0:F, 0:F]
    return float(np.real(np.sum(c * np.exp(2j * np.pi * (k1 * m + k2 * n) / F))))


def image(img, mask, b, B, F, K, rho, delta, gamma, order, N, d, tau=1e-9):
    """Whole pipeline, strictly sequential, committing each block at once."""
    H, W = img.shape
    S = b + 2 * B
    out = np.where(mask > 0, 0, img).astype(np.uint8)
    g_out = np.full((H, W), np.nan)
    seqs = {}
    mc = B + (b - 1) / 2
    mm, nn = np.mgrid[0:S, 0:S]
    wiso = rho ** np.sqrt((mm - mc) ** 2 + (nn - mc) ** 2)
    P = -(-B // b) + 1
    for t, (cx, cy, cw, ch, ex, ey, ew, eh) in enumerate(tiles(W, H, N, d)):
        st = np.where(mask[ey:ey + eh, ex:ex + ew] > 0, 1, 0)      # 0 known, 1 pending, 2 done
        val = img[ey:ey + eh, ex:ex + ew].astype(float)
        blocks = []
        for I in range(-(-eh // b)):
            for J in range(-(-ew // b)):
                if (st[I * b:(I + 1) * b, J * b:(J + 1) * b] == 1).any():
                    key = ((I % P) * P + (J % P), I, J) if order == "phased" else (0, I, J)
                    blocks.append((key, I, J))
        blocks.sort()
        for _, I, J in blocks:
            w = np.zeros((S, S))
            r = np.zeros((S, S))
            for m in range(S):
                for n in range(S):
                    y, x = I * b - B + m, J * b - B + n
                    if 0 <= y < eh and 0 <= x < ew:
                        if st[y, x] == 0:
                            w[m, n], r[m, n] = wiso[m, n], val[y, x]
                        elif st[y, x] == 2 and order != "independent":
                            w[m, n], r[m, n] = delta * wiso[m, n], val[y, x]
            useq, c, _ = fit(w, r, F, K, gamma, tau)
            seqs[(t, I, J)] = useq
            ok = w.sum() > 0
            for yy in range(b):
                for xx in range(b):
                    y, x = I * b + yy, J * b + xx
                    if y >= eh or x >= ew or st[y, x] != 1:
                        continue
                    g = model(c, B + yy, B + xx) if ok else 0.0
                    if ok:
                        st[y, x], val[y, x] = 2, g
                    gx, gy = ex + x, ey + y
                    if cx <= gx < cx + cw and cy <= gy < cy + ch:
                        out[gy, gx] = int(np.rint(min(max(g, 0.0), 255.0)))
                        g_out[gy, gx] = g
    return out, g_out, seqs

"""FP64 CPU oracle for FSE on overlapping tiles -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library does not use it and
shares no code with it.

``fse_oracle.c`` holds the arithmetic (tiling per Algorithm 1 / Eqs. 1-5 of the
paper, FSE per Sec. II with explicit spatial-domain projections); this module
compiles it with gcc and marshals numpy arrays through ctypes.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fse_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libfse_oracle.so")

ORDER = {"phased": 0, "raster": 1, "independent": 2}
OK, EINVAL, EDEGENERATE = 0, -1, -2


def build(force=False):
    """Compile the oracle (plain C, -O2, OpenMP when available)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _BlkReport(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("I", ctypes.c_int32), ("J", ctypes.c_int32),
                ("status", ctypes.c_int32), ("W0", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        i32, f64 = ctypes.c_int32, ctypes.c_double
        _lib.oracle_plan_tiles.argtypes = [i32, i32, i32, i32, P(i32), i32, P(i32)]
        _lib.oracle_fse_fit.restype = f64
        _lib.oracle_fse_fit.argtypes = [P(f64), P(f64), P(f64), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, f64, f64, P(i32), P(f64), P(f64), P(f64),
                                        P(f64), P(f64)]
        _lib.oracle_fse_model.restype = f64
        _lib.oracle_fse_model.argtypes = [P(f64), P(f64), ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.oracle_fse_image.argtypes = [P(ctypes.c_uint8), P(ctypes.c_uint8), i32, i32, i32, i32,
                                          i32, i32, f64, f64, f64, i32, i32, i32, f64,
                                          P(ctypes.c_uint8), P(f64), P(_BlkReport), P(i32), i32,
                                          P(i32), i32, i32, ctypes.c_int64, P(ctypes.c_int64), i32]
        _lib.oracle_plan_vertical.argtypes = [i32, i32, i32, i32, P(i32), i32, P(i32)]
        _lib.oracle_threads.restype = ctypes.c_int
        _lib.oracle_fse_block_alone.restype = f64
        _lib.oracle_fse_block_alone.argtypes = [P(ctypes.c_uint8), P(ctypes.c_uint8)] + [i32] * 10 + \
            [f64, f64, f64, i32, i32, P(f64)]
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def threads():
    return lib().oracle_threads()


def plan_tiles(W, H, N, d, tiling="alg1"):
    """Algorithm 1 (or the vertical stripes) + overlap stripe d.  Returns
    (rc, int32 array [n, 8]): columns x, y, w, h, ex, ey, ew, eh."""
    out = np.zeros((max(N, 1), 8), np.int32)
    n = ctypes.c_int32(0)
    fn = lib().oracle_plan_vertical if tiling == "vertical" else lib().oracle_plan_tiles
    rc = fn(W, H, N, d, _ptr(out, ctypes.c_int32), max(N, 1), ctypes.byref(n))
    return rc, out[: n.value]


def fse_fit(w, r, F, K, gamma, tau=1e-9):
    """Greedy FSE fit of one S x S support.  r may be complex.
    Returns dict(W0, useq, c (complex F x F), energy (K+1), r (final residual))."""
    w = np.ascontiguousarray(w, np.float64)
    S = w.shape[0]
    r = np.asarray(r)
    rre = np.ascontiguousarray(r.real, np.float64)
    rim = np.ascontiguousarray(r.imag if np.iscomplexobj(r) else np.zeros_like(rre), np.float64)
    useq = np.zeros(max(K, 1), np.int32)
    cre = np.zeros(F * F)
    cim = np.zeros(F * F)
    energy = np.zeros(K + 1)
    ore = np.zeros(S * S)
    oim = np.zeros(S * S)
    f64 = ctypes.c_double
    W0 = lib().oracle_fse_fit(_ptr(w, f64), _ptr(rre, f64), _ptr(rim, f64), S, F, K, gamma, tau,
                              _ptr(useq, ctypes.c_int32), _ptr(cre, f64), _ptr(cim, f64),
                              _ptr(energy, f64), _ptr(ore, f64), _ptr(oim, f64))
    return dict(W0=W0, useq=useq[:K], c=(cre + 1j * cim).reshape(F, F), energy=energy,
                r=(ore + 1j * oim).reshape(S, S))


def fse_model(c, m, n):
    c = np.ascontiguousarray(c)
    F = c.shape[0]
    cre = np.ascontiguousarray(c.real.ravel(), np.float64)
    cim = np.ascontiguousarray(c.imag.ravel(), np.float64)
    return lib().oracle_fse_model(_ptr(cre, ctypes.c_double), _ptr(cim, ctypes.c_double), F, m, n)


def fse_block_alone(img, mask, tile, I, J, *, block, border, fft, K, rho=0.8, gamma=0.5,
                    tau=1e-9, **_):
    """One block (I, J) of extended tile `tile` (x, y, w, h, ex, ey, ew, eh) with
    all lost pixels pending -- what a PHASED phase-0 block sees.  Returns
    (W0, g[b, b])."""
    img = np.ascontiguousarray(img, np.uint8)
    mask = np.ascontiguousarray(mask, np.uint8)
    H, W = img.shape
    g = np.zeros(block * block)
    ex, ey, ew, eh = (int(v) for v in tile[4:8])
    W0 = lib().oracle_fse_block_alone(_ptr(img, ctypes.c_uint8), _ptr(mask, ctypes.c_uint8), W, H,
                                      ex, ey, ew, eh, block, border, fft, K, rho, gamma, tau,
                                      I, J, _ptr(g, ctypes.c_double))
    return W0, g.reshape(block, block)


def fse_image(img, mask, *, block, border, fft, K, rho=0.8, delta=0.5, gamma=0.5,
              order="phased", n_tiles=1, overlap=32, tau=1e-9, report=False, threads=0,
              literal_seq=False, max_blocks=0, tiling="alg1"):
    """Whole-image FSE on the overlapping tiles of Algorithm 1.
    Returns dict(rc, out (u8), g (f64, NaN at known pixels), stats, blocks, useq)."""
    img = np.ascontiguousarray(img, np.uint8)
    mask = np.ascontiguousarray(mask, np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), np.uint8)
    g = np.zeros((H, W), np.float64)
    stats = np.zeros(4, np.int64)
    cap = 0
    rep = useq = None
    if report:
        nbmax = sum(((int(t[6]) + block - 1) // block) * ((int(t[7]) + block - 1) // block)
                    for t in plan_tiles(W, H, n_tiles, overlap, tiling)[1])
        cap = max(nbmax, 1)
        rep = (_BlkReport * cap)()
        useq = np.zeros((cap, max(K, 1)), np.int32)
    nrep = ctypes.c_int32(0)
    rc = lib().oracle_fse_image(
        _ptr(img, ctypes.c_uint8), _ptr(mask, ctypes.c_uint8), W, H, block, border, fft, K, rho,
        delta, gamma, ORDER[order], n_tiles, overlap, tau, _ptr(out, ctypes.c_uint8),
        _ptr(g, ctypes.c_double), rep, _ptr(useq, ctypes.c_int32), cap, ctypes.byref(nrep),
        threads, int(literal_seq), max_blocks, _ptr(stats, ctypes.c_int64),
        1 if tiling == "vertical" else 0)
    res = dict(rc=rc, out=out, g=g, stats=dict(processed=int(stats[0]), empty=int(stats[1]),
                                               tiles=int(stats[2]), core_lost=int(stats[3])))
    if report:
        n = nrep.value
        res["blocks"] = np.array([(rep[i].tile, rep[i].I, rep[i].J, rep[i].status) for i in range(n)],
                                 np.int32).reshape(n, 4)
        res["W0"] = np.array([rep[i].W0 for i in range(n)])
        res["useq"] = useq[:n, :K]
    return res

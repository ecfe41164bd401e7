"""C ABI checks that need no GPU: every function declared in include/fse.h is
exported by the built library, and the library's host-side tilings match the
oracle bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2207_00238_gb300 as fse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fse.build()
    return fse.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "fse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fse_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_function_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(fse.EXPORTS) <= set(names)


@pytest.mark.parametrize("tiling", ["alg1", "vertical"])
def test_library_tiling_bit_exact_with_oracle(lib, oracle_lib, tiling):
    rng = np.random.default_rng(17)
    cases = [(1024, 480, 22, 0), (1024, 1024, 16, 32), (6024, 4024, 32, 32), (3840, 2160, 16, 8),
             (480, 1024, 22, 5), (64, 25, 16, 0)]
    cases += [(int(rng.integers(1, 3000)), int(rng.integers(1, 3000)), int(rng.integers(1, 70)),
               int(rng.integers(0, 64))) for _ in range(600)]
    n_deg = 0
    for W, H, N, d in cases:
        rc, ref = oracle_lib.plan_tiles(W, H, N, d, tiling)
        if rc != 0:
            with pytest.raises(fse.FseError) as e:
                fse.plan_tiles(W, H, N, d, tiling)
            assert e.value.code == rc
            n_deg += 1
            continue
        got = fse.plan_tiles(W, H, N, d, tiling)
        assert (got == ref).all(), (W, H, N, d)
    if tiling == "alg1":
        assert n_deg > 0


def test_tiling_errors(lib):
    for args in [(0, 10, 1, 0), (10, 10, 0, 0), (10, 10, 1, -1)]:
        with pytest.raises(fse.FseError) as e:
            fse.plan_tiles(*args)
        assert e.value.code == fse.EINVAL
    with pytest.raises(fse.FseError) as e:
        fse.plan_tiles(32, 32, 23, 0)
    assert e.value.code == fse.EDEGENERATE
    with pytest.raises(fse.FseError) as e:
        fse.plan_tiles(10, 10, 11, 0, "vertical")
    assert e.value.code == fse.EDEGENERATE


def test_last_error_is_a_string(lib):
    with pytest.raises(fse.FseError):
        fse.plan_tiles(0, 0, 0, 0)
    assert "invalid" in lib.fse_last_error().decode()


def test_binding_constants_match_header():
    """The binding's status codes, option keys and enum values equal the
    header's #defines (the two are maintained side by side)."""
    import re
    import paper_2207_00238_gb300 as fse
    hdr = open(os.path.join(ROOT, "include", "fse.h")).read()
    defs = {m.group(1): int(m.group(2))
            for m in re.finditer(r"#define FSE_(\w+)\s+\(?(-?\d+)\)?", hdr)}
    for name in ["OK", "EINVAL", "EDEGENERATE", "ENOMEM", "EBUSY", "ETIMEOUT", "ECUDA", "ENOTFOUND",
                 "ECANCELLED"]:
        assert getattr(fse, name) == defs[name], name
    for key, val in fse.ORDER.items():
        assert val == defs["ORDER_" + key.upper()], key
    for key, val in fse.TILING.items():
        assert val == defs["TILING_" + key.upper()], key
    for key, val in fse.EXEC.items():
        assert val == defs["EXEC_" + key.upper()], key
    opts = [n for n in dir(fse) if n.startswith("OPT_")]
    assert len(opts) == len([d for d in defs if d.startswith("OPT_")])
    for n in opts:
        assert getattr(fse, n) == defs[n], n

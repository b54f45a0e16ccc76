"""love_cache_load refuses any file whose header does not describe exactly the
buffers the library writes for such a cache, before it allocates or copies
anything (host logic only: these calls return LOVE_ERR_ARG without touching a
GPU).  A file that the loader accepted with a wrong size or leading dimension
would let the predict and sampler kernels read past a device buffer.

The header layout is the library's versioned cache-file format (magic
"LOVECACH", version 2); the matching GPU test saves and reloads a real cache.
"""
import ctypes as C
import struct

import numpy as np
import pytest

LOVE_ERR_ARG = 1
HDR = struct.Struct("<8sIi3q3d3d3d2d2iI7i6Q2i")   # 224 bytes, the C struct with its natural alignment
assert HDR.size == 224


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1803_06058_gb300 import _lib
    return _lib.load()


def _base():
    """A consistent header: 1-D grid of 40 points, k_eff = 10, FP32 cache with
    the mean column (ld = 12), no sampler, no gradient tables."""
    return dict(magic=b"LOVECACH", version=2, dim=1, g=[40, 1, 1], lo=[-0.1, 0.0, 0.0], h=[1 / 35, 1.0, 1.0],
                ls=[0.2, 1.0, 1.0], sf=1.0, noise=0.01, dtype=0, cache_dtype=0, flags=1, k_eff=10, ld=12, ks=0,
                ld_s=0, ld_g=0, cg_iters=5, fallback=0, bytes_rc=40 * 12 * 4, bytes_s=0, bytes_p=0, bytes_kdp=0,
                bytes_b=0, bytes_minv=0, additive=0)


def _payload_bytes(h):
    return (16 * h["k_eff"] + h["bytes_rc"] + h["bytes_s"] + h["bytes_p"] + h["bytes_kdp"] + h["bytes_b"]
            + h["bytes_minv"])


def _write(path, h, payload=None):
    hdr = HDR.pack(h["magic"], h["version"], h["dim"], *h["g"], *h["lo"], *h["h"], *h["ls"], h["sf"], h["noise"],
                   h["dtype"], h["cache_dtype"], h["flags"], h["k_eff"], h["ld"], h["ks"], h["ld_s"], h["ld_g"],
                   h["cg_iters"], h["fallback"], h["bytes_rc"], h["bytes_s"], h["bytes_p"], h["bytes_kdp"],
                   h["bytes_b"], h["bytes_minv"], h["additive"], 0)
    n = _payload_bytes(h) if payload is None else payload
    with open(path, "wb") as f:
        f.write(hdr + bytes(n))


def _load(lib, path):
    h = C.c_void_p()
    rc = lib.love_cache_load(str(path).encode(), None, None, C.byref(h))
    return rc, h.value


def _variants():
    def v(**kw):
        h = _base()
        h.update(kw)
        return h
    b = _base()
    n = _payload_bytes(b)
    return {
        "magic": (v(magic=b"LOVECACX"), None),
        "version": (v(version=1), None),
        "dim 4": (v(dim=4), None),
        "unused dimension sized": (v(g=[40, 2, 1]), None),
        "grid of 3 points": (v(g=[3, 1, 1], bytes_rc=3 * 12 * 4), None),
        "NaN spacing": (v(h=[float("nan"), 1.0, 1.0]), None),
        "k_eff past ld": (v(k_eff=20), None),
        "ld below k_eff + 1": (v(ld=8, bytes_rc=40 * 8 * 4), None),
        "Rc bytes short": (v(bytes_rc=40 * 12 * 4 - 16), None),
        "file truncated": (b, n - 1),
        "trailing byte": (b, n + 1),
        "FP64 data, FP32 cache": (v(dtype=1), None),
        "unknown cache dtype": (v(cache_dtype=7), None),
        "sampler sized wrong": (v(ks=4, ld_s=4, bytes_s=40 * 4 * 4 - 4), None),
        "sampler without ks": (v(ks=0, ld_s=4, bytes_s=40 * 4 * 4), None),
        "gradient tables partial": (v(ld_g=12, bytes_p=40 * 10 * 4), None),
        "tables without P": (v(bytes_minv=10 * 10 * 4), None),
        "k_eff 0": (v(k_eff=0), None),
        "negative noise": (v(noise=-1.0), None),
    }


@pytest.mark.parametrize("name", sorted(_variants()))
def test_inconsistent_cache_file_is_refused(lib, tmp_path, name):
    h, payload = _variants()[name]
    p = tmp_path / "c.love"
    _write(p, h, payload)
    rc, handle = _load(lib, p)
    assert rc == LOVE_ERR_ARG and not handle, name


def test_missing_file_is_refused(lib, tmp_path):
    rc, handle = _load(lib, tmp_path / "absent.love")
    assert rc == LOVE_ERR_ARG and not handle


def test_base_header_describes_its_payload():
    """The base case really is consistent (so each variant above differs from
    an acceptable file in the one field it changes)."""
    b = _base()
    m = b["g"][0]
    vec = 16 // 4
    assert b["ld"] == -(-(b["k_eff"] + 1) // vec) * vec
    assert b["bytes_rc"] == m * b["ld"] * 4
    assert _payload_bytes(b) == 16 * b["k_eff"] + b["bytes_rc"]
    assert np.all(np.isfinite(b["h"]))


def _consistent():
    b = _base()

    def v(**kw):
        h = dict(b)
        h.update(kw)
        return h
    return {
        "mean only": b,
        "sampler root and gradient tables": v(flags=7, ks=7, ld_s=8, bytes_s=40 * 8 * 4, ld_g=12,
                                              bytes_p=40 * 10 * 4, bytes_kdp=40 * 12 * 4, bytes_b=10 * 10 * 4,
                                              bytes_minv=10 * 10 * 4),
        "FP64 additive 2-D": v(dim=2, g=[40, 30, 1], additive=1, h=[1 / 35, 1 / 25, 1.0], ls=[0.2, 0.2, 1.0],
                               dtype=1, cache_dtype=1, ld=12, bytes_rc=70 * 12 * 8),
        "BF16 cache": v(cache_dtype=2, ld=16, bytes_rc=40 * 16 * 2),
    }


@pytest.mark.parametrize("name", sorted(_consistent()))
def test_consistent_cache_file_passes_the_checks(lib, tmp_path, name):
    """A header that matches its payload gets past the checks: without a GPU
    the load then fails at the first device allocation (LOVE_ERR_OOM or a CUDA
    error), with one it loads; it is never refused as an argument error."""
    p = tmp_path / "c.love"
    _write(p, _consistent()[name])
    rc, handle = _load(lib, p)
    if handle:
        lib.love_cache_destroy(C.c_void_p(handle))
    assert rc != LOVE_ERR_ARG, name

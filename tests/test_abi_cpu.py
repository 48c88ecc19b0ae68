"""Host-side checks of the C ABI that need no GPU.

The library loads on a machine without a GPU; every function declared in
include/fastttc.h is exported; argument validation happens on the host before any
CUDA call; the host-only functions (output dims, status strings, multi-scale
selection) agree with the oracle and the hand-worked fixtures.
"""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import oracle
import paper_1612_08825_gb300 as ft
from paper_1612_08825_gb300 import build as ftbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    ftbuild.build_library()
    return ft.load()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            prefix = text[:m.start()].rstrip()
            if name in ("if", "while", "sizeof", "defined") or prefix.endswith("#define"):
                continue
            # a declaration: preceded by a type token at statement start
            line_start = text.rfind(";", 0, m.start())
            stmt = text[line_start + 1:m.start()]
            if "typedef" in stmt or "#" in stmt.split("\n")[-1]:
                continue
            if re.search(r"[A-Za-z_]", stmt):
                names.add(name)
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared_functions()
    assert {"fastconv_nd", "fastconv_out_dims", "ttc_derivatives", "ttc_solve",
            "ttc_solve_sequence", "ttc_select_level", "ttc_ctx_create"} <= names
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_status_strings_and_version(L):
    assert L.ft_status_string(0) == b"FT_OK"
    assert L.ft_status_string(2) == b"FT_ERR_SHAPE"
    assert L.ft_status_string(6) == b"FT_ERR_TIMEOUT"
    assert L.ft_status_string(99) == b"FT_ERR_UNKNOWN"
    assert L.ft_version() >= 10000


def test_out_dims(L):
    assert ft.fastconv_out_dims((1080, 1920), (3, 3)) == (1082, 1922)
    assert ft.fastconv_out_dims((64, 256, 256), (5, 5, 5)) == (68, 260, 260)
    assert ft.fastconv_out_dims((2, 3), (5, 4)) == (6, 6)
    for dims, kd in [((1080, 1920), (2, 2)), ((7,), (11,)), ((1, 2, 3, 4, 5, 6, 7, 8), (2,) * 8)]:
        assert ft.fastconv_out_dims(dims, kd) == oracle.conv_out_dims(dims, kd)
    with pytest.raises(ft.FtError):
        ft.fastconv_out_dims((0, 4), (1, 1))
    with pytest.raises(ft.FtError):
        ft.fastconv_out_dims((2,) * 9, (1,) * 9)


def test_fastconv_validation_before_launch(L):
    d = (ctypes.c_int64 * 2)(4, 4)
    k = (ctypes.c_int64 * 2)(3, 3)
    bad = (ctypes.c_int64 * 2)(4, 0)
    # null pointers
    assert L.fastconv_nd(None, d, 2, 8, k, 8, None) == 1
    # bad shape with (fake, never dereferenced) pointers: rejected on the host
    assert L.fastconv_nd(8, bad, 2, 8, k, 8, None) == 2
    assert L.fastconv_nd(8, d, 0, 8, k, 8, None) == 2
    assert L.fastconv_nd(8, d, 9, 8, k, 8, None) == 2


def test_ttc_validation_before_launch(L):
    h = ctypes.c_void_p()
    assert L.ttc_ctx_create(None, 64, 64, 3, 1) == 1
    assert L.ttc_ctx_create(ctypes.byref(h), 1, 64, 3, 1) == 2
    assert L.ttc_ctx_create(ctypes.byref(h), 64, 64, 8, 1) == 3
    assert L.ttc_ctx_create(ctypes.byref(h), 64, 64, 0, 1) == 1
    # derivatives: bad dtype / shapes / pitch, with fake pointers never dereferenced
    f = ctypes.c_void_p(16)
    assert L.ttc_derivatives(f, f, 7, 8, 8, 8, f, f, f, None, None) == 1
    assert L.ttc_derivatives(f, f, 0, 1, 8, 8, f, f, f, None, None) == 2
    assert L.ttc_derivatives(f, f, 1, 8, 8, 16, f, f, f, None, None) == 2   # pitch < 4 W
    assert L.ttc_derivatives(None, f, 0, 8, 8, 8, f, f, f, None, None) == 1
    assert L.ttc_solve(None, f, f, 0, 8, 8, 8, 1, 1, f, None) == 1


def test_select_level_matches_golden_and_oracle(L):
    with open(os.path.join(ROOT, "tests", "golden", "multiscale_rule.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        n = len(case["ttc"])
        r = np.zeros(n, dtype=ft.RESULT_DTYPE)
        r["ttc"] = case["ttc"]
        r["resid"] = case["resid"]
        r["flags"] = case["flags"]
        assert ft.select_level(r, 0) == case["rule0"]
        assert ft.select_level(r, 1) == case["rule1"]
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = int(rng.integers(1, 8))
        r = np.zeros(n, dtype=ft.RESULT_DTYPE)
        o = np.zeros(n, dtype=oracle.RESULT_DTYPE)
        ttc = rng.choice([-3.0, 5.0, 10.0, 20.0, 30.0], n)
        res = rng.choice([0.1, 0.2, 0.3], n)
        fl = rng.choice([0, 0, 0, 1, 2, 4], n)
        for a in (r, o):
            a["ttc"] = ttc
            a["resid"] = res
            a["flags"] = fl
        for rule in (0, 1):
            assert ft.select_level(r, rule) == oracle.select_level(o, rule)
    with pytest.raises(ValueError):
        ft.select_level(np.zeros(2, dtype=ft.RESULT_DTYPE), 3)


def test_result_layout_matches_header():
    text = open(os.path.join(ROOT, "include", "fastttc.h")).read()
    assert "double sums[10];" in text
    assert ft.RESULT_DTYPE.itemsize == 152
    assert ft.RESULT_DTYPE.fields["n"][1] == 136 and ft.RESULT_DTYPE.fields["flags"][1] == 148


def test_pyramid_layout_and_pair_desc(L):
    """Pyramid blocks: level l of floor(H/2^l) x floor(W/2^l) pixels, uint16 for
    uint8 frames up to level 4 and float beyond, rows padded to 16 bytes, images
    aligned to 256 bytes; the descriptor mirrors the header's struct."""
    lay = ft.pyramid_layout(1080, 1920, 6)
    es = [0, 2, 2, 2, 2, 4]
    off = 0
    for l in range(1, 6):
        w, h = 1920 >> l, 1080 >> l
        assert lay["pitches"][l] == -(-(w * es[l]) // 16) * 16
        assert lay["offsets"][l] == off
        off += -(-(lay["pitches"][l] * h) // 256) * 256
    assert lay["bytes"] == off
    assert ft.pyramid_layout(100, 100, 1)["bytes"] == 0
    f32 = ft.pyramid_layout(33, 70, 2, dtype=__import__("torch").float32)
    assert f32["pitches"][1] == 144 and f32["bytes"] == 256 * -(-(144 * 16) // 256)
    b = ctypes.c_int64()
    assert L.ttc_pyramid_layout(8, 8, 4, 0, None, None, ctypes.byref(b)) == 2        # level 3 is 1 x 1
    assert L.ttc_pyramid_layout(64, 64, 8, 0, None, None, ctypes.byref(b)) == 3
    assert L.ttc_pyramid_layout(64, 64, 2, 5, None, None, ctypes.byref(b)) == 1
    assert L.ttc_pyramid_layout(64, 64, 2, 0, None, None, None) == 1
    rows = (ctypes.c_int * 2)(64, 16)
    assert L.ttc_batch_set_plan(None, rows, 2) == 1
    text = open(os.path.join(ROOT, "include", "fastttc.h")).read()
    assert "const void *prev_pyramid;" in text and "void *cur_pyramid;" in text
    assert ctypes.sizeof(ft.PairDesc) == 48 and ft.PairDesc.cur_pyramid.offset == 40


def test_fastconv_factor_rank_one_test(L):
    """Separable kernels (Gaussian, Sobel, 3-D box) factor and their factors' outer
    product reproduces the kernel; general kernels do not factor; bad arguments -1."""
    g1 = np.exp(-0.5 * ((np.arange(7) - 3) / 1.3) ** 2)
    gauss = np.outer(g1, g1).astype(np.float32)
    sobel = np.array([[1, 0, -1], [2, 0, -2], [1, 0, -1]], np.float32)
    box = np.full((3, 4, 5), 1.0 / 60, np.float32)
    for k in (gauss, sobel, box, np.array([2.5, -1.0, 0.25], np.float32)):
        f = ft.factor_kernel(k, rel_tol=1e-6)
        assert f is not None and [len(x) for x in f] == list(k.shape)
        prod = f[0].astype(np.float64)
        for x in f[1:]:
            prod = np.multiply.outer(prod, x.astype(np.float64))
        np.testing.assert_allclose(prod, k, atol=2e-6 * np.abs(k).max())
    rng = np.random.default_rng(3)
    assert ft.factor_kernel(rng.standard_normal((5, 5)).astype(np.float32)) is None
    assert ft.factor_kernel(np.eye(3, dtype=np.float32)) is None
    z = ft.factor_kernel(np.zeros((2, 3), np.float32))
    assert z is not None and not any(x.any() for x in z)
    f = (ctypes.c_float * 4)()
    k = (ctypes.c_float * 4)(1, 2, 3, 4)
    dims = (ctypes.c_int64 * 2)(2, 2)
    assert L.fastconv_factor(None, dims, 2, 1e-6, f) == -1
    assert L.fastconv_factor(k, dims, 0, 1e-6, f) == -1
    assert L.fastconv_factor(k, dims, 2, -1.0, f) == -1


def test_fastconv_separable_validation(L):
    f = ctypes.c_void_p(16)
    dims = (ctypes.c_int64 * 2)(8, 8)
    kd = (ctypes.c_int64 * 2)(3, 3)
    facs = (ctypes.c_void_p * 2)(16, None)
    assert L.fastconv_separable(f, dims, 2, facs, kd, f, ctypes.c_void_p(32), None) == 1   # null factor
    facs = (ctypes.c_void_p * 2)(16, 16)
    assert L.fastconv_separable(f, dims, 2, facs, kd, ctypes.c_void_p(48), None, None) == 1  # no scratch
    assert L.fastconv_separable(f, dims, 2, facs, kd, ctypes.c_void_p(48), ctypes.c_void_p(48), None) == 1
    assert L.fastconv_separable(f, dims, 9, facs, kd, ctypes.c_void_p(48), ctypes.c_void_p(64), None) == 2


def test_checked_build_flag_plumbing(monkeypatch):
    """FASTTTC_CHECK selects the checked build's define, and the record flag it reports has the
    same value in the header and the binding."""
    import re
    from paper_1612_08825_gb300 import build as b
    monkeypatch.delenv("FASTTTC_CHECK", raising=False)
    assert b.extra_flags() == []
    monkeypatch.setenv("FASTTTC_CHECK", "1")
    assert b.extra_flags() == ["-DFT_CHECK=1"]
    monkeypatch.setenv("FASTTTC_CHECK", "0")
    assert b.extra_flags() == []
    hdr = open(os.path.join(ROOT, "include", "fastttc.h")).read()
    m = re.search(r"#define FT_FLAG_BOUNDS (\d+)", hdr)
    assert m and int(m.group(1)) == ft.FLAG_BOUNDS
    flags = [int(v) for v in re.findall(r"#define FT_FLAG_\w+ (\d+)", hdr)]
    assert len(set(flags)) == len(flags) and all(f & (f - 1) == 0 for f in flags)   # distinct bits

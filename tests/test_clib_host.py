"""Host-side checks of the C-ABI library: it loads, exports every entry point
the public header declares, and validates geometries and layouts on the host
(no GPU needed: nothing here launches a kernel).
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bloomgb.h")


@pytest.fixture(scope="module")
def L():
    from paper_2512_15595_gb300 import build
    build.build()
    from paper_2512_15595_gb300 import _lib
    return _lib


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bf_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_what_the_binding_wraps(L):
    assert declared_functions() == sorted(L.EXPORTED)


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version(L):
    assert L.bf_status_str(0) == "BF_OK"
    assert L.bf_status_str(4) == "BF_EUNSUPPORTED"
    assert "sm_103a" in L.bf_version()


def P(L, b=1000, B=256, S=32, k=8, seed=0, groups=0):
    return L.bf_params(b, B, S, k, groups, seed)


def test_params_check(L):
    ok = [(256, 32, 8), (256, 32, 16), (512, 64, 8), (64, 64, 4), (1024, 64, 16), (128, 32, 4), (64, 32, 16)]
    for B, S, k in ok:
        assert L.bf_params_check(P(L, B=B, S=S, k=k)) == L.BF_OK, (B, S, k)
    # not an SBF (Sec. II-A: k >= s, s | k) or malformed
    bad = [(256, 32, 4), (512, 32, 8), (512, 64, 4), (256, 32, 12), (96, 32, 6), (256, 16, 16), (2048, 64, 32)]
    for B, S, k in bad:
        assert L.bf_params_check(P(L, B=B, S=S, k=k)) == L.BF_EINVAL, (B, S, k)
    assert L.bf_params_check(P(L, b=0)) == L.BF_EINVAL
    assert L.bf_params_check(P(L, groups=3)) == L.BF_EINVAL   # groups must divide s
    assert L.bf_params_check(P(L, groups=16)) == L.BF_EINVAL  # more groups than words
    # admissible but not compiled (k outside {4, 8, 16})
    assert L.bf_params_check(P(L, B=256, S=32, k=24)) == L.BF_EUNSUPPORTED
    assert L.bf_params_check(P(L, B=1024, S=32, k=32)) == L.BF_EUNSUPPORTED


def test_every_valid_layout_is_compiled(L):
    from paper_2512_15595_gb300 import valid_layouts
    geoms = [(64, 32), (128, 32), (256, 32), (512, 32), (64, 64), (128, 64), (256, 64), (512, 64), (1024, 64)]
    n = 0
    for B, S in geoms:
        s = B // S
        for k in (4, 8, 16):
            if k < s or k % s:
                continue
            for cg, phi in valid_layouts(B, S):
                for kpt in (1, 2, 4):
                    for op in (L.BF_OP_ADD, L.BF_OP_CONTAINS):
                        lay = L.bf_layout(cg, phi, kpt, 256, 0, 0)
                        assert L.bf_layout_check(P(L, B=B, S=S, k=k), op, lay) == L.BF_OK
                        n += 1
    assert n > 500


def test_fig2_layouts_are_valid_and_others_rejected(L):
    # the five layouts of Fig. 2 (B = 256, S = 32)
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "fig2_layouts.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for _, theta, phi, steps in rows:
        theta, phi, steps = int(theta), int(phi), int(steps)
        assert 8 // (theta * phi) == steps
        lay = L.bf_layout(theta, phi, 1, 256, 0, 0)
        assert L.bf_layout_check(P(L), L.BF_OP_CONTAINS, lay) == L.BF_OK
    from paper_2512_15595_gb300 import valid_layouts
    assert {(int(r[1]), int(r[2])) for r in rows} <= set(valid_layouts(256, 32))
    assert len(valid_layouts(256, 32)) == 10
    for cg, phi in [(3, 1), (16, 1), (4, 4), (2, 8), (1, 16)]:
        assert L.bf_layout_check(P(L), L.BF_OP_CONTAINS, L.bf_layout(cg, phi, 1, 256, 0, 0)) == L.BF_EINVAL
    for kpt, threads in [(3, 256), (8, 256), (1, 48), (1, 1024)]:
        assert L.bf_layout_check(P(L), L.BF_OP_ADD, L.bf_layout(1, 1, kpt, threads, 0, 0)) == L.BF_EINVAL
    assert L.bf_layout_check(P(L), 7, None) == L.BF_EINVAL
    # zeros resolve to defaults
    assert L.bf_layout_check(P(L), L.BF_OP_ADD, L.bf_layout(0, 0, 0, 0, 0, 0)) == L.BF_OK


def test_null_arguments_rejected_without_gpu(L):
    import ctypes
    lib = L.lib()
    assert lib.bf_add(None, None, 0, None) == L.BF_EINVAL
    assert lib.bf_contains(None, None, 5, None, None) == L.BF_EINVAL
    assert lib.bf_destroy(None) == L.BF_EINVAL
    assert lib.bf_create(None, None, None) == L.BF_EINVAL
    h = ctypes.c_void_p()
    assert lib.bf_create(ctypes.byref(P(L, b=0)), None, ctypes.byref(h)) == L.BF_EINVAL
    assert h.value is None
    assert "num_blocks" in L.bf_last_error()
    # gups argument checks happen before any CUDA call
    assert lib.bf_gups(5, None, 0, 32, None, 0, None, None, None) == L.BF_EINVAL
    assert lib.bf_gups(0, None, 1 << 20, 48, None, 10, None, None, None) == L.BF_EINVAL


def test_csbf_params_and_layouts(L):
    # cache-sectorized (Sec. II-A): z | s, z | k, k + z <= 64
    for B, S, k, z in [(512, 64, 16, 2), (1024, 64, 16, 4), (256, 32, 4, 1), (256, 32, 8, 4), (1024, 64, 8, 8)]:
        assert L.bf_params_check(P(L, B=B, S=S, k=k, groups=z)) == L.BF_OK, (B, S, k, z)
    # z = s is the sectorized filter
    assert L.bf_params_check(P(L, B=256, S=32, k=8, groups=8)) == L.BF_OK
    for B, S, k, z in [(512, 64, 6, 4), (512, 64, 16, 3)]:
        assert L.bf_params_check(P(L, B=B, S=S, k=k, groups=z)) == L.BF_EINVAL, (B, S, k, z)
    p = P(L, B=1024, S=64, k=16, groups=4)
    for cg in (1, 2, 4):
        for kpt in (1, 2, 4):
            for op in (0, 1):
                assert L.bf_layout_check(p, op, L.bf_layout(cg, 1, kpt, 256, 0, 0)) == L.BF_OK
    assert L.bf_layout_check(p, 0, L.bf_layout(8, 1, 1, 256, 0, 0)) == L.BF_EINVAL  # cg must divide groups
    assert L.bf_layout_check(p, 1, L.bf_layout(1, 2, 1, 256, 0, 0)) == L.BF_EINVAL  # phi must be 1

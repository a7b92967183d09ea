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


def test_layout_flags(L):
    """The four hint bits are accepted for both operations (the L2 prefetch
    hint is used by the batched kernels, the warp aggregation by the
    construction kernels, each ignored by the others); any other bit is
    rejected before a launch."""
    every = (L.BF_HINT_FILTER_EVICT_LAST | L.BF_HINT_KEYS_EVICT_NORMAL | L.BF_HINT_PREFETCH_L2
             | L.BF_HINT_WARP_AGGREGATE)
    for flags in (0, L.BF_HINT_FILTER_EVICT_LAST, L.BF_HINT_KEYS_EVICT_NORMAL, L.BF_HINT_PREFETCH_L2,
                  L.BF_HINT_WARP_AGGREGATE, every):
        for op in (L.BF_OP_ADD, L.BF_OP_CONTAINS):
            assert L.bf_layout_check(P(L), op, L.bf_layout(0, 0, 0, 0, 0, flags)) == L.BF_OK, flags
    for bad in (1 << 4, 1 << 31):
        assert L.bf_layout_check(P(L), L.BF_OP_ADD, L.bf_layout(0, 0, 0, 0, 0, bad)) == L.BF_EINVAL


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


def test_mlp_int8_struct_layout_matches_the_header(L, tmp_path):
    """The ctypes mirror of bf_mlp_int8 has the C struct's size and offsets (gcc, host only)."""
    import ctypes
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "lay.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "bloomgb.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(bf_mlp_int8),'
                   'offsetof(bf_mlp_int8,w2), offsetof(bf_mlp_int8,w3), offsetof(bf_mlp_int8,b1),'
                   'offsetof(bf_mlp_int8,b2), offsetof(bf_mlp_int8,b3), offsetof(bf_mlp_int8,sh1),'
                   'offsetof(bf_mlp_int8,sh2), offsetof(bf_mlp_int8,unit)); return 0;}\n')
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    S = L.bf_mlp_int8
    want = [ctypes.sizeof(S)] + [getattr(S, f).offset for f in ("w2", "w3", "b1", "b2", "b3", "sh1", "sh2", "unit")]
    assert got == want


def test_mlp_arguments_rejected_without_gpu(L):
    lib = L.lib()
    assert lib.bf_mlp_workspace_bytes(1024) >= 4 * (1024 * (2 * 128 + 2 * 64 + 2) + 2 * L.BF_MLP_PARAMS)
    ws = lib.bf_mlp_workspace_bytes(64)
    # null pointers, empty batch, unaligned workspace, n too large, multiplier not coprime to n
    assert lib.bf_mlp_grad(None, 256, 256, 10, 0, 1, 64, 256, None, 256, ws, None) == L.BF_EINVAL
    assert lib.bf_mlp_grad(256, 256, 256, 10, 0, 1, 0, 256, None, 256, ws, None) == L.BF_EINVAL
    assert lib.bf_mlp_grad(256, 256, 256, 10, 0, 1, 64, 256, None, 128, ws, None) == L.BF_EINVAL
    assert lib.bf_mlp_grad(256, 256, 256, 10, 0, 1, 64, 256, None, 256, ws - 4, None) == L.BF_EINVAL
    assert lib.bf_mlp_grad(256, 256, 256, 1 << 32, 0, 1, 64, 256, None, 256, ws, None) == L.BF_EINVAL
    assert lib.bf_mlp_grad(256, 256, 256, 10, 0, 4, 64, 256, None, 256, ws, None) == L.BF_EINVAL
    assert lib.bf_mlp_grad(256, 256, 256, 10, 0, 0, 64, 256, None, 256, ws, None) == L.BF_EINVAL
    assert lib.bf_mlp_train(256, 256, 256, 256, 256, 10, 3, 64, 0, 5, 1e-3, 0.9, 0.999, 1e-8, None, 256, ws,
                            None) == L.BF_EINVAL
    assert lib.bf_mlp_adam(256, 256, 256, 256, 0, 1e-3, 0.9, 0.999, 1e-8, None) == L.BF_EINVAL
    assert lib.bf_mlp_load(None, None) == L.BF_EINVAL
    bad = L.bf_mlp_int8()
    bad.sh1 = 63
    import ctypes
    h = ctypes.c_void_p()
    assert lib.bf_mlp_load(ctypes.byref(bad), ctypes.byref(h)) == L.BF_EINVAL
    assert lib.bf_mlp_free(None) == L.BF_EINVAL
    assert lib.bf_mlp_scores(None, 256, 4, 256, None) == L.BF_EINVAL
    assert lib.bf_mlp_contains(None, 0, None, 256, 4, 256, None) == L.BF_EINVAL
    assert lib.bf_mlp_select_below(None, 0, 256, 4, 256, 256, None) == L.BF_EINVAL
    assert lib.bf_mlp_export(None, None, 0, None, None) == L.BF_EINVAL


def test_mma_cost_arguments_rejected_without_gpu(L):
    import ctypes
    lib = L.lib()
    c = ctypes.c_double()
    assert lib.bf_mma_cost(48, 0, 10, ctypes.byref(c)) == L.BF_EINVAL
    assert lib.bf_mma_cost(64, 0, 0, ctypes.byref(c)) == L.BF_EINVAL
    assert lib.bf_mma_cost(64, 0, 1 << 25, ctypes.byref(c)) == L.BF_EINVAL
    assert lib.bf_mma_cost(64, 1, 10, None) == L.BF_EINVAL


def test_parquet_salt_set_params(L):
    ok = L.bf_params(100, 256, 32, 8, 0, 0, 1, 0)
    assert L.bf_params_check(ok) == L.BF_OK
    assert L.bf_params_check(L.bf_params(100, 256, 32, 8, 8, 0, 1, 0)) == L.BF_OK  # groups = s is sectorized
    for bad in [(100, 256, 32, 16, 0, 0, 1, 0), (100, 512, 32, 16, 0, 0, 1, 0), (100, 256, 64, 8, 0, 0, 1, 0),
                (100, 256, 32, 8, 2, 0, 1, 0), (100, 256, 32, 8, 0, 0, 2, 0)]:
        assert L.bf_params_check(L.bf_params(*bad)) == L.BF_EINVAL, bad


def test_params_struct_layout_matches_the_header(L, tmp_path):
    import ctypes
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "p.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "bloomgb.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(bf_params), offsetof(bf_params, seed),'
                   'offsetof(bf_params, salts), offsetof(bf_params, reserved)); return 0;}\n')
    exe = tmp_path / "p"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    S = L.bf_params
    assert got == [ctypes.sizeof(S), S.seed.offset, S.salts.offset, S.reserved.offset]


def test_partition_struct_layout_matches_the_header(L, tmp_path):
    import ctypes
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    fields = ("mode", "slice_log2", "chunk_keys", "cap_override", "window_log2", "lookup_mode",
              "lookup_chunk_keys", "passes", "part_ctas")
    src = tmp_path / "q.c"
    offs = ", ".join(f"offsetof(bf_partition, {f})" for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "bloomgb.h"\n'
                   'int main(void){printf("' + " ".join(["%zu"] * (len(fields) + 1)) + '\\n", '
                   'sizeof(bf_partition), ' + offs + '); return 0;}\n')
    exe = tmp_path / "q"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    S = L.bf_partition
    assert got == [ctypes.sizeof(S)] + [getattr(S, f).offset for f in fields]


def test_timing_struct_layout_matches_the_header(L, tmp_path):
    import ctypes
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "t.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "bloomgb.h"\n'
                   'int main(void){printf("%zu %zu %d %d %d\\n", sizeof(bf_timing), offsetof(bf_timing, launches),'
                   ' BF_PHASES, BF_PHASE_RECORD_INSERT, BF_PHASE_BITMAP_EXPAND); return 0;}\n')
    exe = tmp_path / "t"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    T = L.bf_timing
    assert got == [ctypes.sizeof(T), T.launches.offset, L.BF_PHASES,
                   L.PHASE_NAMES.index("record_insert"), L.PHASE_NAMES.index("bitmap_expand")]


def test_status_timing_and_partition_arguments_rejected_without_gpu(L):
    """The index-check status, the phase timing and the overlapped-schedule
    settings reject NULL handles and out-of-range values on the host."""
    import ctypes
    lib = L.lib()
    v = ctypes.c_uint32(7)
    assert lib.bf_device_status(None, None, ctypes.byref(v)) == L.BF_EINVAL
    assert lib.bf_noalloc_status(None) == L.BF_EINVAL
    assert lib.bf_set_timing(None, 1) == L.BF_EINVAL
    t = L.bf_timing()
    assert lib.bf_get_timing(None, ctypes.byref(t)) == L.BF_EINVAL
    assert lib.bf_set_partition(None, ctypes.byref(L.bf_partition())) == L.BF_EINVAL

"""Host-side arithmetic of bench.py's roofline: the algorithmic bytes each
kernel moves per call (no GPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_phase_bytes_of_the_4gib_workload():
    w = bench.WORKLOADS["4GiB"]
    b, n_ins, n_q = bench.wl_sizes(w)
    assert (b, n_ins, n_q) == (1 << 27, 3_435_973_836, 10**9)
    part = {"chunk_keys": 1 << 32, "lookup_chunk_keys": 1 << 29}
    pb = lambda ph: bench.phase_bytes(ph, w, n_ins, n_q, part)  # noqa: E731
    assert pb("partition_add") == 16 * n_ins
    assert pb("record_insert") == 8 * n_ins + 2 * (4 << 30)          # one pass: every window read and written once
    assert pb("partition_lookup") == 20 * n_q
    assert pb("record_probe") == 12 * n_q + 2 * (4 << 30)            # two passes of 2^29 queries
    assert pb("bitmap_expand") == n_q // 8 + n_q
    assert pb("add_direct") == 72 * n_ins and pb("contains_direct") == 41 * n_q
    assert pb("host_stage") == 8 * (n_ins + n_q)
    # more construction passes re-read the windows once per pass
    assert bench.phase_bytes("record_insert", w, n_ins, n_q, dict(part, chunk_keys=1 << 31)) == \
        8 * n_ins + 2 * 2 * (4 << 30)


def test_every_phase_has_a_kernel_name():
    from paper_2512_15595_gb300 import _lib
    assert set(bench.PHASE_KERNELS) == set(_lib.PHASE_NAMES)

"""Host logic of the autotuner: the tuned-table lookups and the batched
block-width choice at a false-positive band (no GPU)."""
import json

import pytest

from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS, autotune


def _res(B, S, ms, fp, q=1 << 27):
    return dict(block_bits=B, word_bits=S, k=8, step_ms=ms, fp=fp, queries=q)


def test_fp_count_limit():
    assert autotune.fp_count_limit(0) == pytest.approx(3.0)
    assert autotune.fp_count_limit(1) == pytest.approx(4.0)
    assert autotune.fp_count_limit(100) == pytest.approx(130.0)


def test_choose_fastest_within_band():
    res = [_res(256, 32, 10.0, 2), _res(128, 64, 6.0, 40), _res(512, 64, 9.0, 5), _res(64, 32, 7.0, 7)]
    c = autotune.choose_batch_geometry(res, (256, 32))
    # limit 2 + 3*sqrt(2) = 6.24: 128/64 (40) and 64/32 (7) are out, 512/64 (5) is the fastest left
    assert (c["block_bits"], c["word_bits"]) == (512, 64)
    assert c["fp_limit"] == pytest.approx(2 + 3 * 2 ** 0.5)
    assert c["reference"] == {"block_bits": 256, "word_bits": 32, "fp": 2, "step_ms": 10.0}


def test_choose_reference_when_fastest():
    res = [_res(256, 32, 5.0, 0), _res(128, 32, 6.0, 0)]
    c = autotune.choose_batch_geometry(res, (256, 32))
    assert (c["block_bits"], c["word_bits"]) == (256, 32)


def test_choose_keeps_reference_within_noise():
    """A geometry less than min_gain faster does not replace the reference."""
    res = [_res(256, 32, 10.0, 2), _res(128, 32, 9.8, 5)]
    assert autotune.choose_batch_geometry(res, (256, 32))["block_bits"] == 256
    assert autotune.choose_batch_geometry(res, (256, 32), min_gain=0.01)["block_bits"] == 128


def test_choose_needs_reference():
    with pytest.raises(ValueError):
        autotune.choose_batch_geometry([_res(128, 32, 1.0, 0)], (256, 32))


def test_tuned_tables(tmp_path, monkeypatch):
    path = tmp_path / "tuned.json"
    table = {
        "B256_S32_K8_hbm": {"add": {"layout": {"cg": 2, "phi": 4, "kpt": 4}},
                            "contains": {"layout": {"cg": 1, "phi": 8, "kpt": 2}}},
        "batch_B512_S64_K8": {"add": {"layout": {"cg": 8, "phi": 1, "kpt": 1}},
                              "contains": {"layout": {"cg": 1, "phi": 8, "kpt": 4}}},
    }
    path.write_text(json.dumps(table))
    monkeypatch.setattr(autotune, "TUNED_PATH", str(path))
    assert autotune.tuned_layout(256, 32, 8, "hbm", BF_OP_ADD) == {"cg": 2, "phi": 4, "kpt": 4}
    assert autotune.tuned_layout(256, 32, 8, "l2", BF_OP_ADD) is None
    assert autotune.tuned_batch_layout(512, 64, 8, BF_OP_CONTAINS) == {"cg": 1, "phi": 8, "kpt": 4}
    assert autotune.tuned_batch_layout(256, 32, 8, BF_OP_ADD) is None
    table["batch_K8_geometry"] = {"block_bits": 512}
    autotune.save_tuned(table)
    assert autotune.load_tuned() == table


def test_regime_and_keys():
    assert autotune.regime_of(32 << 20, 126 << 20) == "l2"
    assert autotune.regime_of(4 << 30, 126 << 20) == "hbm"
    assert autotune.key_of(256, 32, 8, "hbm") == "B256_S32_K8_hbm"
    assert autotune.batch_key(128, 64, 8) == "batch_B128_S64_K8"


def test_bench_batch_geometries_are_valid():
    """Every geometry the batched sweep tries is a valid K = 8 filter for the
    library (host-side parameter check, no GPU), and the workload's own
    256-bit / 32-bit geometry is among them."""
    import bench
    from paper_2512_15595_gb300 import _lib, build
    build.build()
    for B, S in bench.BATCH_GEOMETRIES:
        assert _lib.bf_params_check(_lib.bf_params(1000, B, S, 8, 0, 0, 0, 0)) == _lib.BF_OK, (B, S)
    assert (256, 32) in bench.BATCH_GEOMETRIES


class _FakeEvent:
    """Stands in for torch.cuda.Event: elapsed time from a shared fake clock."""
    clock = [0.0]

    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = _FakeEvent.clock[0]

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.t - self.t


class _FakeTorch:
    class cuda:
        Event = _FakeEvent

        @staticmethod
        def current_stream():
            return None


class _FakeBatch:
    """A batch whose calls advance the fake clock by a cost that depends on
    its layout, so the sweep's choice is known in advance."""

    def __init__(self, cost):
        self.params = type("P", (), {"block_bits": 256, "word_bits": 32, "k": 8})()
        self.total_keys = 1000
        self.nfilters = 3
        self.cost = cost
        self.lay = {}

    def set_layout(self, op, **lay):
        self.lay[op] = dict(lay)

    def _run(self, op):
        _FakeEvent.clock[0] += self.cost(op, self.lay[op])

    def add(self, keys):
        self._run(BF_OP_ADD)

    def contains(self, keys, out=None):
        self._run(BF_OP_CONTAINS)


def test_sweep_batch_picks_the_fastest_layout_per_operation():
    def cost(op, lay):
        base = 5.0 if op == BF_OP_ADD else 3.0
        if op == BF_OP_ADD and (lay["cg"], lay["phi"], lay["kpt"], lay["flags"], lay["grid_ctas"]) == (4, 2, 4, 4, 304):
            return 1.0
        if op == BF_OP_CONTAINS and (lay["cg"], lay["phi"], lay["kpt"], lay["grid_ctas"]) == (1, 8, 2, 0):
            return 0.5 + 0.1 * lay["flags"]
        return base + 0.01 * lay["cg"]

    b = _FakeBatch(cost)
    res = autotune.sweep_batch(_FakeTorch, b, None, None, None, kpts=(1, 2, 4), reps=3,
                               flag_sets=(0, 4), grids=(0, 304))
    assert res["key"] == "batch_B256_S32_K8"
    e = res["entry"]
    assert e["add"]["layout"] == dict(cg=4, phi=2, kpt=4, flags=4, grid_ctas=304)
    assert e["contains"]["layout"] == dict(cg=1, phi=8, kpt=2, flags=0, grid_ctas=0)
    assert e["add"]["ms"] == pytest.approx(1.0) and e["contains"]["ms"] == pytest.approx(0.5)
    assert e["step_ms"] == pytest.approx(1.5)
    assert e["add"]["gkeys_s"] == pytest.approx(1000 / 1e-3 / 1e9)
    # every (cg, phi) of a 256/32 block x 3 kpt x 2 flag sets x 2 grids, per operation
    from paper_2512_15595_gb300 import valid_layouts
    assert len(res["rows"]) == 2 * len(valid_layouts(256, 32)) * 3 * 2 * 2
    # the batch is left at the best layouts
    assert b.lay[BF_OP_ADD] == e["add"]["layout"] and b.lay[BF_OP_CONTAINS] == e["contains"]["layout"]

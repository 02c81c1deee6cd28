"""The launch-shape cache around mpm_autotune (paper_2103_11050_gb300/autotune.py): keys,
hits, misses and stale entries, with a stand-in for the library context.  CPU only."""
import json

from paper_2103_11050_gb300 import autotune as AT

NAMES = ["local_threads", "local_stage", "ds_threads", "ds_stage", "transport_rows", "sweep_terms"]


class FakeCtx:
    """get_tuning / set_tuning / autotune as the binding's Context exposes them."""

    def __init__(self, best):
        self.current = {k: 0 for k in NAMES}
        self.best = best
        self.autotuned = 0

    def get_tuning(self):
        return dict(self.current)

    def set_tuning(self, tune):
        self.current = dict(tune)

    def autotune(self, reps=5):
        self.autotuned += 1
        self.current = dict(self.best)
        return dict(self.best), [0.1, 0.2, 0.3, 0.4]


def test_shape_key_run_length():
    assert AT._runs([16, 16, 16, 8, 20, 20]) == "16*3,8,20*2"
    assert AT._runs([12]) == "12"
    k = AT.shape_key(256, 128, 128, [16] * 8, [8, 12, 12], "fp32", "GB300")
    assert k == "GB300|R=256|128x128|cols=16*8|rows=8,12*2|prec=fp32"
    assert k != AT.shape_key(256, 128, 128, [16] * 8, [8, 12, 12], "fp64", "GB300")


def test_miss_autotunes_and_caches_then_hit_reuses(tmp_path):
    path = str(tmp_path / "cache.json")
    best = dict(zip(NAMES, [128, 0, 256, 1, 16, 8]))
    key = AT.shape_key(1, 64, 64, [16] * 4, [16] * 4, "fp32", "dev")
    a = FakeCtx(best)
    tune, src = AT.tuned(a, key, path)
    assert src == "autotune" and tune == best and a.autotuned == 1
    stored = json.load(open(path))
    assert stored[key]["tuning"] == best and set(stored[key]["best_ms"]) == {
        "transport", "local_solve", "downscale_solve", "interface_sweeps"}
    assert AT.cached(key, NAMES, path) == best
    b = FakeCtx({k: -1 for k in NAMES})
    tune, src = AT.tuned(b, key, path)
    assert src == "cache" and b.autotuned == 0 and b.current == best
    # another shape misses
    c = FakeCtx(best)
    assert AT.tuned(c, key + "x", path)[1] == "autotune"
    assert len(json.load(open(path))) == 2


def test_entry_with_other_parameters_is_retuned(tmp_path):
    path = str(tmp_path / "cache.json")
    key = "k"
    json.dump({key: {"tuning": {"local_threads": 64}, "best_ms": {}}}, open(path, "w"))
    assert AT.cached(key, NAMES, path) is None
    best = dict(zip(NAMES, [64, 1, 128, 0, 8, 16]))
    ctx = FakeCtx(best)
    assert AT.tuned(ctx, key, path) == (best, "autotune")
    assert AT.cached(key, NAMES, path) == best


def test_unreadable_cache_counts_as_empty(tmp_path):
    path = tmp_path / "cache.json"
    path.write_text("{not json")
    assert AT.cached("k", NAMES, str(path)) is None
    ctx = FakeCtx(dict(zip(NAMES, [128] * 6)))
    assert AT.tuned(ctx, "k", str(path))[1] == "autotune"
    assert json.load(open(path))["k"]["tuning"] == ctx.best

"""Host logic of the launch-shape tuner's binding (RT.autotune): the rows that
rt_autotune reports are unpacked, the chosen shape per stage is stored in the
JSON cache under a key of device, systems and parameters, and a context with
the same key takes its shapes from the cache without timing.  The library
calls are replaced by a fake (no GPU); rt_default_params runs for real."""
import ctypes
import json

import numpy as np
import pytest

import synth

rtm = pytest.importorskip("paper_1404_5776_gb300")


class FakeLib:
    """rt_autotune / rt_set_launch_shape / rt_get_launch_shape as the binding
    calls them through ctypes: it reports 4 + 4 rows for stages 0 and 1."""

    ROWS = [(0, 2, 0, 1, 31.7), (0, 2, 1, 0, 34.4), (0, 3, 0, 0, 41.0), (0, 3, 1, 0, 40.3),
            (1, 2, 0, 0, 17.7), (1, 2, 1, 1, 17.1), (1, 3, 0, 0, 24.5), (1, 3, 1, 0, 24.3)]

    def __init__(self):
        self.tuned = 0
        self.shapes = {}

    def rt_autotune(self, ctx, reps, mx, n_ref, rows_p, ms_p):
        self.tuned += 1
        n_ref._obj.value = len(self.ROWS)
        rows = np.ctypeslib.as_array(ctypes.cast(rows_p, ctypes.POINTER(ctypes.c_int32)), shape=(mx, 4))
        ms = np.ctypeslib.as_array(ctypes.cast(ms_p, ctypes.POINTER(ctypes.c_double)), shape=(mx,))
        for i, (st, ns, pers, ch, t) in enumerate(self.ROWS):
            rows[i] = (st, ns, pers, ch)
            ms[i] = t
            if ch:
                self.shapes[st] = (ns, pers)
        return 0

    def rt_set_launch_shape(self, ctx, st, ns, pers):
        self.shapes[st] = (ns, pers)
        return 0

    def rt_get_launch_shape(self, ctx, st, a_ref, b_ref):
        a_ref._obj.value, b_ref._obj.value = self.shapes.get(st, (2, 0))
        return 0


def _fake_ctx(system, lib, **params):
    ctx = object.__new__(rtm.RT)
    ctx.systems = [system]
    ctx.params = rtm.make_params(**params)
    ctx.lib = lib
    ctx.ctx = ctypes.c_void_p(1)
    return ctx


def test_tuned_rows_chosen_shapes_and_cache(tmp_path):
    s = synth.diamond_system(2, "spd13", 6.0, 6.0)
    cache = str(tmp_path / "sub" / "tune.json")
    lib = FakeLib()
    a = _fake_ctx(s, lib, precision="fp32", incremental=1)
    res = a.autotune(reps=2, cache=cache)
    assert res["source"] == "tuned" and lib.tuned == 1
    assert len(res["rows"]) == len(FakeLib.ROWS)
    assert res["rows"][0]["what"] == "M, 13 functions" and res["rows"][0]["ms"] == pytest.approx(31.7)
    assert res["chosen"] == {0: (2, 0), 1: (2, 1)}
    with open(cache) as f:
        stored = json.load(f)
    assert list(stored.values()) == [{"0": [2, 0], "1": [2, 1]}]

    # same systems and parameters: shapes from the cache, no timing
    lib2 = FakeLib()
    b = _fake_ctx(s, lib2, precision="fp32", incremental=1)
    res2 = b.autotune(cache=cache)
    assert res2["source"] == "cache" and lib2.tuned == 0
    assert lib2.shapes == {0: (2, 0), 1: (2, 1)}
    assert b.get_launch_shape(1) == (2, 1)

    # another parameter set (scalar FMAs) is another key: tuned again, both kept
    lib3 = FakeLib()
    c = _fake_ctx(s, lib3, precision="fp32", incremental=1, packed_fma=0)
    assert c.autotune(cache=cache)["source"] == "tuned" and lib3.tuned == 1
    with open(cache) as f:
        assert len(json.load(f)) == 2


def test_no_cache_always_tunes():
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    lib = FakeLib()
    a = _fake_ctx(s, lib, precision="fp32", incremental=1)
    a.autotune()
    a.autotune()
    assert lib.tuned == 2

"""Grouped products of the reference split and the launch-shape tuner.

In the reference split on the CUDA cores, every (system, kick) pair of one
block size is multiplied by one launch per product (M = cut(dU dK), then
dK' = dK + R + M + cut(W dU^dagger), Sec. II.A), the pairs with the most block
triples first.  The tuner (rt_autotune) times, per product stage, the stages
per warp of the 13-function kernel and a one-shot or persistent grid, and
keeps the fastest.  An item's arithmetic does not depend on which launch
carries it or on the launch shape, so K must come out bit for bit the same
whether a system runs alone or in a batch, and under every shape.  The batch
against the oracle is in test_gpu_batch.py.
"""
import json

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

R = 6.0
KAPPA = 1e-3


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def systems():
    pos, species = synth.si_h_cluster(target=60)
    cluster = synth.build_system(pos, None, species, 5.0, 5.0)         # 1 + 4 functions, open
    syss = [synth.diamond_system(2, "spd13", 6.0, 6.0),                # 64 atoms x 13
            cluster,
            synth.diamond_system(3, "sp4", 6.0, 6.0, seed=3)]          # 216 atoms x 4
    k0 = [synth.ground_state_dense(s, int(np.sum(s.bsize)) // 2)[0] for s in syss]
    return syss, k0


def _ctx(rt, syss, k0s, full_step=1):
    kw = dict(prop="em", precision="fp32", n_kick=3, incremental=1, full_step=full_step,
              r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)
    if full_step:
        kw["field_poly"] = 1
    ctx = rt.RT(syss, **kw)
    ctx.inverse()
    for si, K0 in enumerate(k0s):
        for d in range(3):
            ctx.set_density_dense(si, d, K0)
            ctx.kick(si, d, d, KAPPA)
    if not full_step:
        ctx.propagator(0.0)
    return ctx


def _all_k(rt, ctx, n_sys):
    return [[ctx.matrix(si, rt.RT_MAT_K, kick=d) for d in range(3)] for si in range(n_sys)]


def test_one_launch_per_product_and_block_size(rt, systems):
    """Three systems (block sizes 13, 4 and 4) with three kicks each: every step
    launches the M product twice (once per block size) and the K' product
    twice, not once per (system, kick) pair."""
    syss, k0 = systems
    ctx = _ctx(rt, syss, k0)
    ctx.step(2)
    ctx.profile(True)
    ctx.step(3)
    prof = ctx.profile_read()
    ctx.profile(False)
    assert prof["gemm_M=UK"]["launches"] == 2 * 3
    assert prof["gemm_K=MUdag"]["launches"] == 2 * 3
    ctx.close()


@pytest.mark.parametrize("full_step", [0, 1])
def test_batched_equals_alone_bit_for_bit(rt, systems, full_step):
    """Each system of the batch gives the same K, bit for bit, as the same
    system in a context of its own (its three kicks still grouped)."""
    syss, k0 = systems
    steps = 6
    ctx = _ctx(rt, syss, k0, full_step)
    ctx.step(steps)
    batched = _all_k(rt, ctx, len(syss))
    ctx.close()
    for si in range(len(syss)):
        alone = _ctx(rt, [syss[si]], [k0[si]], full_step)
        alone.step(steps)
        for d in range(3):
            assert np.array_equal(alone.matrix(0, rt.RT_MAT_K, kick=d), batched[si][d]), (si, d)
        alone.close()


def test_every_launch_shape_gives_the_same_k(rt, systems):
    """Stages per warp 2 or 3, one-shot or persistent grids: the same K bit for
    bit after several steps, for both block sizes."""
    syss, k0 = systems
    ref = None
    for ns, pers in ((2, 0), (2, 1), (3, 0), (3, 1)):
        ctx = _ctx(rt, syss, k0)
        for st in range(4):
            ctx.set_launch_shape(st, ns if st < 2 else 2, pers)
            assert ctx.get_launch_shape(st) == (ns if st < 2 else 2, pers)
        ctx.step(5)
        ks = _all_k(rt, ctx, len(syss))
        ctx.close()
        if ref is None:
            ref = ks
            continue
        for si in range(len(syss)):
            for d in range(3):
                assert np.array_equal(ks[si][d], ref[si][d]), (ns, pers, si, d)


def test_tuner_times_every_shape_keeps_k_and_caches(rt, systems, tmp_path):
    """rt_autotune reports every candidate of every stage present, chooses one
    per stage, leaves the densities untouched, and a second context with the
    same systems and parameters takes the shapes from the JSON cache."""
    syss, k0 = systems
    cache = str(tmp_path / "tune.json")
    ctx = _ctx(rt, syss, k0)
    ctx.step(2)
    before = _all_k(rt, ctx, len(syss))
    res = ctx.autotune(reps=2, cache=cache)
    assert res["source"] == "tuned"
    stages = sorted({r["stage"] for r in res["rows"]})
    assert stages == [0, 1, 2, 3]
    for st in stages:
        rows = [r for r in res["rows"] if r["stage"] == st]
        assert len(rows) == (4 if st < 2 else 2)
        assert sum(r["chosen"] for r in rows) == 1
        assert all(r["ms"] > 0 for r in rows)
        best = min(rows, key=lambda r: r["ms"])
        assert best["chosen"]
        assert ctx.get_launch_shape(st) == (best["stages_per_warp"], best["persistent"])
    after = _all_k(rt, ctx, len(syss))
    for si in range(len(syss)):
        for d in range(3):
            assert np.array_equal(after[si][d], before[si][d]), (si, d)
    ctx.step(2)  # steps after tuning run (a new graph with the chosen shapes)
    chosen = {st: ctx.get_launch_shape(st) for st in range(4)}
    ctx.close()
    with open(cache) as f:
        assert len(json.load(f)) == 1
    ctx2 = _ctx(rt, syss, k0)
    res2 = ctx2.autotune(cache=cache)
    assert res2["source"] == "cache"
    assert {st: ctx2.get_launch_shape(st) for st in range(4)} == chosen
    ctx2.close()


def test_tuner_needs_grouped_products(rt, systems):
    """The FP64 path has no grouped products: the tuner refuses with RT_ESTATE."""
    syss, _ = systems
    ctx = rt.RT(syss[:1], prop="em", precision="fp64", r_Sinv=R, r_T=R, r_U=R, r_K=R, r_M=R)
    with pytest.raises(rt.RTError) as e:
        ctx.autotune()
    assert e.value.status == rt.RT_ESTATE
    ctx.close()

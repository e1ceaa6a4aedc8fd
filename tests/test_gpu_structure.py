"""Structural check of every triple list a context has built (rt_debug_check:
the lists and patterns are read back from the device and checked on the host
against the definition of the truncated product): one writer per output block,
operand indices inside their patterns, k ascending and complete.  Run for every
propagator in both precisions (after a kick, steps and the unitarity lists),
for items without triples (r_T < r_U / 2), block-diagonal patterns, a single
atom and a batched context of uneven systems with three kicks."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_5776_gb300 as m
    m.build()
    return m


def _exercise(rt, systems, n_kick=1, **params):
    ctx = rt.RT(systems, n_kick=n_kick, **params)
    ctx.inverse()
    for si, s in enumerate(systems if isinstance(systems, list) else [systems]):
        K0, _, _ = synth.ground_state_dense(s, int(np.sum(s.bsize)) // 2)
        for d in range(n_kick):
            ctx.set_density_dense(si, d, K0)
            ctx.kick(si, d, d, 1e-3)
    ctx.step(2)
    ctx.unitarity(0, True)
    ctx.unitarity(0, False)
    n = ctx.debug_check()
    ctx.close()
    return n


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("prop", ["em", "cn", "etrs", "m4"])
def test_every_list_of_each_propagator(rt, prop, precision):
    s = synth.diamond_system(2, "spd13", 6.0, 6.0)
    assert _exercise(rt, s, prop=prop, precision=precision, r_Sinv=6.0, r_T=7.0, r_U=6.0, r_K=6.0, r_M=6.0) > 0


@pytest.mark.parametrize("basis,radii", [("sp4", dict(r_Sinv=6.0, r_T=2.5, r_U=6.0, r_K=6.0, r_M=6.0)),
                                         ("spd13", dict(r_Sinv=2.0, r_T=2.0, r_U=2.0, r_K=2.0, r_M=2.0))])
def test_degenerate_patterns(rt, basis, radii):
    s = synth.diamond_system(2, basis, 6.0, 6.0)
    assert _exercise(rt, s, precision="fp32", **radii) > 0


def test_single_atom(rt):
    s = synth.build_system(np.array([[1.0, 2.0, 3.0]]), None, ["spd13"], 6.0, 6.0)
    assert _exercise(rt, s, r_Sinv=6.0, r_T=6.0, r_U=6.0, r_K=6.0, r_M=6.0) > 0


def test_batched_uneven_systems(rt):
    pos, species = synth.si_h_cluster(target=60)
    systems = [synth.diamond_system(2, "spd13", 6.0, 6.0), synth.build_system(pos, None, species, 5.0, 5.0),
               synth.diamond_system(3, "sp4", 6.0, 6.0, seed=3)]
    assert _exercise(rt, systems, n_kick=3, precision="fp32", r_Sinv=6.0, r_T=6.0, r_U=6.0, r_K=6.0,
                     r_M=6.0) > 0

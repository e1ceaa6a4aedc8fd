"""Degenerate and edge cases of the step, CUDA path against the oracle:
output blocks without triples (r_T < r_U / 2), block-diagonal patterns (radius
below the nearest-neighbour distance), a single atom, a one-term series
(U = I), and a zero kick.  FP64 at 1e-10 relative; the mixed path at its bar."""
import numpy as np
import pytest

import oracle
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


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _pair(rt, s, radii, steps, precision="fp64", kappa=1e-3, **extra):
    n_occ = int(np.sum(s.bsize)) // 2
    K0, _, _ = synth.ground_state_dense(s, n_occ)
    ctx = rt.RT(s, dt=0.05, precision=precision, **radii, **extra)
    ctx.inverse()
    ctx.set_density_dense(0, 0, K0)
    ctx.kick(0, 0, 0, kappa)
    ctx.step(steps)
    obs = ctx.observables(0, 0)
    Kg = ctx.matrix(0, rt.RT_MAT_K)
    ctx.close()
    ref = oracle.Propagator(s, oracle.Params(dt=0.05, **radii, **{k: v for k, v in extra.items()
                                                                 if k in ("taylor_terms", "prop")}))
    ref.set_density_dense(K0)
    ref.kick(0, kappa)
    rows = np.array([[z.real for z in ref.step()["obs"]] for _ in range(steps)])
    return obs, Kg, rows, ref


@pytest.mark.parametrize("basis,precision", [("spd13", "fp64"), ("spd13", "fp32"), ("sp4", "fp32")])
def test_items_without_triples(rt, basis, precision):
    """r_T = 2.5 A < r_U / 2: T^n blocks of P_U farther than 2 r_T have no triples
    and must come out zero."""
    s = synth.diamond_system(2, basis, 6.0, 6.0)
    radii = dict(r_Sinv=6.0, r_T=2.5, r_U=6.0, r_K=6.0, r_M=6.0)
    obs, Kg, rows, ref = _pair(rt, s, radii, 4, precision)
    bar = 1e-10 if precision == "fp64" else 1e-6
    assert relerr(obs[:, 3], rows[:, 1]) < bar
    assert relerr(obs[:, 1], rows[:, 0]) < bar
    if precision == "fp64":
        assert relerr(Kg, ref.K.val) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_block_diagonal_patterns(rt, precision):
    """Every radius below the nearest-neighbour distance (2.35 A): each atom sees
    only itself; the step reduces to independent 13 x 13 problems."""
    s = synth.diamond_system(2, "spd13", 6.0, 6.0)
    radii = dict(r_Sinv=2.0, r_T=2.0, r_U=2.0, r_K=2.0, r_M=2.0)
    ctx = rt.RT(s, **radii)
    rp, col = ctx.pattern(0, rt.RT_PAT_K)
    ctx.close()
    assert np.array_equal(col, np.arange(s.n_atoms)) and np.array_equal(rp, np.arange(s.n_atoms + 1))
    obs, Kg, rows, ref = _pair(rt, s, radii, 5, precision)
    bar = 1e-10 if precision == "fp64" else 1e-6
    assert relerr(obs[:, 3], rows[:, 1]) < bar
    if precision == "fp64":
        assert relerr(Kg, ref.K.val) < 1e-10


def test_single_atom(rt):
    pos = np.array([[1.0, 2.0, 3.0]])
    s = synth.build_system(pos, None, ["spd13"], 6.0, 6.0)
    radii = dict(r_Sinv=6.0, r_T=6.0, r_U=6.0, r_K=6.0, r_M=6.0)
    for precision in ("fp64", "fp32"):
        obs, Kg, rows, ref = _pair(rt, s, radii, 6, precision)
        bar = 1e-10 if precision == "fp64" else 1e-6
        assert relerr(obs[:, 1], rows[:, 0]) < bar, precision
        assert relerr(obs[:, 3], rows[:, 1]) < bar, precision


def test_one_term_series_keeps_k(rt):
    """taylor_terms = 1: U = I, K is only made hermitian (it already is)."""
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    radii = dict(r_Sinv=6.0, r_T=6.0, r_U=6.0, r_K=6.0, r_M=6.0)
    obs, Kg, rows, ref = _pair(rt, s, radii, 3, "fp64", taylor_terms=1)
    assert relerr(Kg, ref.K.val) < 1e-10
    assert np.allclose(obs[:, 3], obs[0, 3], rtol=1e-13, atol=0)


def test_zero_kick_ground_state_is_stationary(rt):
    """No field, no kick: the ground state moves only by truncation (FP64 vs oracle)."""
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    radii = dict(r_Sinv=8.0, r_T=8.0, r_U=8.0, r_K=8.0, r_M=8.0)
    obs, Kg, rows, ref = _pair(rt, s, radii, 10, "fp64", kappa=0.0)
    assert relerr(obs[:, 3], rows[:, 1]) < 1e-10
    # stationary up to the truncation of U (P_U misses one block pair per row)
    assert np.abs(obs[:, 3] - obs[0, 3]).max() < 1e-4 * abs(obs[0, 3])


def test_cn_fp64_iteration_count_validated(rt):
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    for bad in (0, 3):
        with pytest.raises(rt.RTError) as e:
            rt.RT(s, prop="cn", precision="fp32", hot_step_iters=2, hot_fp64_iters=bad)
        assert e.value.status == rt.RT_EINVAL


def test_cn_all_fp64_iterations_match_oracle_in_mixed_mode(rt):
    """hot_fp64_iters = hot_step_iters: the mixed CN path with every Hotelling
    iteration in FP64 (only the sandwich in FP32)."""
    s = synth.diamond_system(2, "spd13", 6.0, 6.0)
    radii = dict(r_Sinv=6.0, r_T=6.0, r_U=6.0, r_K=6.0, r_M=6.0)
    obs, Kg, rows, ref = _pair(rt, s, radii, 6, "fp32", prop="cn", hot_fp64_iters=2)
    assert relerr(obs[:, 3], rows[:, 1]) < 1e-6

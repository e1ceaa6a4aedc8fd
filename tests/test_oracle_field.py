"""Pin of the external-field path of the oracle (Sec. II.B: dv = -E_j(t) r,
H(t) = H0 - E(t) D_j; Gaussian pulse of Sec. IV.A) through the delta-kick
limit: in linear response a pulse of area kappa = int E dt centred at t0
produces, after it has passed, the response of a kick of strength kappa at t0,
with corrections that vanish with the pulse width (second order in
sigma * omega).  This fixes the sign and scale of the field term, the midpoint
sampling of eq. EM and the kick's exp(+i kappa S^-1 D)."""
import math

import numpy as np

import oracle
import synth


def _small_open_system():
    # one conventional diamond cell as an open 8-atom cluster (well conditioned)
    pos, _ = synth.diamond_positions(1)
    return synth.build_system(pos, None, ["sp4"] * 8, 20.0, 20.0)


def _response(sys, K0, dt, nsteps, field=None, kick=None):
    p = oracle.Params(r_Sinv=50.0, r_T=50.0, r_U=50.0, r_K=50.0, r_M=50.0, dt=dt, field=field, field_dir=0,
                      taylor_terms=10)
    pr = oracle.Propagator(sys, p)
    pr.set_density_dense(K0)
    p0 = oracle.observables(pr.K, pr.S, pr.D)[1].real
    if kick is not None:
        pr.kick(0, kick)
    out = []
    for _ in range(nsteps):
        o = pr.step()
        out.append((o["t"], o["obs"][1].real - p0))
    return np.array(out)


def test_pulse_approaches_kick():
    s = _small_open_system()
    n_occ = s.n // 2
    K0, _, _ = synth.ground_state_dense(s, n_occ)
    dt, t0, kappa = 0.01, 0.5, 1e-4
    T = 2.0
    n = int(round(T / dt))
    devs = []
    for sigma in (0.08, 0.04):
        E0 = kappa / (sigma * math.sqrt(2 * math.pi))
        pulse = _response(s, K0, dt, n, field={"kind": "gaussian", "E0": E0, "t0": t0, "sigma": sigma})
        # kick applied at t0: run the free propagation from t0 (H is static after it)
        kick = _response(s, K0, dt, n - int(round(t0 / dt)), kick=kappa)
        tail = pulse[int(round((t0 + 6 * sigma) / dt)):]
        tk = {round(t + t0, 6): v for t, v in kick}
        diffs = [v - tk[round(t, 6)] for t, v in tail if round(t, 6) in tk]
        amp = np.abs(kick[:, 1]).max()
        assert amp > 0
        devs.append(np.abs(diffs).max() / amp)
    # same sign and scale (1e-3 at these widths) and converging as sigma^2
    assert devs[0] < 2e-3
    assert devs[1] < devs[0] / 3.0

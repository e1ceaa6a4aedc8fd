"""Writes the stored trajectories of the 64-atom correctness workloads.

Workload 1: 2x2x2 conventional diamond cells (64 atoms, a = 5.43 A, seeded
jitter 0.05 A), 4 s+p functions per atom (n = 256), r_S = r_H = 6 A and all
step radii 8 A (nearly dense), K0 by dense generalised diagonalisation at half
filling, delta kick kappa = 1e-3 along x (Sec. II.B), dt = 0.05 a.u., 200
steps of the EM propagator (Sec. II.A, eq. EM) and of the Crank-Nicolson form.

Workload 2 (13 functions per atom, the block size of the mixed-precision
reference split): the same cell with 2s+2p+1d atoms (n = 832), r_S = r_H = 6 A,
every step radius 6 A (truncated: 42 of 64 blocks per atom), K0 by dense
diagonalisation with two doubly occupied states per atom, dt = 0.05 a.u., 200
steps: the EM full step (U rebuilt at every midpoint) after a delta kick
kappa = 1e-3 along x and under a Gaussian pulse along x (E0 = 5e-3, t0 = 0.5,
sigma = 0.3, omega = 0.8 a.u.; no kick), and the propagation step (U built
once at t = 0, then reused) after the kick for the CN, ETRS and M4
propagators.

Every value comes from the CPU oracle (oracle/); run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

STEPS = 200
KAPPA = 1e-3
RADII = dict(r_Sinv=8.0, r_T=8.0, r_U=8.0, r_K=8.0, r_M=8.0)


def workload():
    s = synth.diamond_system(2, "sp4", 6.0, 6.0)
    K0, _, gap = synth.ground_state_dense(s, s.n // 2)
    return s, K0, gap


def trajectory(prop, steps=STEPS):
    s, K0, _ = workload()
    ref = oracle.Propagator(s, oracle.Params(dt=0.05, prop=prop, **RADII))
    ref.set_density_dense(K0)
    ref.kick(0, KAPPA)
    rows = []
    for _ in range(steps):
        out = ref.step()
        rows.append([out["t"]] + [z.real for z in out["obs"]])
    return np.array(rows)


def path(prop):
    return os.path.join(HERE, f"diamond64_sp4_r8_kick_x_{prop}.txt")


RADII13 = dict(r_Sinv=6.0, r_T=6.0, r_U=6.0, r_K=6.0, r_M=6.0)
PULSE13 = {"kind": "gaussian", "E0": 5e-3, "t0": 0.5, "sigma": 0.3, "omega": 0.8}


def workload13():
    s = synth.diamond_system(2, "spd13", 6.0, 6.0)
    K0, _, gap = synth.ground_state_dense(s, 2 * s.n_atoms)
    return s, K0, gap


def trajectory13(prop, drive, rebuild, steps=STEPS):
    """drive: 'kick' (delta kick along x at t = 0) or 'pulse' (Gaussian pulse along x)."""
    s, K0, _ = workload13()
    field = PULSE13 if drive == "pulse" else None
    ref = oracle.Propagator(s, oracle.Params(dt=0.05, prop=prop, field=field, field_dir=0, **RADII13))
    ref.set_density_dense(K0)
    if drive == "kick":
        ref.kick(0, KAPPA)
    rows = []
    for _ in range(steps):
        out = ref.step(rebuild=rebuild)
        rows.append([out["t"]] + [z.real for z in out["obs"]])
    return np.array(rows)


CASES13 = [("em", "kick", True), ("em", "pulse", True), ("cn", "kick", False), ("etrs", "kick", False),
           ("m4", "kick", False)]


def path13(prop, drive, rebuild):
    return os.path.join(HERE, f"diamond64_spd13_r6_{drive}_x_{prop}_{'full' if rebuild else 'prop'}.txt")


def main(which=("sp4", "spd13")):
    if "spd13" in which:
        for prop, drive, rebuild in CASES13:
            rows = trajectory13(prop, drive, rebuild)
            what = "full step (U rebuilt every step)" if rebuild else "propagation step (U built once at t = 0)"
            hdr = (f"64-atom diamond, 13 functions/atom, radii 6 A, {drive} along x, dt 0.05, {STEPS} steps, "
                   f"propagator {prop.upper()} (Sec. II.A), {what}; written by tests/golden/make_golden.py "
                   "from the oracle\ncolumns: t, Re Tr(K S), Re Tr(K Dx), Re Tr(K Dy), Re Tr(K Dz)")
            np.savetxt(path13(prop, drive, rebuild), rows, fmt="%.17e", header=hdr)
            print(path13(prop, drive, rebuild), flush=True)
    if "sp4" not in which:
        return
    for prop in ("em", "cn"):
        rows = trajectory(prop)
        hdr = (f"64-atom diamond, 4 functions/atom, radii 8 A, kick 1e-3 along x, dt 0.05, {STEPS} steps, "
               f"propagator {prop.upper()} (Sec. II.A); written by tests/golden/make_golden.py from the oracle\n"
               "columns: t, Re Tr(K S), Re Tr(K Dx), Re Tr(K Dy), Re Tr(K Dz)")
        np.savetxt(path(prop), rows, fmt="%.17e", header=hdr)
        print(path(prop))


if __name__ == "__main__":
    main(tuple(sys.argv[1:]) or ("sp4", "spd13"))

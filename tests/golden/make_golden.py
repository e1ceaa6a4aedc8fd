"""Writes the stored trajectories of the 64-atom correctness workload.

Workload: 2x2x2 conventional diamond cells (64 atoms, a = 5.43 A, seeded
jitter 0.05 A), 4 s+p functions per atom (n = 256), r_S = r_H = 6 A and all
step radii 8 A (nearly dense), K0 by dense generalised diagonalisation at half
filling, delta kick kappa = 1e-3 along x (Sec. II.B), dt = 0.05 a.u., 200
steps of the EM propagator (Sec. II.A, eq. EM) and of the Crank-Nicolson form.

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


def main():
    for prop in ("em", "cn"):
        rows = trajectory(prop)
        hdr = (f"64-atom diamond, 4 functions/atom, radii 8 A, kick 1e-3 along x, dt 0.05, {STEPS} steps, "
               f"propagator {prop.upper()} (Sec. II.A); written by tests/golden/make_golden.py from the oracle\n"
               "columns: t, Re Tr(K S), Re Tr(K Dx), Re Tr(K Dy), Re Tr(K Dz)")
        np.savetxt(path(prop), rows, fmt="%.17e", header=hdr)
        print(path(prop))


if __name__ == "__main__":
    main()

"""Write the stored expected values of the shear-channel workload (calls only oracle/).

The benchmark's default workload (periodic-in-x channel, k = 3, ARS(3,4,3), dt = 2e-3, the seeded
shear layer u = (tanh((y - 1/2)/0.05), 1e-3 sin 2 pi x) plus N(0,1) 1e-4 noise per nodal value,
seed 0) on an N x N mesh (N = 32, or the first argument): the oracle projects the field to divergence-free (Step II with c = 1),
reconstructs the pressure (Sec. 2.7) and takes one IMEX step of Alg. 1 with monolithic direct
stage solves (the exact stage solutions). The result (nodal Q, p, lambda in the exchange layout)
goes to c2_step1_<N>.npz beside this script.

    python tests/golden/make_c2_golden.py [N]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Mesh, HDG, Oracle, TABLEAUS   # noqa: E402
import hdg_workloads as W                          # noqa: E402

K, DT, WIDTH, AMP, NOISE, SEED = 3, 2e-3, 0.05, 1e-3, 1e-4, 0


def main(N=32):
    h = HDG(Mesh(N, periodic_x=True), K)
    o = Oracle(h)
    raw = W.nodal_velocity(N, K, lambda x, y: W.shear_layer(x, y, WIDTH, AMP), noise=NOISE, seed=SEED)
    Q, _, _ = o.div_free_project(raw.reshape(-1))
    _, p, lam = o.reconstruct_pressure(Q)
    Q1, p1, l1 = o.imex_step(TABLEAUS['ARS343'](), DT, 0.0, Q, p, lam, solver='direct')
    np.savez_compressed(os.path.join(HERE, f'c2_step1_{N}.npz'), Q=Q1, p=p1, lam=l1,
                        meta=np.array([N, K, DT, WIDTH, AMP, NOISE, SEED]))


if __name__ == '__main__':
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 32)

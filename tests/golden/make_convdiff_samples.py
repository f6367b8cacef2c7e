"""Writes sampled oracle values of phi_l(-tau*A)v for the full-size 3D convection-diffusion
workload (n = 128 per dimension, 2,097,152 unknowns, tau = 1e-2, l = 0..3, v ~ U(-1,1)
seed 0).

Calls only the oracle (O3: scipy's expm_multiply on the sparse augmented matrix, the plain
definition of Eq. (3)) and the seeded input generator.  The full vectors are too large to
store, so the file keeps 16384 seeded sample indices with the value of every phi_l there,
plus each full phi_l's 2-norm and inf-norm.  Run from the repository root:

    python tests/golden/make_convdiff_samples.py [n]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import phi as P  # noqa: E402


def main(n: int = 128, samples: int = 16384):
    prob = W.convdiff3d(n=n, tau=1e-2, l_max=3, tol=1e-10, seed=0)
    v = prob.vector()
    t0 = time.time()
    out = P.phi_sparse(prob.factors, prob.tau, v, prob.l_max)
    dt = time.time() - t0
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(prob.N, size=samples, replace=False))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        f"convdiff3d_n{n}_tau1e-2_seed0_samples.txt")
    with open(path, "w") as f:
        f.write(f"# phi_l(-tau*A)v, A^d = -0.01*D2 + D1_upwind on n={n} interior points of [0,1],\n")
        f.write(f"# tau=1e-2, v = workloads.uniform_vector(({n},{n},{n}), seed=0); oracle O3 "
                f"(scipy.sparse.linalg.expm_multiply), {dt:.1f} s\n")
        f.write("# norm2 " + " ".join(repr(float(np.linalg.norm(out[l]))) for l in range(4)) + "\n")
        f.write("# norminf " + " ".join(repr(float(np.max(np.abs(out[l])))) for l in range(4)) + "\n")
        f.write("# index phi_0 phi_1 phi_2 phi_3\n")
        for i in idx:
            f.write(f"{i} " + " ".join(repr(float(out[l][i])) for l in range(4)) + "\n")
    print(path, dt)


def load(path):
    """Returns (idx, values (4, S), norm2 (4,), norminf (4,))."""
    norm2 = norminf = None
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("# norm2"):
                norm2 = np.array([float(t) for t in line.split()[2:]])
            elif line.startswith("# norminf"):
                norminf = np.array([float(t) for t in line.split()[2:]])
            elif not line.startswith("#") and line.strip():
                rows.append([float(t) for t in line.split()])
    a = np.array(rows)
    return a[:, 0].astype(np.int64), a[:, 1:].T.copy(), norm2, norminf


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 128)

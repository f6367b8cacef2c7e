"""The 3D convection-diffusion workload at its full size (A^d = -0.01*D2 + D1_upwind on n = 128
points per dimension, 2,097,152 unknowns, tau = 1e-2, phi_0..phi_3, v ~ U(-1,1) seed 0) against
the stored oracle values (O3: expm_multiply on the sparse augmented matrix, written by
tests/golden/make_convdiff_samples.py, which calls only the oracle).

Gates (relative 2-norm error per phi_l, estimated on the stored sample indices as
rms(diff) / rms(phi_l) with rms(phi_l) from the stored full-vector 2-norm):
  * float64 path, Gauss, tol 1e-10: 1e-10;
  * mixed path at tol 1e-6 with 3 digit slices (FP32-class products): 1e-6;
  * mixed path at tol 1e-6 with the slice count the library picks for it (4): 1e-6;
  * mixed path as timed by the benchmark (tol 1e-9, 4 digit slices): 1e-8, the accuracy the
    throughput metric is quoted at;
  * mixed path at tol 1e-10 (5 digit slices): 1e-10.
Each case uses the plan the library makes for that tolerance (Algorithm 5's (s, m)), so the
quadrature, the squaring steps and the tensor-core digit products all enter the error.
"""
import math
import os
import sys

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "convdiff3d_n128_tau1e-2_seed0_samples.txt")


def _golden():
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_convdiff_samples import load
    return load(GOLDEN)


def _sampled_errors(out, golden, N):
    idx, vals, norm2, _ = golden
    errs = []
    for l in range(vals.shape[0]):
        d = out[l][idx] - vals[l]
        errs.append(float(np.sqrt(np.mean(d * d)) / (norm2[l] / math.sqrt(N))))
    return errs


@pytest.fixture(scope="module")
def problem():
    prob = W.convdiff3d()
    assert prob.N == 128 ** 3
    return prob, torch.from_numpy(prob.vector()).cuda(), _golden()


CASES = [
    # (precision, tol, slices (0 = from tol), gate, expected slices)
    ("fp64", 1e-10, 0, 1e-10, 0),
    ("mixed", 1e-6, 3, 1e-6, 3),
    ("mixed", 1e-6, 0, 1e-6, 4),
    ("mixed", 1e-9, 4, 1e-8, 4),
    ("mixed", 1e-10, 0, 1e-10, 5),
]


@pytest.mark.parametrize("prec,tol,slices,gate,expect_slices", CASES)
def test_convdiff3d_128_full_size_against_oracle(problem, prec, tol, slices, gate, expect_slices):
    import paper_2211_00696_gb300 as pk
    prob, V, golden = problem
    pid = pk.PREC_FP64 if prec == "fp64" else pk.PREC_OZAKI_BF16
    plan = pk.Plan(prob.factors, prob.tau, prob.l_max, tol, precision=pid, slices=slices)
    info = plan.info()
    assert info["slices"] == expect_slices
    out = plan.apply(V).cpu().numpy()
    plan.check_status()
    assert np.all(np.isfinite(out))
    errs = _sampled_errors(out, golden, prob.N)
    print(f"{prec} tol={tol:g} slices={info['slices']} (s,m)=({info['s']},{info['m']}): errors {errs}")
    for l, e in enumerate(errs):
        assert e <= gate, (prec, tol, l, e)
    plan.close()


def test_convdiff3d_128_repeated_applies_are_bitwise_equal(problem):
    """The graph-replayed mixed apply is deterministic: two applies of the same input agree bit
    for bit (no race between the grouped launches of one apply)."""
    import paper_2211_00696_gb300 as pk
    prob, V, _ = problem
    plan = pk.Plan(prob.factors, prob.tau, prob.l_max, 1e-9, precision=pk.PREC_OZAKI_BF16, slices=4)
    a = plan.apply(V).cpu().numpy()
    b = plan.apply(V).cpu().numpy()
    plan.check_status()
    assert np.array_equal(a, b)
    plan.close()

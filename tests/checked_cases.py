"""Cases for the bounds-checked library (libphikron_checked.so), run by test_gpu_checked.py in
a child process with PHIKRON_CHECKED=1 (a process loads one of the two libraries).

Small and uneven shapes through every apply path that has kernels: the float64 path (Gauss,
Clenshaw-Curtis, adaptive Clenshaw-Curtis, the Remark's combination), the mixed path on
padded sizes (3..8 points per dimension) and on multiples of 16 with each mode-kernel variant
(warp-specialised, single-role, double-buffered) and the fused node-weight pass, half-step and
skip_phi0 outputs, batched applies, the exponential integrators, the float64 Kronecker
products (with and without a work buffer) and the batched expm.  Each case records its error
against the oracle and the checked build's violation record after the case.

    python tests/checked_cases.py [--shrink]

--shrink runs one mixed apply only (the parent sets PHIKRON_CHECKED_SHRINK so that the last
bytes of every library allocation count as outside) and reports check_status's code.  Prints
one JSON line.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_2211_00696_gb300 as pk  # noqa: E402
from paper_2211_00696_gb300 import phikron as B  # noqa: E402
import workloads as W  # noqa: E402
from oracle import phi as P  # noqa: E402
from oracle import erk as OE  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rand_factor(n, seed):
    """A nonsymmetric factor with a dominant negative diagonal (a convection-diffusion-like
    operator on n points)."""
    rng = np.random.default_rng(seed)
    return W.convdiff_factor(n) + 0.1 * rng.standard_normal((n, n)) / n


class Runner:
    def __init__(self):
        self.cases = []

    def record(self, name, err, gate):
        torch.cuda.synchronize()
        v = B.checked_violation()
        self.cases.append({"name": name, "err": float(err), "gate": float(gate), "violation": v})

    def phi_case(self, name, factors, tau, p, tol, gate, **kw):
        N = int(np.prod([a.shape[0] for a in factors]))
        v = W.uniform_vector((N,), 7)
        plan = pk.Plan(factors, tau, p, tol, **kw)
        out = plan.apply(dev(v)).cpu().numpy()
        plan.check_status()
        # the dense augmented-matrix definition (O1) on small N, the sparse one (O3) above
        ref = P.phi_dense if N <= 1500 else P.phi_sparse
        exact = ref(factors, tau, v, p)
        rows = range(1 if kw.get("skip_phi0") else 0, p + 1)
        err = max(P.rel_err_2(out[l], exact[l]) for l in rows)
        if kw.get("half_step"):
            half = ref(factors, tau / 2, v, p)
            err = max(err, max(P.rel_err_2(out[p + 1 + l], half[l]) for l in rows))
        plan.close()
        self.record(name, err, gate)


def run_all():
    R = Runner()
    F64, MIX = pk.PREC_FP64, pk.PREC_OZAKI_BF16
    small = [rand_factor(n, 10 + n) for n in (3, 5, 4)]
    R.phi_case("fp64 gauss 3x5x4", small, 0.05, 3, 1e-10, 1e-9, precision=F64)
    R.phi_case("fp64 cc 7x3", [rand_factor(7, 1), rand_factor(3, 2)], 0.05, 2, 1e-10, 1e-9, precision=F64,
               quad=pk.QUAD_CC)
    R.phi_case("fp64 adaptive cc 6x5", [rand_factor(6, 3), rand_factor(5, 4)], 0.05, 2, 1e-10, 1e-8,
               precision=F64, quad=pk.QUAD_CC_ADAPTIVE)
    R.phi_case("mixed padded 3x5x4", small, 0.05, 3, 1e-9, 5e-8, precision=MIX, slices=4)
    R.phi_case("mixed padded 8x6x7 s>0", [rand_factor(n, 20 + n) for n in (8, 6, 7)], 2.0, 3, 1e-9, 5e-8,
               precision=MIX, slices=4, force_s=2, force_m=12)
    R.phi_case("mixed padded 5x8 half step", [rand_factor(5, 30), rand_factor(8, 31)], 1.0, 2, 1e-9, 5e-8,
               precision=MIX, slices=4, half_step=True, force_s=2, force_m=12)
    R.phi_case("mixed padded 7x4 skip phi0", [rand_factor(7, 32), rand_factor(4, 33)], 0.5, 2, 1e-9, 5e-8,
               precision=MIX, slices=4, skip_phi0=True)
    R.phi_case("mixed 1D n=6", [rand_factor(6, 34)], 0.5, 3, 1e-9, 5e-8, precision=MIX, slices=4)
    shape16 = [rand_factor(n, 40 + n) for n in (16, 32, 48)]
    for kern in ("ws", "classic", "db"):
        os.environ["PHIKRON_MODE_KERNEL"] = kern
        fac = shape16 if kern != "db" else [rand_factor(64, 50), rand_factor(64, 51)]
        R.phi_case(f"mixed {kern} kernel", fac, 0.05, 3, 1e-9, 5e-8, precision=MIX, slices=4)
    os.environ.pop("PHIKRON_MODE_KERNEL", None)
    os.environ["PHIKRON_FUSED_WEIGHTS"] = "1"
    R.phi_case("mixed fused pass 16x32x48", shape16, 0.05, 3, 1e-9, 5e-8, precision=MIX, slices=4)
    R.phi_case("mixed fused pass 16x48 s=0", [rand_factor(16, 60), rand_factor(48, 61)], 0.02, 2, 1e-9, 5e-8,
               precision=MIX, slices=4)
    os.environ.pop("PHIKRON_FUSED_WEIGHTS", None)

    # combination of the Remark after Algorithm 2 (float64, s = 0)
    fac = [rand_factor(5, 70), rand_factor(6, 71)]
    plan = pk.Plan(fac, 0.02, 3, 1e-12, precision=F64, force_s=0)
    N = 30
    Bv = np.stack([W.uniform_vector((N,), 80 + j) for j in range(3)])
    got = plan.apply_combo(dev(Bv)).cpu().numpy()
    want = sum(P.phi_dense(fac, 0.02, Bv[j], 3)[j + 1] for j in range(3))
    plan.close()
    R.record("fp64 combination 5x6", P.rel_err_2(got, want), 1e-10)

    # batched applies: two instances x two right-hand sides
    plans = [pk.Plan([W.laplacian_factor(n, 0.5) for n in shape], 1e-3, 2, 1e-9, precision=MIX, slices=4)
             for shape in ((16, 32, 16), (32, 16, 16))]
    bt = pk.Batch(plans, nrhs=2)
    Vs = [W.uniform_vector((2, p.N), 90 + i).reshape(2, p.N) for i, p in enumerate(plans)]
    outs = bt.apply([dev(v) for v in Vs])
    bt.check_status()
    err = 0.0
    for i, p in enumerate(plans):
        o = outs[i].cpu().numpy().reshape(2, 3, p.N)
        for r in range(2):
            ex = P.phi_sparse(p._facs, 1e-3, Vs[i][r], 2)
            err = max(err, max(P.rel_err_2(o[r, l], ex[l]) for l in range(3)))
    bt.close()
    for p in plans:
        p.close()
    R.record("batch 2 instances x 2 rhs", err, 5e-8)

    # exponential integrators (Allen-Cahn), float64 and mixed, against the oracle's stepper
    a = W.periodic_diffusion_factor(16, 1e-2)
    u0 = W.uniform_vector((256,), 5) * 0.5
    for prec, gate in ((F64, 1e-9), (MIX, 1e-7)):
        it = pk.Integrator([a, a], 0.05, pk.ERK_RK2, 1e-10, precision=prec, slices=4 if prec == MIX else 0)
        U = dev(u0.copy())
        it.step(U, 2)
        it.check_status()
        it.close()
        tab = OE.rk2()
        A_apply = lambda u: OE.kron_sum_apply([a, a], u)  # noqa: E731
        phi = lambda tau, v, p: P.phi_dense([a, a], tau, v, p)  # noqa: E731
        ref = OE.integrate(tab, u0, 0.05, 2, OE.allen_cahn, A_apply, phi)
        R.record(f"integrator rk2 {'fp64' if prec == F64 else 'mixed'}", P.rel_err_2(U.cpu().numpy(), ref), gate)

    # float64 Kronecker products and the batched expm
    mats = [np.random.default_rng(100 + d).standard_normal((n, n)) for d, n in enumerate((3, 4, 5))]
    V = np.random.default_rng(110).standard_normal(60)
    got = pk.phikron.kron_apply_f64([dev(m) for m in mats], dev(V)).cpu().numpy()
    want = P.apply_kron(mats, V.reshape(3, 4, 5)).ravel()
    R.record("kron apply 3x4x5", np.max(np.abs(got - want)) / np.max(np.abs(want)), 1e-13)
    import ctypes as C
    L = pk.lib()
    dm = [dev(m) for m in mats]
    ns = (C.c_int * 3)(3, 4, 5)
    ptrs = (C.c_void_p * 3)(*[m.data_ptr() for m in dm])
    dv = dev(V)
    out = torch.empty_like(dv)
    rc = L.phikron_kron_apply_f64_noalloc(3, ns, ptrs, dv.data_ptr(), out.data_ptr(), None)
    assert rc == 0, L.phikron_last_error()
    R.record("kron apply no-alloc 3x4x5", np.max(np.abs(out.cpu().numpy() - want)) / np.max(np.abs(want)), 1e-13)
    import scipy.linalg
    A3 = np.stack([rand_factor(7, 120 + b) for b in range(3)])
    scales = (-0.5, -1.0, -2.0)
    E = pk.phikron.expm_batched(dev(A3), list(scales)).cpu().numpy()
    err = 0.0
    for b, c in enumerate(scales):
        ref = scipy.linalg.expm(c * A3[b])
        err = max(err, np.linalg.norm(E[b] - ref) / np.linalg.norm(ref))
    R.record("expm batched 3 x 7x7", err, 1e-12)
    return R.cases


def run_shrink():
    fac = [rand_factor(n, 10 + n) for n in (16, 32)]
    v = W.uniform_vector((512,), 7)
    plan = pk.Plan(fac, 0.05, 2, 1e-9, precision=pk.PREC_OZAKI_BF16, slices=4)
    plan.apply(dev(v))
    torch.cuda.synchronize()
    code = 0
    try:
        plan.check_status()
    except pk.PhikronError as e:
        code = e.code
    viol = B.checked_violation()
    plan.close()
    return {"status_code": code, "violation": viol}


def main():
    if not B.CHECKED or pk.lib().phikron_checked() != 1:
        raise SystemExit("run with PHIKRON_CHECKED=1 and a built libphikron_checked.so")
    res = {"checked": 1}
    if "--shrink" in sys.argv:
        res.update(run_shrink())
    else:
        res["cases"] = run_all()
    print(json.dumps(res))


if __name__ == "__main__":
    main()

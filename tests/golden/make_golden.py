"""Writes the stored expected values under tests/golden/ by calling only the oracle.

  hartree1d_n20000_p50_optimum.json   f* of the 1D Hartree workload (n = 20000, p = 50,
                                      alpha = 1, q = 1/4, seeded orthonormal start): the
                                      oracle's PCAL (beta = 1e3) run to relative KKT 1e-9,
                                      then orthonormalised (Householder QR).
  stencil3d_n262144_p256_optimum.json f* of the 3D workload (7-point Dirichlet Laplacian on
                                      64^3 plus the seeded potential V iid U[0,1], p = 256):
                                      half the sum of the 256 smallest eigenvalues (Ky Fan),
                                      oracle.objectives.trace_min_optimum (about 40 minutes).
  stencil3d_separable_n2097152_p1024_optimum.json
                                      f* of the 128^3, p = 1024 companion workload whose potential
                                      is separable, V = v_x(x) + v_y(y) + v_z(z) (each v_k iid
                                      U[0, 1/3], seeded stream 3 of configuration 5): half the sum
                                      of the 1024 smallest eigenvalues, exact through the
                                      Kronecker-sum spectrum (oracle.objectives.
                                      separable_trace_min_optimum, seconds).
  section54_n10000_p1000.json         Section 5.4's parallel forms of Problems 1 (blocks of 5
                                      rows, alpha = 1, q = 1/2) and 2 (tridiagonal A, random
                                      G_lin), n = 10000, p = 1000, seeded starts: the oracle's PCAL
                                      (beta = 1, eq. lambda2, ABB) to relative KKT 1e-6 and 1e-8,
                                      iterations, f and feasibility (a few minutes).

Run from the repository root:
    python tests/golden/make_golden.py [hartree1d] [stencil3d] [section54] [separable128]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import objectives as oo  # noqa: E402
from oracle import plam as op  # noqa: E402
from workloads import (stencil3d_separable_potential, workload_block_hartree,  # noqa: E402
                       workload_hartree1d, workload_stencil3d, workload_tridiag_linear)


def hartree_optimum():
    w = workload_hartree1d()
    obj = oo.HartreeObjective(w.n, w.alpha, w.quad_scale)
    t0 = time.time()
    r = op.solve(obj, w.X0, variant="pcal", beta=1000.0, tol=1e-9, maxit=20000, record=False)
    assert r.converged
    return {"workload": w.name, "n": w.n, "p": w.p, "alpha": w.alpha, "quad_scale": w.quad_scale,
            "beta": 1000.0, "tol_kkt_rel": 1e-9, "f_star": r.f_orth, "kkt_orth": r.kkt_orth,
            "feas_orth": r.feas_orth, "K0": r.K0, "oracle_iters": r.iters,
            "oracle_seconds": round(time.time() - t0, 1),
            "source": "oracle/plam.py solve() run by tests/golden/make_golden.py"}


def stencil_optimum():
    w = workload_stencil3d(m=64, p=256)
    obj = oo.Stencil3DObjective(w.m, w.V)
    t0 = time.time()
    f, ev = oo.trace_min_optimum(obj.H, w.p)
    return {"workload": w.name, "n": w.n, "p": w.p, "m": w.m, "f_star": f,
            "lambda_1": float(ev[0]), "lambda_p": float(ev[-1]),
            "oracle_seconds": round(time.time() - t0, 1),
            "source": "oracle/objectives.py trace_min_optimum() run by tests/golden/make_golden.py"}


def separable128_optimum():
    m, p = 128, 1024
    t0 = time.time()
    V, vx, vy, vz = stencil3d_separable_potential(m)
    f, ev = oo.separable_trace_min_optimum(vx, vy, vz, p)
    return {"workload": "stencil3d_separable_n2097152_p1024", "n": m ** 3, "p": p, "m": m,
            "potential": "V[x + m (y + m z)] = v_x[x] + v_y[y] + v_z[z], v_k iid U[0, 1/3], "
                         "workloads.stencil3d_separable_potential (seed stream 3 of config 5)",
            "f_star": f, "lambda_1": float(ev[0]), "lambda_p": float(ev[p - 1]),
            "lambda_p_plus_1": float(ev[p]), "gap": float(ev[p] - ev[p - 1]),
            "oracle_seconds": round(time.time() - t0, 1),
            "source": "oracle/objectives.py separable_trace_min_optimum() run by "
                      "tests/golden/make_golden.py"}


def section54_runs():
    out = {}
    for w in (workload_block_hartree(), workload_tridiag_linear()):
        obj = oo.objective_for(w)
        d = {"n": w.n, "p": w.p, "alpha": w.alpha, "quad_scale": w.quad_scale, "block": w.block,
             "beta": 1.0}
        for tol in (1e-6, 1e-8):
            t0 = time.time()
            r = op.solve(obj, w.X0, variant="pcal", beta=1.0, tol=tol, maxit=3000, record=False)
            assert r.converged
            d[f"tol_{tol:g}"] = {"iters": r.iters, "f_stop": r.f_stop, "f_orth": r.f_orth,
                                 "kkt_orth": r.kkt_orth, "feas_orth": r.feas_orth, "K0": r.K0,
                                 "oracle_seconds": round(time.time() - t0, 1)}
        out[w.name] = d
    out["source"] = "oracle/plam.py solve() run by tests/golden/make_golden.py"
    return out


if __name__ == "__main__":
    which = sys.argv[1:] or ["hartree1d"]
    if "hartree1d" in which:
        d = hartree_optimum()
        with open(os.path.join(HERE, "hartree1d_n20000_p50_optimum.json"), "w") as fh:
            json.dump(d, fh, indent=1)
        print(d)
    if "section54" in which:
        d = section54_runs()
        with open(os.path.join(HERE, "section54_n10000_p1000.json"), "w") as fh:
            json.dump(d, fh, indent=1)
        print(d)
    if "separable128" in which:
        d = separable128_optimum()
        with open(os.path.join(HERE, "stencil3d_separable_n2097152_p1024_optimum.json"), "w") as fh:
            json.dump(d, fh, indent=1)
        print(d)
    if "stencil3d" in which:
        d = stencil_optimum()
        with open(os.path.join(HERE, "stencil3d_n262144_p256_optimum.json"), "w") as fh:
            json.dump(d, fh, indent=1)
        print(d)

"""bench.py's command-line contract, checked without a GPU.

* The reference arm (the FP64 oracle on the host cores, the only reference this
  paper has) prints one JSON line with the keys the benchmark contract names.
* The default workload (128^3, p = 1024) samples the oracle on the grid's first
  z-planes, a Dirichlet problem of its own whose cost per iteration is the full
  grid's times the row fraction.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_the_contract_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "3", "--slab-planes", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d, key
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "iters/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "stencil3d_n2097152_p1024"
    assert "the first 1 of the 128 z-planes (n = 16384" in d["cpu_baseline"]["sample"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_slab_sample_of_the_128_grid():
    """The oracle's sample of the 128^3 workload: the first 8 z-planes (n = 131072 rows, the
    same p), the potential of exactly those grid points (index x + 128 (y + 128 z), z < 8), and
    an orthonormal start; its rate scales to the full grid by 8 / 128."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from workloads import rng_for, uniform_potential
    wl = dict(bench.WORKLOADS["stencil3d_128"], p=16)      # a narrow start keeps the test quick
    V = uniform_potential(wl["n"], rng_for(5, 0))
    grid, Vs, X0, ns = bench.slab_problem(wl, V, wl["slab_planes"])
    assert grid == (128, 128, 8) and ns == 131072 and ns / wl["n"] == 8 / 128
    assert np.array_equal(Vs, V.reshape(128, 128, 128)[:8].ravel())
    assert X0.shape == (ns, 16) and np.abs(X0.T @ X0 - np.eye(16)).max() < 1e-13


def test_width_override_applies_to_section54_workloads_only():
    """--p sets Section 5.4's width (the paper sweeps p = 500 ... 2500 at n = 10000) and names the
    workload by it; other workloads and widths above n/2 are refused before any GPU work."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    wl = bench.workload_config(argparse.Namespace(workload="block_hartree", p=2500))
    assert wl["p"] == 2500 and wl["name"] == "block_hartree_n10000_p2500_b5"
    assert bench.WORKLOADS["block_hartree"]["p"] == 1000
    wl = bench.workload_config(argparse.Namespace(workload="tridiag_linear", p=0))
    assert wl["p"] == 1000 and wl["name"] == "tridiag_linear_n10000_p1000"
    r = _run("--workload", "hartree1d", "--p", "500")
    assert r.returncode != 0 and "--p applies" in (r.stderr + r.stdout)
    r = _run("--workload", "block_hartree", "--p", "6000")
    assert r.returncode != 0 and "--p must lie" in (r.stderr + r.stdout)
    wl = bench.workload_config(argparse.Namespace(workload="block_hartree", p=2000, beta=4.1))
    assert wl["beta"] == 4.1 and wl["name"] == "block_hartree_n10000_p2000_b5_beta4.1"
    r = _run("--workload", "hartree1d", "--beta", "2")
    assert r.returncode != 0 and "--beta applies" in (r.stderr + r.stdout)


def test_output_feasibility_check_of_the_bench():
    """bench's check of the output, ||Q^T Q - I||_F on the (p, ld) column-major layout the library
    writes: about 1e-15 for an orthonormal Q, and hypot(0.21, -0.19) for one whose first two
    columns are scaled by 1.1 and 0.9 (the diagonal of Q^T Q - I; the columns stay orthogonal)."""
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    n, p, ld = 50, 4, 56
    Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((n, p)))
    t = torch.zeros((p, ld), dtype=torch.float64)
    t[:, :n] = torch.as_tensor(Q.T)
    assert bench.orth_feasibility(t, n, torch) < 1e-14
    t[0, :n] *= 1.1
    t[1, :n] *= 0.9
    expect = float(np.hypot(1.1 ** 2 - 1.0, 0.9 ** 2 - 1.0))
    assert abs(bench.orth_feasibility(t, n, torch) - expect) < 1e-13


def test_flop_accounting_matches_table_cost():
    """Table "cost": one PLAM or PCAL iteration is 7np^2 + O(np) flops, namely grad f^T X (2np^2),
    X^T X (np^2), X (X^T X - I) (2np^2) and X Psi(grad f^T X) (2np^2).  The roofline flops of the
    fused kernels add up to it: the Grams X^T [X | G] (3np^2) and the update's two products
    X M and X E (2np^2 each), for every workload the bench runs on the graph engine."""
    sys.path.insert(0, ROOT)
    import bench
    for name, wl in bench.WORKLOADS.items():
        if wl["kind"] == "batched":
            continue
        n, p = wl["n"], wl["p"]
        kf = bench.kernel_flops(wl)
        assert kf["gram_partial"] == 3 * n * p * p and kf["update"] == 4 * n * p * p, name
        assert kf["gram_partial"] + kf["update"] == 7 * n * p * p, name


def test_a_collapsed_solve_is_reported_not_raised(monkeypatch):
    """A solve whose final Cholesky-QR fails (the iterate lost rank in an ABB transient) becomes
    a "failed" record with the last iterate's KKT value and feasibility, so that the benchmark
    still prints its line; a completed solve carries its status and iteration count."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1810_03930_gb300._lib import PlamError

    class FakeSolver:
        def history(self):
            return [(0, 5.0, 1.0, 1e-14, 1.0), (1, 4.0, 0.5, 2.3, 0.5), (2, 3.0, 1e-6, 1023.0, 0.5)]

    def collapse(*a):
        raise PlamError(6, "plam_solve")

    monkeypatch.setattr(bench, "timed_solve_e2e", collapse)
    out = bench.solve_or_report(FakeSolver(), None, None, None, None, None)
    assert out["status"] == "failed" and "plam_solve" in out["error"]
    assert out["iters"] == 2 and out["kkt_rel_last"] == 1e-6
    assert out["feas_last"] == 1023.0 and out["feas_max"] == 1023.0
    json.dumps(out)

    class Info:
        iters = 953

    monkeypatch.setattr(bench, "timed_solve_e2e", lambda *a: (55.6, 56.0, 0, Info()))
    ok = bench.solve_or_report(FakeSolver(), None, None, None, None, None)
    assert ok["status"] == "converged" and ok["iters"] == 953 and ok["time_s"] == 55.6
    assert ok["result"][3].iters == 953
    assert bench.pcal_name(bench.WORKLOADS["stencil3d_128"]) == "PCAL eq.(Lambda1), ABB"

"""Host logic of bench.py on CPU: the time-to-tol figure with a fake solver (one warm-up solve
that is not timed, the median of the timed solves per seed, the median over the seeds, and the
worst status and residual over all of them), the closed-form eigenvalues behind the per-eigenpair
errors, and the scaled oracle sample of the reference arm."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeSolves:
    """solve(seed) -> a result dict; the first call (the warm-up) is an outlier."""

    def __init__(self, ms, iters, status=None, resid=None):
        self.ms, self.iters = ms, iters
        self.status = status or {}
        self.resid = resid or {}
        self.calls = {}
        self.warmed = False
        self.first = min(ms)

    def __call__(self, seed):
        k = self.calls.get(seed, 0)
        self.calls[seed] = k + 1
        warm = not self.warmed
        self.warmed = True
        solve_ms = 1e9 if warm else self.ms[seed][k - 1 if seed == self.first else k]
        return dict(solve_ms=solve_ms, setup_ms=5.0, iters=self.iters[seed], fp64_sweeps=1,
                    status_name=self.status.get(seed, "ok"), max_rel_resid=self.resid.get(seed, 1e-9),
                    lam=[float(seed), float(k)])


def test_medians_over_runs_then_seeds():
    f = FakeSolves(ms={2: [100.0, 300.0, 200.0], 3: [90.0, 95.0, 400.0], 4: [500.0, 510.0, 505.0]},
                   iters={2: 64, 3: 52, 4: 70})
    first, d = bench.time_to_tol_over_seeds(f, [2, 3, 4], 3)
    assert f.calls == {2: 4, 3: 3, 4: 3}                 # one warm-up, then 3 timed per seed
    per = {p["seed"]: p["time_to_tol_s"] for p in d["per_seed"]}
    assert per == pytest.approx({2: 0.2, 3: 0.095, 4: 0.505})
    assert d["time_to_tol_s"] == pytest.approx(0.2)      # median of 0.2, 0.095, 0.505
    assert d["iters"] == 64 and d["iters_per_s"] == pytest.approx(64 / 0.2)
    assert d["seeds"] == [2, 3, 4] and d["runs_per_seed"] == 3 and d["status"] == "ok"
    assert first["lam"] == [2.0, 1.0]                    # the first timed solve of the first seed


def test_worst_status_and_residual():
    f = FakeSolves(ms={s: [10.0, 10.0] for s in (5, 6, 7)}, iters={5: 10, 6: 11, 7: 12},
                   status={6: "not_converged"}, resid={7: 3e-7})
    _, d = bench.time_to_tol_over_seeds(f, [5, 6, 7], 2)
    assert d["status"] == "not_converged"
    assert d["max_rel_resid"] == 3e-7
    assert d["iters"] == 11


def test_single_thread_oracle_sample_runs_in_a_child_process():
    """The reference arm's one-thread oracle figure at the 48^3 workload: a child process with
    every thread-count variable at 1 times one oracle iteration."""
    out = bench.cpu_single_thread_sample("c1", iters=1)
    assert out is not None
    ips, per = out
    assert ips > 0 and per > 0 and abs(ips * per - 1.0) < 1e-9


def test_closed_form_eigenvalues_and_errors():
    """Section 4.1's formula with the h^-2 scale: the smallest eigenvalue of the 464^3 cube is
    3 * 4 * 465^2 * sin^2(pi / 930), the next three are equal (index triples (2,1,1) permuted)."""
    import math
    lam = bench.closed_form_eigenvalues((464, 464, 464), 465.0 ** 2, 8)
    assert lam[0] == pytest.approx(3 * 4 * 465 ** 2 * math.sin(math.pi / 930) ** 2, rel=1e-15)
    assert lam[1] == lam[2] == lam[3] > lam[0]
    assert lam[4] == lam[5] == lam[6] and lam[7] > lam[6]
    errs = bench.rel_errors([x * (1 + 1e-12) for x in lam], (464, 464, 464), 8)
    assert max(errs) == pytest.approx(1e-12, rel=1e-3)
    box = bench.closed_form_eigenvalues((6, 7, 8), 1.0, 3)
    assert box == sorted(box) and len(box) == 3


def test_cpu_sample_scaling():
    key, n_s, factor, text = bench.cpu_sample_desc("c4")
    assert key == "s4" and n_s == 128 ** 3 and factor == pytest.approx(128 ** 3 / 464 ** 3)
    assert "scaled" in text and "m=8" in text
    key, _, factor, _ = bench.cpu_sample_desc("c1")
    assert key == "c1" and factor == 1.0


def test_roofline_bytes_and_traffic_keys():
    """The algorithmic bytes of the two roofline lines, and the source hashes their recorded DRAM
    traffic is keyed to (an edit of the kernel source must drop the recorded traffic)."""
    n, m = 1000, 8
    assert bench.update_bytes_per_launch(n, m) == (3 * m + 2 * m) * 8 * n       # 3m read, 2m written
    assert bench.gram_bytes_per_launch(n, m) == 2 * 3 * m * 8 * n               # [S AS] read once
    h = bench.source_hash("k_tsmm_oz.cu", "oz_digits.cuh")
    assert len(h) == 16 and h == bench.source_hash("k_tsmm_oz.cu", "oz_digits.cuh")
    assert h != bench.source_hash("k_gram_oz.cu", "oz_digits.cuh")
    assert bench.kernel_source_hash() == bench.source_hash("k_gram_oz.cu", "oz_digits.cuh")
    # the recorded traffic is per launch / per iteration of the 464^3 workload, near the algorithmic bytes
    n4 = 464 ** 3
    for (w, key), t in bench.NCU_TRAFFIC_UPDATE.items():
        assert w == "c4" and 0.8 < t / bench.update_bytes_per_launch(n4, 8) < 1.2
    for (w, key), t in bench.NCU_TRAFFIC.items():
        assert w == "c4" and 1.5 < t / bench.gram_bytes_per_launch(n4, 8) < 2.5

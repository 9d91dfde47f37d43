"""Host logic of the time-to-log Z sweep: the cost order of the grid, the selection of the
first cell within tolerance, and the reference taken at the most expensive cell, driven by
a stand-in runner whose log Z spread shrinks with N (no GPU)."""
import math

from paper_2511_15196_gb300 import time_to_logz as ttl


def test_cells_are_in_increasing_cost():
    assert ttl.cells([16384, 8192], [0.9, 0.5]) == [(8192, 0.5, 20), (8192, 0.9, 20), (16384, 0.5, 20),
                                                    (16384, 0.9, 20)]
    # sweeps as an axis: ordered by N x sweeps, then rho, then N
    assert ttl.cells([8192, 16384], [0.5], [20, 40]) == [(8192, 0.5, 20), (8192, 0.5, 40), (16384, 0.5, 20),
                                                         (16384, 0.5, 40)]
    assert ttl.cells([8192, 32768], [0.5], [10, 40]) == [(8192, 0.5, 10), (8192, 0.5, 40), (32768, 0.5, 10),
                                                         (32768, 0.5, 40)]


def test_first_within_needs_both_bias_and_spread():
    rows = [{"logz_mean": -10.2, "logz_sd": 0.01}, {"logz_mean": -10.01, "logz_sd": 0.2},
            {"logz_mean": -10.03, "logz_sd": 0.04}, {"logz_mean": -10.0, "logz_sd": 0.0}]
    assert ttl.first_within(rows, -10.0, 0.05) is rows[2]
    assert ttl.first_within(rows[:2], -10.0, 0.05) is None


def test_measure_with_a_stand_in_runner():
    # log Z bias -200/N and seed spread 400/N around -100: within 0.05 from N = 8192
    def runner(L, N, rho, form, seed, n_mcmc):
        return -100.0 - 200.0 / N + (400.0 / N) * math.sin(seed + 1.0), N * (1.0 + rho)

    out = ttl.measure(8, [1024, 4096, 8192, 16384], [0.5, 0.9], ["mixed"], "fp64", 8, 0.05, 10, runner=runner,
                      emit=lambda s: None)
    r = out["mixed"]
    assert r["cell"] == {"N": 8192, "rho": 0.5, "n_mcmc": 10}
    assert r["time_to_logz_s"] == 8192 * 1.5 * 1e-3
    assert abs(r["logz_ref"] + 100.0) < 0.05


def test_measure_with_sweeps_as_an_axis():
    # a bias of +3/n_mcmc that no N removes: only the 200-sweep cells reach 0.05, and the
    # reference comes from the most expensive cell (N = 4096 with 200 sweeps, rho = 0.9)
    def runner(L, N, rho, form, seed, n_mcmc):
        return -100.0 + 3.0 / n_mcmc + (40.0 / N) * math.sin(seed + 1.0), N * n_mcmc * (1.0 + rho)

    out = ttl.measure(8, [1024, 4096], [0.5, 0.9], ["mixed"], "fp64", 8, 0.05, [10, 200], runner=runner,
                      emit=lambda s: None)
    r = out["mixed"]
    assert r["cell"] == {"N": 1024, "rho": 0.5, "n_mcmc": 200}
    assert abs(r["logz_ref"] - (-100.0 + 3.0 / 200)) < 0.01


def test_free_field_closed_form_matches_the_pinned_values():
    # the module's closed form (the reference of --free) against tests/golden/exact_logz.txt
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "exact_logz.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for kind, L, m2, lam, lz in rows:
        if kind == "free":
            assert abs(ttl.free_field_logz(int(L), float(m2)) - float(lz)) < 1e-9


def test_measure_against_an_exact_value_and_confirm_the_second_form():
    # with a closed form as the reference no reference runs are made; the second form is
    # run only at the first form's cell and the one before it
    calls = []

    def runner(L, N, rho, form, seed, n_mcmc):
        calls.append((form, N))
        return -100.0 + 100.0 / N + (4.0 / N) * math.sin(seed + 1.0), N * (10.0 if form == "fp32" else 1.0)

    out = ttl.measure(8, [256, 1024, 4096], [0.5], ["mixed", "fp32"], "fp64", 4, 0.05, 10, runner=runner,
                      emit=lambda s: None, exact=-100.0, confirm_seeds=2)
    assert out["mixed"]["cell"] == {"N": 4096, "rho": 0.5, "n_mcmc": 10}
    assert out["fp32"]["cell"] == out["mixed"]["cell"] and out["fp32"]["within_tol_at_cell"]
    assert out["fp32"]["time_to_logz_s"] == 4096 * 10.0 * 1e-3
    assert sorted(set(n for f, n in calls if f == "fp32")) == [1024, 4096]


def test_cells_far_from_the_reference_are_given_up_early():
    # a cell whose first seeds sit far outside the tolerance is not run to all its seeds
    calls = []

    def runner(L, N, rho, form, seed, n_mcmc):
        calls.append(N)
        return -100.0 + 200.0 / N + (1.0 / N) * math.sin(seed + 1.0), float(N)

    out = ttl.measure(8, [256, 8192], [0.5], ["mixed"], "fp64", 16, 0.05, 10, runner=runner,
                      emit=lambda s: None, exact=-100.0, early=4)
    assert out["mixed"]["cell"] == {"N": 8192, "rho": 0.5, "n_mcmc": 10}
    assert calls.count(256) == 4 and calls.count(8192) == 16

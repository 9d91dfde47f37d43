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

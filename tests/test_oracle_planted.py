"""Planted mistakes: the oracle's pins must catch plausible errors in the oracle.

Each case below plants one mistake (a dropped term, a wrong sign, index or power, a
transposed operand, an off-by-one search, a missing compensation ...) in a copy of one
oracle module's source, installs the copy in place of the module for the duration of the
case (every oracle and test module that imported the module, or a name from it, sees the
copy), and runs the pins named for it: each of them must fail (an AssertionError; for one case a
run that cannot continue counts too).
The unmodified oracle passes the same pins in ``tests/test_oracle_*.py``.

Everything runs on the CPU; nothing here touches the CUDA path.
"""
import importlib
import inspect
import sys
import types

import numpy as np
import pytest

import oracle
import test_oracle_action as t_action
import test_oracle_covariance as t_cov
import test_oracle_hmc as t_hmc
import test_oracle_irmh as t_irmh
import test_oracle_mutation as t_mut
import test_oracle_ns as t_ns
import test_oracle_observables as t_obs
import test_oracle_philox as t_philox
import test_oracle_resample as t_res
import test_oracle_smc as t_smc
import test_oracle_tempering as t_temp


def _planted_copy(modname, edits, monkeypatch):
    orig = importlib.import_module(modname)
    src = inspect.getsource(orig)
    for old, new in edits:
        assert src.count(old) == 1, f"{modname}: the text to replace must occur once: {old!r}"
        src = src.replace(old, new)
    copy = types.ModuleType(modname)
    copy.__file__ = orig.__file__
    copy.__package__ = "oracle"
    monkeypatch.setitem(sys.modules, modname, copy)
    exec(compile(src, f"<{modname} with a planted mistake>", "exec"), copy.__dict__)
    return orig, copy


def _install(orig, copy, monkeypatch):
    """Rebind the module, and functions or classes imported from it, in every oracle and
    test module, so that the pins and the rest of the oracle call the planted copy."""
    monkeypatch.setattr(oracle, orig.__name__.rsplit(".", 1)[1], copy)
    for mod in list(sys.modules.values()):
        name = getattr(mod, "__name__", "") or ""
        if mod is orig or mod is copy or not (name.startswith("oracle") or name.startswith("test_")):
            continue
        for k, v in list(vars(mod).items()):
            if v is orig:
                monkeypatch.setattr(mod, k, copy)
            elif ((inspect.isfunction(v) or inspect.isclass(v)) and getattr(v, "__module__", None) == orig.__name__
                  and hasattr(copy, v.__name__)):
                monkeypatch.setattr(mod, k, getattr(copy, v.__name__))


def P(fn, **kw):
    return (fn, kw)


# (id, oracle module, [(original text, planted text)], pins that must fail
#  [, exceptions that count as failing, AssertionError alone by default])
CASES = [
    # ---- action, Eq. (1) ----
    ("stencil: second axis replaced by the first", "oracle.lattice",
     [("np.roll(f, 1, axis=-2) + np.roll(f, -1, axis=-2)", "np.roll(f, 1, axis=-1) + np.roll(f, -1, axis=-1)")],
     [P(t_action.test_single_fourier_mode, L=6, k=(1, 2)), P(t_action.test_matches_bond_brute_force, L=3)]),
    ("stencil: neighbour at distance 2", "oracle.lattice",
     [("np.roll(f, -1, axis=-1)", "np.roll(f, -2, axis=-1)")],
     [P(t_action.test_single_fourier_mode, L=8, k=(3, 1)), P(t_action.test_matches_bond_brute_force, L=5)]),
    ("kinetic diagonal 2 instead of 4", "oracle.lattice",
     [("f * (4.0 * f - nb)", "f * (2.0 * f - nb)")],
     [P(t_action.test_single_fourier_mode, L=4, k=(1, 0)), P(t_action.test_matches_bond_brute_force, L=3)]),
    ("quartic term with the wrong power", "oracle.lattice",
     [("lam * f ** 4", "lam * f ** 3")],
     [P(t_action.test_constant_field, L=2), P(t_action.test_matches_bond_brute_force, L=2)]),
    ("mass coefficient dropped", "oracle.lattice",
     [("c_mass * m2 * f * f", "m2 * f * f")],
     [P(t_action.test_constant_field, L=3), P(t_action.test_paper_and_unhalved_forms_map)]),
    ("reference log-normaliser dropped from the incremental weight", "oracle.lattice",
     [("+ 0.5 * np.asarray(sq, dtype=np.float64) + log_gauss_const(D)", "+ 0.5 * np.asarray(sq, dtype=np.float64)")],
     [P(t_action.test_loglik_and_target),
      P(t_smc.test_evidence_matches_exact, kind="one_site", L=1, m2=-4.0, lam=8.0)]),
    # ---- random-walk sweep (App. A) ----
    ("proposal with the transposed factor", "oracle.mutation",
     [("(np.asarray(Z, np.float64) @ np.asarray(Lchol, np.float64).T)",
       "(np.asarray(Z, np.float64) @ np.asarray(Lchol, np.float64))")],
     [P(t_mut.test_proposal_increment_covariance_is_s2_LLT)]),
    ("wrong sign of the action difference in log alpha", "oracle.mutation",
     [("return -beta * dS - (1.0 - beta) * 0.5 * dsq", "return beta * dS - (1.0 - beta) * 0.5 * dsq")],
     [P(t_mut.test_accept_rule_signs), P(t_mut.test_invariance_free_field, keep_reference=False)]),
    ("reference term dropped from log alpha", "oracle.mutation",
     [("return -beta * dS - (1.0 - beta) * 0.5 * dsq", "return -beta * dS")],
     [P(t_mut.test_accept_rule_signs), P(t_mut.test_invariance_free_field, keep_reference=False)]),
    ("accept test reversed", "oracle.mutation",
     [("acc = log_u < log_alpha", "acc = log_u > log_alpha")],
     [P(t_mut.test_accept_rule_signs), P(t_mut.test_invariance_free_field, keep_reference=True)]),
    # ---- tempering (Sec. 2 (i), App. A) ----
    ("ESS without the square of the weight sum", "oracle.tempering",
     [("return w.sum() ** 2 / (w * w).sum()", "return w.sum() / (w * w).sum()")],
     [P(t_temp.test_ess_bounds_and_monotone), P(t_temp.test_ess_equal_weights_is_n_and_single_spike_is_one)]),
    ("bisection returns the upper bracket end", "oracle.tempering",
     [("        return hi, used\n    return lo, used", "        return hi, used\n    return hi, used")],
     [P(t_temp.test_bisection_matches_independent_root_finder)]),
    ("log Z increment without the 1/N of the mean", "oracle.tempering",
     [("math.log(w.sum()) - math.log(len(ell))", "math.log(w.sum())")],
     [P(t_temp.test_reweight_closed_forms), P(t_smc.test_every_stage_of_free_field_path)]),
    ("log Z increment without the max shift", "oracle.tempering",
     [("inc = dbeta * ell.max() + math.log(w.sum())", "inc = math.log(w.sum())")],
     [P(t_temp.test_reweight_closed_forms), P(t_smc.test_every_stage_of_free_field_path)]),
    ("running log Z without compensation", "oracle.tempering",
     [("self.c = (t - self.s) - y", "self.c = 0.0")],
     [P(t_temp.test_kahan_matches_exact_rounded_sum)]),
    # ---- systematic resampling ----
    ("ancestor search takes the first cumulative sum >= p (bisect_left)", "oracle.resample",
     [("bisect.bisect_right(C, p)", "bisect.bisect_left(C, p)")],
     [P(t_res.test_equal_and_degenerate_weights)]),
    ("offset word ignored", "oracle.resample",
     [("p = (((i << 32) + int(U)) * Q) // (n << 32)", "p = ((i << 32) * Q) // (n << 32)")],
     [P(t_res.test_brute_force_tiny, n=8), P(t_res.test_agrees_with_textbook_float_form_away_from_ties)]),
    # ---- covariance and its factor (App. A) ----
    ("covariance divided by N", "oracle.covariance",
     [("return mu, (Xc.T @ Xc) / (n - 1)", "return mu, (Xc.T @ Xc) / n")],
     [P(t_cov.test_sample_covariance_matches_numpy_cov_and_two_point_case)]),
    ("covariance not centred", "oracle.covariance",
     [("Xc = X - mu", "Xc = X")],
     [P(t_cov.test_sample_covariance_matches_numpy_cov_and_two_point_case)]),
    ("ridge level not carried to the next step", "oracle.covariance",
     [("for _ in range(start_level):", "for _ in range(0):")],
     [P(t_cov.test_regularised_cholesky_rank_deficient)]),
    ("Gaussian-part covariance: reference weight 1 - beta when it is kept", "oracle.covariance",
     [("a = 1.0 if keep_reference else 1.0 - beta", "a = 1.0 - beta")],
     [P(t_cov.test_gaussian_part_covariance_inverts_the_hessian_of_the_tempered_target, L=4, beta=0.7,
        keep=True)]),
    ("Gaussian-part covariance: the factor 2 of the quadratic form dropped", "oracle.covariance",
     [("P = a * np.eye(D) + 2.0 * beta * (c_kin * K + c_mass * m2 * np.eye(D))",
       "P = a * np.eye(D) + beta * (c_kin * K + c_mass * m2 * np.eye(D))")],
     [P(t_cov.test_gaussian_part_covariance_inverts_the_hessian_of_the_tempered_target, L=3, beta=1.0,
        keep=False), P(t_cov.test_gaussian_part_covariance_spectrum_is_the_closed_form)]),
    ("Gaussian-part covariance: one neighbour direction only", "oracle.covariance",
     [("for rr, cc in (((r + 1) % L, c), ((r - 1) % L, c), (r, (c + 1) % L), (r, (c - 1) % L)):",
       "for rr, cc in (((r + 1) % L, c), ((r - 1) % L, c)):")],
     [P(t_cov.test_gaussian_part_covariance_inverts_the_hessian_of_the_tempered_target, L=4, beta=0.7,
        keep=True), P(t_cov.test_gaussian_part_covariance_spectrum_is_the_closed_form)]),
    # ---- SMC driver ----
    ("resampling skipped after reweighting", "oracle.smc",
     [("self.phi, self.S, self.sq = self.phi[anc], self.S[anc], self.sq[anc]", "pass")],
     [P(t_smc.test_every_stage_of_free_field_path)]),
    ("incremental weights not refreshed after the sweeps", "oracle.smc",
     [("        self.ell = lattice.tempering_loglik(self.S, self.sq, c.D, c.keep_reference)\n        self.beta = beta_new",
       "        self.beta = beta_new")],
     [P(t_smc.test_every_stage_of_free_field_path)]),
    # ---- observables (Sec. 2, App. F) ----
    ("susceptibility with <|M|> in place of <M>", "oracle.observables",
     [('"chi": D * (mean_M2 - mean_M ** 2)', '"chi": D * (mean_M2 - mean_absM ** 2)')],
     [P(t_obs.test_weighted_moments_by_hand), P(t_obs.test_free_field_moments_from_exact_draws)]),
    ("weights not normalised", "oracle.observables",
     [("w = w / w.sum()", "w = w")],
     [P(t_obs.test_weighted_moments_by_hand), P(t_obs.test_free_field_moments_from_exact_draws)]),
    ("mode balance counts zeros as positive", "oracle.observables",
     [("pos = float(w[M > 0].sum())", "pos = float(w[M >= 0].sum())")],
     [P(t_obs.test_mode_balance_edge_cases)]),
    # ---- Philox4x32-10 ----
    ("Philox key schedule with one Weyl constant swapped", "oracle.philox",
     [("k1 = np.uint64((int(k1) + PHILOX_W1) & MASK32)", "k1 = np.uint64((int(k1) + PHILOX_W0) & MASK32)")],
     [P(t_philox.test_known_answer_vectors)]),
    ("Philox round with the product halves exchanged", "oracle.philox",
     [("c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0",
       "c0, c1, c2, c3 = (lo1 ^ c1 ^ k0), hi1, (hi0 ^ c3 ^ k1), lo0")],
     [P(t_philox.test_known_answer_vectors)]),
    # ---- HMC transition (sampler (iii)) ----
    ("gradient with the wrong sign of the mass term", "oracle.hmc",
     [("+ 2.0 * c_mass * m2 * f", "- 2.0 * c_mass * m2 * f")],
     [P(t_hmc.test_gradient_matches_finite_differences, L=3, c=(1.0, 1.0))]),
    ("gradient of the kinetic term halved", "oracle.hmc",
     [("c_kin * (8.0 * f - 2.0 * nb)", "c_kin * (4.0 * f - nb)")],
     [P(t_hmc.test_gradient_matches_finite_differences, L=4, c=(0.5, 0.5))]),
    ("last leapfrog momentum step a full step", "oracle.hmc",
     [("(eps if i + 1 < n else 0.5 * eps)", "eps")],
     [P(t_hmc.test_leapfrog_is_reversible_and_second_order)]),
    ("kinetic energy with 1/v", "oracle.hmc",
     [("kin0 = 0.5 * (v[None, :] * p0 * p0)", "kin0 = 0.5 * (p0 * p0 / v[None, :])"),
      ("kin1 = 0.5 * (v[None, :] * p1 * p1)", "kin1 = 0.5 * (p1 * p1 / v[None, :])")],
     [P(t_hmc.test_invariance_free_field, keep_reference=False)]),
    ("momenta scaled by sqrt(v) instead of 1/sqrt(v)", "oracle.hmc",
     [("p0 = Z / np.sqrt(v)[None, :]", "p0 = Z * np.sqrt(v)[None, :]")],
     [P(t_hmc.test_invariance_free_field, keep_reference=False)]),
    # (a wrong force leaves the transition exact -- the leapfrog map stays reversible and
    # volume-preserving and the accept test uses the true energy -- so only a pin on the
    # force itself can see it)
    ("reference term dropped from the target's gradient", "oracle.hmc",
     [("- a * np.asarray(phi, np.float64)", "")],
     [P(t_hmc.test_target_gradient_matches_finite_differences, keep_reference=False),
      P(t_hmc.test_target_gradient_matches_finite_differences, keep_reference=True)]),
    # ---- independence sweep (sampler (ii)) ----
    ("Hastings term dropped", "oracle.irmh",
     [("+ 0.5 * (zz - r)", "")],
     [P(t_irmh.test_log_alpha_is_the_metropolis_hastings_ratio, keep_reference=False),
      P(t_irmh.test_invariance_free_field, keep_reference=False)]),
    ("Hastings term reversed", "oracle.irmh",
     [("+ 0.5 * (zz - r)", "+ 0.5 * (r - zz)")],
     [P(t_irmh.test_log_alpha_is_the_metropolis_hastings_ratio, keep_reference=True),
      P(t_irmh.test_invariance_free_field, keep_reference=True)]),
    ("whitened norm not updated on acceptance", "oracle.irmh",
     [("np.where(acc, zz, r), acc, log_alpha", "r, acc, log_alpha")],
     [P(t_irmh.test_invariance_free_field, keep_reference=False)]),
    # ---- nested sampling (sampler (iv)) ----
    ("prior slice bracket for E instead of 2E", "oracle.ns",
     [("disc = math.sqrt(b * b + 2.0 * E * a)", "disc = math.sqrt(b * b + E * a)")],
     [P(t_ns.test_prior_bracket_roots)]),
    ("prior volume shrinks by 1/N per removal within a batch", "oracle.ns",
     [("shrink = 1.0 / (N - j + 1)", "shrink = 1.0 / N")],
     [P(t_ns.test_one_site_evidence_and_error_bar)]),
    ("slice bracket shrunk on the wrong side", "oracle.ns",
     [("            if t < 0.0:\n                t_lo = t\n            else:\n                t_hi = t",
       "            if t < 0.0:\n                t_hi = t\n            else:\n                t_lo = t")],
     [P(t_ns.test_one_site_evidence_and_error_bar)],
     # the live points collapse onto a few and the run stops at a singular covariance
     (AssertionError, np.linalg.LinAlgError)),
    ("deletion threshold at the lowest deleted point", "oracle.ns",
     [("lstar = float(self.logl[dead[-1]])", "lstar = float(self.logl[dead[0]])")],
     [P(t_ns.test_one_site_evidence_and_error_bar)]),
    ("replacement started from any point, deleted ones included", "oracle.ns",
     [("start = int(survivors[int(math.floor(u * (N - k)))])", "start = int(order[int(math.floor(u * N))])")],
     [P(t_ns.test_one_site_evidence_and_error_bar)]),
    ("live points weighted X instead of X / N", "oracle.ns",
     [("logw_live = self.logX - math.log(c.N)", "logw_live = self.logX")],
     [P(t_ns.test_evidence_with_the_live_points_at_any_stopping_point)]),
    ("stopping rule reversed", "oracle.ns",
     [("- self.logZ < math.log(c.stop_frac)", "- self.logZ > math.log(c.stop_frac)")],
     [P(t_ns.test_information_and_stopping_rule)]),
    ("information without the -log Z", "oracle.ns",
     [("H = float((p * all_l).sum()) - logZ", "H = float((p * all_l).sum())")],
     [P(t_ns.test_information_and_stopping_rule)]),
    # ---- more of the same modules ----
    ("Box-Muller with the cosine twice", "oracle.philox",
     [("    ang = 2.0 * np.pi * u2\n    return r * np.cos(ang), r * np.sin(ang)\n\n\ndef box_muller_24",
       "    ang = 2.0 * np.pi * u2\n    return r * np.cos(ang), r * np.cos(ang)\n\n\ndef box_muller_24")],
     [P(t_philox.test_box_muller_special_points), P(t_philox.test_normals_moments)]),
    ("Box-Muller radius uniform without the +1 (u1 may be 0)", "oracle.philox",
     [("u1 = (wa.astype(np.float64) + 1.0) * 2.0 ** -32", "u1 = wa.astype(np.float64) * 2.0 ** -32")],
     [P(t_philox.test_box_muller_special_points)]),
    ("independence proposal without the population mean", "oracle.irmh",
     [("prop = np.asarray(mu, np.float64)[None, :] + Z @ np.asarray(Lchol, np.float64).T",
       "prop = Z @ np.asarray(Lchol, np.float64).T")],
     [P(t_irmh.test_log_alpha_is_the_metropolis_hastings_ratio, keep_reference=False)]),
    ("leapfrog drift without the inverse mass", "oracle.hmc",
     [("phi = phi + eps * v * p", "phi = phi + eps * p")],
     [P(t_hmc.test_leapfrog_is_reversible_and_second_order), P(t_hmc.test_invariance_free_field, keep_reference=False)]),
    ("ridge without the 1/D of the mean diagonal", "oracle.covariance",
     [("delta = jitter_rel * np.trace(Sigma) / D", "delta = jitter_rel * np.trace(Sigma)")],
     [P(t_cov.test_regularised_cholesky_rank_deficient)]),
    ("<|M|> without the absolute value", "oracle.observables",
     [("mean_absM = float((w * np.abs(M)).sum())", "mean_absM = float((w * M).sum())")],
     [P(t_obs.test_weighted_moments_by_hand), P(t_obs.test_free_field_moments_from_exact_draws)]),
    ("magnetisation as the sum over sites", "oracle.lattice",
     [("return phi.mean(axis=-1)", "return phi.sum(axis=-1)")],
     [P(t_obs.test_weighted_moments_by_hand), P(t_obs.test_free_field_moments_from_exact_draws)]),
    ("paper-mode weight keeps the reference term", "oracle.lattice",
     [("        return -np.asarray(S, dtype=np.float64)\n",
       "        return -np.asarray(S, dtype=np.float64) + 0.5 * np.asarray(sq, dtype=np.float64)\n")],
     [P(t_action.test_loglik_and_target), P(t_smc.test_paper_mode_free_field)]),
    ("bisection halves the wrong side", "oracle.tempering",
     [("            lo = mid\n        else:\n            hi = mid", "            hi = mid\n        else:\n            lo = mid")],
     [P(t_temp.test_bisection_matches_independent_root_finder), P(t_temp.test_bisection_brute_force_grid_tiny)]),
    ("ESS target rho (N - 1)", "oracle.tempering",
     [("target = rho * n\n", "target = rho * (n - 1)\n")],
     [P(t_temp.test_bisection_matches_independent_root_finder)]),
    ("sweeps at the previous temperature", "oracle.smc",
     [("self.phi, self.S, self.sq, Lc, c.scale, beta_new,", "self.phi, self.S, self.sq, Lc, c.scale, self.beta,")],
     [P(t_smc.test_every_stage_of_free_field_path),
      P(t_smc.test_evidence_matches_exact, kind="free", L=2, m2=1.0, lam=0.0)]),
    ("paper-mode accept ignores the kept reference", "oracle.mutation",
     [("        return -beta * dS - 0.5 * dsq\n", "        return -beta * dS - (1.0 - beta) * 0.5 * dsq\n")],
     [P(t_mut.test_invariance_free_field, keep_reference=True)]),
    ("HMC accept with the kinetic difference's sign flipped", "oracle.hmc",
     [("- (kin1 - kin0)", "+ (kin1 - kin0)")],
     [P(t_hmc.test_small_steps_are_accepted), P(t_hmc.test_invariance_free_field, keep_reference=False)]),
    ("whitened norm with the upper triangle", "oracle.irmh",
     [("X, lower=True)", "X, lower=False)")],
     [P(t_irmh.test_whitened_norm_is_the_mahalanobis_distance)]),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_its_pins(case, monkeypatch):
    _, modname, edits, pins = case[:4]
    fails = case[4] if len(case) > 4 else AssertionError
    orig, copy = _planted_copy(modname, edits, monkeypatch)
    _install(orig, copy, monkeypatch)
    for fn, kw in pins:
        with pytest.raises(fails):
            fn(**kw)

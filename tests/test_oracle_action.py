"""Pins for the oracle's lattice action (Eq. (1)) against closed forms, a
brute-force bond sum and the kappa-form identity of App. G."""
import math

import numpy as np
import pytest

import inputs
from oracle import lattice


def bond_form(phi, L, m2, lam, c_kin, c_mass):
    """Brute force: loop over sites and over the two forward bonds of each,
    S = sum_x [ c_kin * sum_mu (phi_{x+mu} - phi_x)^2 + c_mass m2 phi_x^2 + lam phi_x^4 ]."""
    S = 0.0
    for r in range(L):
        for c in range(L):
            f = phi[r * L + c]
            right = phi[r * L + (c + 1) % L]
            down = phi[((r + 1) % L) * L + c]
            S += c_kin * ((right - f) ** 2 + (down - f) ** 2) + c_mass * m2 * f * f + lam * f ** 4
    return S


@pytest.mark.parametrize("L", [1, 2, 3, 4, 7])
def test_constant_field(L):
    for c in (0.0, 0.37, -1.25):
        phi = np.full((1, L * L), c)
        for (m2, lam, ck, cm) in ((-4.0, 8.0, 1.0, 1.0), (1.0, 0.0, 0.5, 0.5), (2.5, 3.0, 0.7, 1.3)):
            want = L * L * (cm * m2 * c * c + lam * c ** 4)
            assert lattice.action(phi, L, m2, lam, ck, cm)[0] == pytest.approx(want, rel=1e-14, abs=1e-14)


@pytest.mark.parametrize("L,k", [(4, (1, 0)), (6, (1, 2)), (8, (3, 1)), (5, (2, 2))])
def test_single_fourier_mode(L, k):
    r, c = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    phi = np.cos(2 * math.pi * (k[0] * r + k[1] * c) / L).ravel()[None, :]
    kin = lattice.kinetic_site_terms(phi, L).sum()
    want = (4 * math.sin(math.pi * k[0] / L) ** 2 + 4 * math.sin(math.pi * k[1] / L) ** 2) * (phi ** 2).sum()
    assert kin == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("L", [1, 2, 3, 5])
def test_matches_bond_brute_force(L):
    phi = inputs.fields(6, L * L, seed=L)
    for (m2, lam, ck, cm) in ((-4.0, 8.0, 1.0, 1.0), (-4.0, 1.0, 0.5, 0.5), (0.3, 0.1, 1.7, 0.2)):
        got = lattice.action(phi, L, m2, lam, ck, cm)
        want = [bond_form(p, L, m2, lam, ck, cm) for p in phi]
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_kappa_form_identity():
    # App. G: kappa/2 sum (phi_{x+mu}-phi_x)^2 + sum[phi^2 + lam (phi^2-1)^2]
    #        = -kappa sum phi_x phi_{x+mu} + (kappa d + 1 - 2 lam) sum phi^2 + lam sum phi^4 + V lam   (d = 2)
    L, kappa, lam = 5, 0.31, 0.7
    phi = inputs.fields(3, L * L, seed=9)
    for p in phi:
        f = p.reshape(L, L)
        hop = (f * np.roll(f, -1, 0)).sum() + (f * np.roll(f, -1, 1)).sum()
        expanded = -kappa * hop + (kappa * 2 + 1 - 2 * lam) * (f * f).sum() + lam * (f ** 4).sum() + L * L * lam
        kappa_form = 0.5 * kappa * (((np.roll(f, -1, 0) - f) ** 2).sum() + ((np.roll(f, -1, 1) - f) ** 2).sum()) \
            + (f * f + lam * (f * f - 1) ** 2).sum()
        assert kappa_form == pytest.approx(expanded, rel=1e-12)
        # the oracle's coefficient form with c_kin = kappa/2, c_mass m2 = 1 - 2 lam reproduces it up to V lam
        ours = lattice.action(p[None, :], L, 1 - 2 * lam, lam, c_kin=0.5 * kappa, c_mass=1.0)[0]
        assert ours + L * L * lam == pytest.approx(kappa_form, rel=1e-12)


def test_paper_and_unhalved_forms_map():
    # S_unhalved(psi / sqrt 2; m2, lam) = S_Eq1(psi; m2, lam / 4)
    L = 4
    psi = inputs.fields(4, L * L, seed=3)
    a = lattice.action(psi / math.sqrt(2), L, -4.0, 8.0, 1.0, 1.0)
    b = lattice.action(psi, L, -4.0, 2.0, 0.5, 0.5)
    np.testing.assert_allclose(a, b, rtol=1e-13)


def test_loglik_and_target():
    D = 9
    S = np.array([1.5, -2.0])
    sq = np.array([3.0, 0.5])
    ell = lattice.tempering_loglik(S, sq, D)
    np.testing.assert_allclose(ell, -S + 0.5 * sq + 0.5 * D * math.log(2 * math.pi))
    np.testing.assert_allclose(lattice.tempering_loglik(S, sq, D, keep_reference=True), -S)
    # log gamma_beta interpolates: beta = 0 is the reference log density up to a constant, beta = 1 is -S
    np.testing.assert_allclose(lattice.log_target(S, sq, 0.0), -0.5 * sq)
    np.testing.assert_allclose(lattice.log_target(S, sq, 1.0), -S)


def test_kappa_form_maps_onto_the_action_coefficients():
    # App. G: (kappa/2) sum_{x,mu} (phi_{x+mu} - phi_x)^2 + sum_x [phi_x^2 + lam (phi_x^2 - 1)^2]
    # equals the library form with c_kin = kappa/2, c_mass = 1, m2 = 1 - 2 lam, plus lam V
    g = np.random.default_rng(9)
    L, kappa, lam = 5, 0.37, 1.3
    phi = g.standard_normal((6, L * L))
    f = phi.reshape(6, L, L)
    kin = sum(((np.roll(f, -1, axis=a) - f) ** 2).sum(axis=(1, 2)) for a in (1, 2))
    s_kappa = 0.5 * kappa * kin + (f ** 2 + lam * (f ** 2 - 1.0) ** 2).sum(axis=(1, 2))
    s_lib = lattice.action(phi, L, 1.0 - 2.0 * lam, lam, 0.5 * kappa, 1.0)
    np.testing.assert_allclose(s_lib + lam * L * L, s_kappa, rtol=1e-13)

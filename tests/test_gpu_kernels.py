"""Per-kernel parity of the CUDA path (through the C ABI) with the FP64 oracle on
identical seeded inputs. Tolerances:
  * FP64 kernels: relative 1e-12 (action), rounding-order bounds elsewhere;
  * FP32 kernels: action of the float fields to 1e-12 of the summed site terms' magnitude
    (exact float products, compensated sums, double combination); GEMMs within the worst-case float
    dot-product bound gamma_K = K u / (1 - K u), u = 2^-24, on sum |a||b|;
  * bf16 tensor-core GEMMs: operand rounding 2 u_b + u_b^2 (u_b = 2^-8) plus gamma_K,
    both on sum |a||b|, plus the fp16 rounding u_h = 2^-11 of the stored increment;
  * mixed covariance (exact Gram of fixed-point digits): the rounding of each centred
    field to its site's grid, propagated through Xc^T Xc, plus one FP64 rounding;
  * integer and index results (resampling, gather): bit-exact.
"""
import math

import numpy as np
import pytest

import inputs
from oracle import covariance as ocov
from oracle import lattice as olat
from oracle import mutation as omut
from oracle import philox as oph
from oracle import resample as ores
from oracle import tempering as otemp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2511_15196_gb300 as p  # noqa: E402

U32 = 2.0 ** -24
UB = 2.0 ** -8
UH = 2.0 ** -11  # fp16 unit roundoff (the mixed proposal stores its increment in fp16)


def cuda(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gamma(k, u=U32):
    return k * u / (1 - k * u)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    p.lib()


# ------------------------------------------------------------------ Philox normals

@pytest.mark.parametrize("n_rows,n_cols,row0", [(3, 1, 0), (17, 7, 5), (64, 64, 0), (300, 257, 11), (2, 4096, 100)])
def test_normals_fp64(n_rows, n_cols, row0):
    out = torch.empty((n_rows, n_cols + 3), dtype=torch.float64, device="cuda")[:, :n_cols]
    p.philox_normals(out, 1234, 5, p.RNG_PROPOSE, 9, 2, row0=row0)
    ref = oph.normals(1234, 5, oph.KIND_PROPOSE, 9, 2, n_rows, n_cols, bits=32, row0=row0)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dtype", ["f32", "bf16_normals"])
def test_normals_single(dtype):
    tdt = torch.float32 if dtype == "f32" else torch.bfloat16
    out = torch.empty((513, 130), dtype=tdt, device="cuda")
    p.philox_normals(out, 99, 0, p.RNG_INIT, 0, 0)
    ref = oph.normals(99, 0, oph.KIND_INIT, 0, 0, 513, 130, bits=24)
    got = out.float().cpu().numpy().astype(np.float64)
    if dtype == "f32":
        # float log / sqrt / sincospi of exact 24-bit uniforms: a few float ulps of |z| <= 6
        np.testing.assert_allclose(got, ref, rtol=4 * U32, atol=8 * U32 * 6)
    else:
        np.testing.assert_allclose(got, ref, rtol=UB * 1.01, atol=8 * U32 * 6)


# ------------------------------------------------------------------ action

@pytest.mark.parametrize("L", [1, 2, 3, 8, 12, 31, 33, 64])
@pytest.mark.parametrize("coef", [(-4.0, 8.0, 1.0, 1.0), (-4.0, 1.0, 0.5, 0.5), (1.0, 0.0, 1.0, 1.0)])
def test_action_fp64(L, coef):
    m2, lam, ck, cm = coef
    N = 37
    phi = inputs.broken_phase_fields(N, L * L, seed=L)
    S, sq = p.action(cuda(phi), L, m2, lam, ck, cm)
    Sr = olat.action(phi, L, m2, lam, ck, cm)
    np.testing.assert_allclose(S.cpu().numpy(), Sr, rtol=1e-12, atol=1e-12 * np.abs(Sr).max())
    np.testing.assert_allclose(sq.cpu().numpy(), olat.sq_norm(phi), rtol=1e-12)


@pytest.mark.parametrize("L", [2, 8, 16, 32, 64])
def test_action_fp32(L):
    N = 200
    phi = inputs.broken_phase_fields(N, L * L, seed=100 + L).astype(np.float32)
    S, sq = p.action(cuda(phi), L, -4.0, 8.0)
    f = phi.astype(np.float64)
    Sr = olat.action(f, L, -4.0, 8.0)
    # relative to the magnitude of the summed site terms (the condition of the sum):
    # near-cancelling actions of small lattices make |S| itself a meaningless scale
    site = olat.kinetic_site_terms(f, L).reshape(N, -1) - 4.0 * f * f + 8.0 * f ** 4
    scale = np.maximum(np.abs(Sr), np.abs(site).sum(axis=1))
    rel = np.abs(S.cpu().numpy() - Sr) / scale
    assert rel.max() <= 1e-12, rel.max()
    np.testing.assert_allclose(sq.cpu().numpy(), olat.sq_norm(phi.astype(np.float64)), rtol=1e-12)


# ------------------------------------------------------------------ ESS bisection + reweighting

@pytest.mark.parametrize("N", [1, 2, 7, 1000, 1024, 8192, 50000])
@pytest.mark.parametrize("beta,rho", [(0.0, 0.5), (0.3, 0.9), (0.97, 0.5)])
def test_bisection_and_reweight(N, beta, rho):
    ell = inputs.log_weights(N, seed=N, spread=20.0, offset=-500.0)
    w, out = p.ess_bisect(cuda(ell), beta, rho, 64)
    out = out.cpu().numpy()
    d_ref, used = otemp.bisect_dbeta(ell, beta, rho, 64)
    w_ref, inc_ref = otemp.reweight(ell, d_ref)
    assert out[0] == pytest.approx(d_ref, rel=1e-12, abs=1e-300)
    b_ref = 1.0 if d_ref >= 1.0 - beta else beta + d_ref
    assert out[1] == pytest.approx(b_ref, rel=1e-12)
    assert out[2] == pytest.approx(w_ref.sum() ** 2 / (w_ref ** 2).sum(), rel=1e-11)
    assert out[3] == pytest.approx(inc_ref, rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(w.cpu().numpy(), w_ref, rtol=1e-11, atol=1e-300)
    assert abs(out[4] - used) <= 2


@pytest.mark.parametrize("N", [1000, 5000])
@pytest.mark.parametrize("rho", [0.99, 0.999])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_bisection_high_ess_targets(N, rho, beta):
    # the target-ESS sweep of App. E (Table 4: 0.9, 0.99, 0.999): at high targets dbeta is a
    # small fraction of the bracket, so a sum rounded in another order may flip one late
    # halving; then both answers must be roots to rounding, ESS(d) = rho N within 1e-11
    ell = inputs.log_weights(N, seed=N + 7, spread=30.0, offset=-800.0)
    w, out = p.ess_bisect(cuda(ell), beta, rho, 64)
    out = out.cpu().numpy()
    d_ref, used = otemp.bisect_dbeta(ell, beta, rho, 64)
    w_ref, inc_ref = otemp.reweight(ell, d_ref)

    def ess(d):
        a = ell - ell.max()
        e = np.exp(d * a)
        return e.sum() ** 2 / (e * e).sum()
    if out[0] != pytest.approx(d_ref, rel=1e-12):
        assert ess(out[0]) == pytest.approx(rho * N, rel=1e-11)
        assert ess(d_ref) == pytest.approx(rho * N, rel=1e-11)
        assert out[0] == pytest.approx(d_ref, rel=1e-6)
    else:
        np.testing.assert_allclose(w.cpu().numpy(), w_ref, rtol=1e-11, atol=1e-300)
        assert out[3] == pytest.approx(inc_ref, rel=1e-12, abs=1e-12)
    assert 0.0 < out[0] < 1.0 - beta
    assert out[2] >= rho * N * (1 - 1e-12)


def test_bisection_steps_to_one():
    ell = inputs.log_weights(4096, seed=3, spread=1e-4)
    _, out = p.ess_bisect(cuda(ell), 0.6, 0.5)
    out = out.cpu().numpy()
    assert out[0] == 0.4 and out[1] == 1.0 and out[4] == 0


# ------------------------------------------------------------------ resampling and gather

@pytest.mark.parametrize("N", [1, 2, 3, 17, 1000, 1024, 8192, 65537])
@pytest.mark.parametrize("kind", ["plain", "zeros", "heavy"])
def test_resample_bit_exact(N, kind):
    w = inputs.positive_weights(N, seed=N + len(kind), zeros=(N // 3 if kind == "zeros" else 0),
                                heavy=(kind == "heavy"))
    for U in (0, inputs.word32(N), 2 ** 32 - 1):
        anc = p.resample_systematic(cuda(w), U).cpu().numpy()
        ref = ores.systematic(w, U)
        np.testing.assert_array_equal(anc, ref)


def test_gather_rows_exact():
    g = inputs.rng(4)
    for (N, D, dt) in ((1000, 64, torch.float64), (513, 4096, torch.float32), (77, 9, torch.float32)):
        src = torch.as_tensor(g.standard_normal((N, D))).to(dt).cuda()
        anc = np.sort(g.integers(0, N, N)).astype(np.int32)
        dst = p.gather_rows(src, cuda(anc))
        assert torch.equal(dst, src[torch.as_tensor(anc, dtype=torch.long).cuda()])


# ------------------------------------------------------------------ covariance

def _cov_bound_terms(X):
    Xc = X - X.mean(0)
    A = np.abs(Xc).T @ np.abs(Xc) / (X.shape[0] - 1)
    return Xc, A


def _digit_bits(N):
    """Fixed-point width B of the mixed covariance: every sum of N digit products stays
    within 2^23 (exact in the fp32 accumulators), at most two 7-bit digits."""
    return min(14, 23 - int(math.ceil(math.log2(N))))


def _mixed_cov_bound(X):
    """|Sigma_gpu - Sigma| for the mixed covariance: each centred field moves by at most
    E_nj = g_j (the grid step 2^(e_j - B) of its site, a full step so that an exponent
    one larger on the device is covered) + float centring and mean errors; through
    Xc^T Xc / (N - 1) that is (|Xc|^T E + E^T |Xc| + E^T E) / (N - 1), plus one FP64
    rounding of the result."""
    N = X.shape[0]
    B = _digit_bits(N)
    mu = X.mean(0)
    Xc = X - mu
    dev = np.abs(Xc).max(0)
    e = np.frexp(dev)[1]
    g = np.ldexp(1.0, e - B)
    E = g[None, :] + 2.0 ** -20 * (np.abs(X) + np.abs(X).mean(0)[None, :])
    A = np.abs(Xc)
    M = (A.T @ E + E.T @ A + E.T @ E) / (N - 1)
    _, ref = ocov.sample_covariance(X)
    return M * 1.0001 + 2.0 ** -50 * np.abs(ref) + 1e-300


@pytest.mark.parametrize("N,L", [(1000, 12), (257, 24), (4096, 32), (300, 3)])
@pytest.mark.parametrize("precision", [p.FP64, p.FP32, p.MIXED_BF16], ids=["fp64", "fp32", "bf16"])
def test_covariance(N, L, precision):
    D = L * L
    X = inputs.broken_phase_fields(N, D, seed=N + D)
    if precision != p.FP64:
        X = X.astype(np.float32).astype(np.float64)
    sig = p.covariance(cuda(X, torch.float64 if precision == p.FP64 else torch.float32), precision).cpu().numpy()
    _, ref = ocov.sample_covariance(X)
    _, A = _cov_bound_terms(X)
    low = np.tril_indices(D)
    err = np.abs(sig - ref)[low]
    if precision == p.FP64:
        bound = 1e-12 * A[low] + 1e-300
    elif precision == p.FP32:
        bound = (2 * U32 + gamma(N)) * A[low] * 1.0001 + 1e-30
    else:
        bound = _mixed_cov_bound(X)[low]
    assert (err <= bound).all(), (err / bound).max()
    # the strictly upper triangle is untouched
    assert (sig[np.triu_indices(D, 1)] == 0).all()


@pytest.mark.parametrize("N,L", [(300, 32), (8192, 8), (2, 4)])
def test_mixed_covariance_is_psd(N, L):
    """The mixed covariance is the Gram matrix of the rounded fields: positive
    semi-definite up to FP64 rounding, also when N <= D makes it singular (with bf16
    operands and fp32 sums over N its null space would come out indefinite)."""
    D = L * L
    X = inputs.broken_phase_fields(N, D, seed=7 + N).astype(np.float32)
    sig = p.covariance(cuda(X), p.MIXED_BF16).cpu().numpy()
    S = np.tril(sig) + np.tril(sig, -1).T
    w = np.linalg.eigvalsh(S)
    assert w[0] >= -1e-13 * max(w[-1], 1e-300) * D, (w[0], w[-1])


def test_mixed_covariance_exact_at_the_digit_bound():
    """Fields whose digits reach the bound (|h| = 2^(B-a), |l| = 2^(a-1)) on N = 8192
    particles, so that the digit-product sums reach 2^23: the device result equals the
    exact Gram matrix of the rounded fields over N - 1, bit for bit."""
    N, L = 8192, 8
    D = L * L
    B = _digit_bits(N)
    a = (B + 1) // 2
    assert (B, a) == (10, 5)
    g = np.random.default_rng(11)
    # per site one magnitude: 1 - 2^-11 rounds half-way up to v = 2^B (h = 32, l = 0);
    # 1008/1024 gives v = 1008 (h = 32, l = -16); 0.5 + 2^-11 rounds half-way down to 512
    mags = np.array([1.0 - 2.0 ** -11, 1008.0 / 1024.0, 0.5 + 2.0 ** -11])[np.arange(D) % 3]
    signs = np.ones((N, D))
    for j in range(D):  # exactly N/2 negative entries per site: the mean is exactly zero
        signs[g.permutation(N)[: N // 2], j] = -1.0
    X = (signs * mags[None, :]).astype(np.float32)
    assert (X.astype(np.float64).sum(0) == 0).all()
    sig = p.covariance(cuda(X), p.MIXED_BF16).cpu().numpy()
    e = np.frexp(np.abs(X.astype(np.float64)).max(0))[1]
    s = B - e
    v = np.rint(np.ldexp(X.astype(np.float64), s[None, :])).astype(np.int64)
    assert np.abs(v).max() == 2 ** B
    G = v.T @ v  # exact integer Gram
    want = np.ldexp(G.astype(np.float64), -(s[:, None] + s[None, :])) * (1.0 / (N - 1))
    low = np.tril_indices(D)
    np.testing.assert_array_equal(sig[low], want[low])


# ------------------------------------------------------------------ Cholesky

@pytest.mark.parametrize("mode", [1, 2], ids=["simt", "tc_emulated"])
@pytest.mark.parametrize("D", [1, 5, 63, 64, 65, 130, 257, 1024])
def test_cholesky_fp64(D, mode):
    A = inputs.spd_matrix(D, seed=D, cond=1e3)
    ridge = 1e-3
    a = cuda(A)
    a, st = p.cholesky(a, ridge, mode=mode)
    assert int(st.cpu()[0]) == 0
    Lg = a.cpu().numpy()
    ref = np.linalg.cholesky(A + ridge * np.eye(D))
    np.testing.assert_allclose(Lg, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    assert (np.triu(Lg, 1) == 0).all()


@pytest.mark.parametrize("mode", [1, 2], ids=["simt", "tc_emulated"])
@pytest.mark.parametrize("D", [1, 5, 9, 144, 400])
def test_cholesky_writes_nothing_past_the_matrix(D, mode):
    """Last diagonal blocks narrower than a warp (D mod 64 < 32): the factorisation
    writes only the D x D matrix (a guard band after it keeps its sentinel)."""
    A = inputs.spd_matrix(D, seed=D + 1, cond=1e3)
    guard = 8192
    buf = torch.full((D * D + guard,), -7.25, dtype=torch.float64, device="cuda")
    buf[: D * D] = torch.as_tensor(A.ravel(), device="cuda")
    a = buf[: D * D].view(D, D)
    a, st = p.cholesky(a, 1e-3, mode=mode)
    assert int(st.cpu()[0]) == 0
    assert (buf[D * D:] == -7.25).all()
    ref = np.linalg.cholesky(A + 1e-3 * np.eye(D))
    np.testing.assert_allclose(a.cpu().numpy(), ref, rtol=0, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("D", [384, 2048, 4096])
def test_cholesky_tensor_update_matches_fp64(D):
    # the exact-digit tensor-core trailing update against the FP64 SIMT update and LAPACK
    g = inputs.rng(D)
    X = g.standard_normal((D + 64, D)) * np.exp(g.uniform(-3, 3, D))[None, :]   # columns of mixed scale
    A = X.T @ X / (D + 63)
    ridge = 1e-6 * np.trace(A) / D
    a1, s1 = p.cholesky(cuda(A), ridge, mode=1)
    a2, s2 = p.cholesky(cuda(A), ridge, mode=2)
    assert int(s1.cpu()[0]) == 0 and int(s2.cpu()[0]) == 0
    L1, L2 = a1.cpu().numpy(), a2.cpu().numpy()
    ref = np.linalg.cholesky(A + ridge * np.eye(D))
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert (np.abs(L2 - ref) <= 1e-10 * scale).all(), (np.abs(L2 - ref) / scale).max()
    assert (np.abs(L2 - L1) <= 1e-10 * scale).all(), (np.abs(L2 - L1) / scale).max()
    # backward error of the emulated factor at FP64 level
    R = L2 @ L2.T - (A + ridge * np.eye(D))
    assert np.abs(R).max() <= 1e-13 * np.abs(A).max() * D ** 0.5


@pytest.mark.parametrize("D", [1, 63, 64, 130, 1024])
def test_cholesky_fp32(D):
    A = inputs.spd_matrix(D, seed=D + 7, cond=1e2)
    ridge = 1e-3
    Lg, st = p.cholesky_f32(cuda(A), ridge)
    assert int(st.cpu()[0]) == 0
    Lg = Lg.cpu().numpy().astype(np.float64)
    ref = np.linalg.cholesky(A.astype(np.float32).astype(np.float64) + ridge * np.eye(D))
    # backward-stable float Cholesky: |L - L_ref| bounded by a modest multiple of D u kappa-free scale
    np.testing.assert_allclose(Lg, ref, rtol=0, atol=64 * D ** 0.5 * U32 * 1e2 * np.abs(ref).max())
    assert (np.triu(Lg, 1) == 0).all()


def test_cholesky_flags_indefinite():
    D = 100
    A = inputs.spd_matrix(D, seed=1)
    A[70, 70] = -1.0
    for mode in (1, 2):
        _, st = p.cholesky(cuda(A), 0.0, mode=mode)
        assert int(st.cpu()[0]) & 2


# ------------------------------------------------------------------ proposal GEMM

def _propose_ref(phi, Lc, scale, N, D, bits, step, sweep, seed=11, sid=3):
    Z = oph.normals(seed, sid, oph.KIND_PROPOSE, step, sweep, N, D, bits=bits)
    return omut.propose(phi, Z, Lc, scale), Z


@pytest.mark.parametrize("N,L", [(300, 12), (1000, 8), (257, 32), (130, 10)])
def test_propose_fp64(N, L):
    D = L * L
    phi = inputs.broken_phase_fields(N, D, seed=5)
    Lc = inputs.lower_factor(D, seed=D)
    s = 2.38 / L
    got = p.rw_propose(cuda(phi), cuda(Lc), p.FP64, s, 11, 3, 4, 2).cpu().numpy()
    ref, Z = _propose_ref(phi, Lc, s, N, D, 32, 4, 2)
    bound = s * (gamma(D, 2.0 ** -53) * 4 * (np.abs(Z) @ np.abs(Lc).T) + 1e-13 * (np.ones_like(Z) @ np.abs(Lc).T)) \
        + 4 * 2.0 ** -53 * np.abs(ref)
    assert (np.abs(got - ref) <= bound).all()


@pytest.mark.parametrize("N,L", [(300, 12), (1000, 8), (257, 32), (130, 10)])
@pytest.mark.parametrize("precision", [p.FP32, p.MIXED_BF16], ids=["fp32", "bf16"])
def test_propose_single(N, L, precision):
    D = L * L
    phi = inputs.broken_phase_fields(N, D, seed=6).astype(np.float32)
    Lc = inputs.lower_factor(D, seed=D + 1)
    s = 2.38 / L
    if precision == p.FP32:
        Lt = cuda(Lc, torch.float32)
        Lr = Lt.double().cpu().numpy()
        op_err = 0.0
    else:
        ld = (D + 7) // 8 * 8
        Lt = torch.zeros((D, ld), dtype=torch.bfloat16, device="cuda")
        Lt[:, :D] = cuda(Lc, torch.bfloat16)
        Lt = Lt  # row pitch ld (multiple of 8)
        Lr = Lc
        op_err = 2 * UB + UB * UB + UH * (1 + 2 * UB)
    got = p.rw_propose(cuda(phi), Lt, precision, s, 11, 3, 4, 2).cpu().numpy().astype(np.float64)
    ref, Z = _propose_ref(phi.astype(np.float64), Lr, s, N, D, 24, 4, 2)
    absprod = np.abs(Z) @ np.abs(Lr).T
    bound = s * ((op_err + gamma(D)) * absprod + 8 * U32 * 6 * (np.ones_like(Z) @ np.abs(Lr).T)) \
        + 2 * U32 * (np.abs(ref) + np.abs(phi))
    err = np.abs(got - ref)
    assert (err <= bound).all(), (err / bound).max()


def test_propose_bf16_full_size_sampled_rows():
    # the timed workload's shape: N = 8192 particles, D = 4096 sites (L = 64)
    N, L = 8192, 64
    D = L * L
    g = inputs.rng(8)
    phi = (0.5 * g.standard_normal((N, D))).astype(np.float32)
    Lc = np.tril(0.02 * g.standard_normal((D, D)))
    Lc[np.diag_indices(D)] = 0.3 + 0.1 * g.random(D)
    Lt = cuda(Lc, torch.bfloat16)
    s = 2.38 / L
    got = p.rw_propose(cuda(phi), Lt, p.MIXED_BF16, s, 21, 0, 1, 0)
    rows = np.concatenate([g.choice(N, 48, replace=False), [0, N - 1]])
    got = got[torch.as_tensor(rows).cuda()].cpu().numpy().astype(np.float64)
    Z = np.stack([oph.normals(21, 0, oph.KIND_PROPOSE, 1, 0, 1, D, bits=24, row0=int(r))[0] for r in rows])
    ref = phi[rows].astype(np.float64) + s * (Z @ Lc.T)
    absprod = np.abs(Z) @ np.abs(Lc).T
    bound = s * ((2 * UB + UB * UB + UH * (1 + 2 * UB) + gamma(D)) * absprod
                 + 8 * U32 * 6 * np.abs(Lc).sum(1)[None, :]) \
        + 2 * U32 * (np.abs(ref) + np.abs(phi[rows]))
    err = np.abs(got - ref)
    assert (err <= bound).all(), (err / bound).max()


# ------------------------------------------------------------------ accept

@pytest.mark.parametrize("L,N", [(8, 1024), (33, 50), (2, 64)])
@pytest.mark.parametrize("keep_reference", [False, True])
def test_accept_fp64(L, N, keep_reference):
    D = L * L
    phi = inputs.broken_phase_fields(N, D, seed=L)
    prop = phi + 0.05 * inputs.fields(N, D, seed=L + 1)
    m2, lam, beta = -4.0, 8.0, 0.37
    S = olat.action(phi, L, m2, lam)
    sq = olat.sq_norm(phi)
    ell = olat.tempering_loglik(S, sq, D, keep_reference)
    tphi, tS, tsq, tell = cuda(phi), cuda(S), cuda(sq), cuda(ell)
    cnt = p.rw_accept(tphi, cuda(prop), L, m2, lam, tS, tsq, tell, beta, 17, 0, 3, 1,
                      keep_reference=keep_reference).cpu().numpy()
    u = oph.uniform53(17, 0, oph.KIND_ACCEPT, 3, 1, np.arange(N))
    rphi, rS, rsq, acc, _, _, la = omut.accept(phi, S, sq, prop, np.log(u), beta, L, m2, lam, 1.0, 1.0,
                                                keep_reference)
    near = np.abs(np.log(u) - la) < 1e-9
    gphi = tphi.cpu().numpy()
    gacc = np.all(gphi == prop, axis=1)
    assert (gacc[~near] == acc[~near]).all()
    assert cnt[0] == gacc.sum() and cnt[1] == 0
    np.testing.assert_allclose(gphi[~near], rphi[~near], rtol=0, atol=0)
    np.testing.assert_allclose(tS.cpu().numpy()[~near], rS[~near], rtol=1e-12)
    np.testing.assert_allclose(tsq.cpu().numpy()[~near], rsq[~near], rtol=1e-12)
    rell = olat.tempering_loglik(rS, rsq, D, keep_reference)
    np.testing.assert_allclose(tell.cpu().numpy()[~near], rell[~near], rtol=1e-12)


@pytest.mark.parametrize("L,N", [(64, 300), (32, 1000), (8, 777), (12, 64)])
def test_accept_delta_matches_oracle(L, N):
    # mixed-form accept: proposal = phi + fp16 increment, formed in float while loading
    D = L * L
    phi = inputs.broken_phase_fields(N, D, seed=L + 40).astype(np.float32)
    delta = (0.02 * inputs.fields(N, D, seed=L + 41)).astype(np.float16)
    prop = (phi + delta.astype(np.float32)).astype(np.float32)  # the float sum the kernel forms
    m2, lam, beta = -4.0, 8.0, 0.6
    phi64, prop64 = phi.astype(np.float64), prop.astype(np.float64)
    S = olat.action(phi64, L, m2, lam)
    sq = olat.sq_norm(phi64)
    ell = olat.tempering_loglik(S, sq, D)
    tphi, tS, tsq, tell = cuda(phi), cuda(S), cuda(sq), cuda(ell)
    cnt = p.rw_accept_delta(tphi, torch.as_tensor(delta).cuda(), L, m2, lam, tS, tsq, tell, beta, 9, 1, 5, 3)
    u = oph.uniform53(9, 1, oph.KIND_ACCEPT, 5, 3, np.arange(N))
    _, _, _, acc, S2, sq2, la = omut.accept(phi64, S, sq, prop64, np.log(u), beta, L, m2, lam, 1.0, 1.0)
    # S' of the float proposal is exact to about 2^-48 of its site terms: the decision can
    # differ only within the FP64 test's band
    near = np.abs(np.log(u) - la) < 1e-9
    gphi = tphi.cpu().numpy()
    gacc = np.all(gphi == prop, axis=1)
    assert (gacc[~near] == acc[~near]).all()
    assert (gacc | np.all(gphi == phi, axis=1)).all()
    assert int(cnt.cpu()[0]) == gacc.sum()
    ok = gacc & ~near
    site = olat.kinetic_site_terms(prop64, L).reshape(N, -1) + m2 * prop64 ** 2 + lam * prop64 ** 4
    scale = np.abs(site).sum(axis=1)
    assert (np.abs(tS.cpu().numpy() - S2)[ok] <= 1e-12 * scale[ok]).all()
    np.testing.assert_allclose(tsq.cpu().numpy()[ok], sq2[ok], rtol=1e-12)


def test_accept_fp32_decisions():
    L, N = 32, 2000
    D = L * L
    phi = inputs.broken_phase_fields(N, D, seed=2).astype(np.float32)
    prop = (phi + 0.02 * inputs.fields(N, D, seed=3)).astype(np.float32)
    m2, lam, beta = -4.0, 8.0, 0.8
    phi64, prop64 = phi.astype(np.float64), prop.astype(np.float64)
    S = olat.action(phi64, L, m2, lam)
    sq = olat.sq_norm(phi64)
    ell = olat.tempering_loglik(S, sq, D)
    tphi = cuda(phi)
    tS, tsq, tell = cuda(S), cuda(sq), cuda(ell)
    p.rw_accept(tphi, cuda(prop), L, m2, lam, tS, tsq, tell, beta, 5, 0, 2, 0)
    u = oph.uniform53(5, 0, oph.KIND_ACCEPT, 2, 0, np.arange(N))
    _, _, _, acc, S2, _, la = omut.accept(phi64, S, sq, prop64, np.log(u), beta, L, m2, lam, 1.0, 1.0)
    # the float action of the proposal is exact to about 2^-48 of its site terms: decisions can
    # only differ inside the FP64 test's band
    band = 1e-9
    near = np.abs(np.log(u) - la) < band
    gacc = np.all(tphi.cpu().numpy() == prop, axis=1)
    assert (gacc[~near] == acc[~near]).all()
    assert 0.05 < acc.mean() < 0.95


def test_kappa_config_action_on_the_gpu():
    # the kappa form of App. G through kappa_config's coefficients, on the action kernel
    g = np.random.default_rng(10)
    L, kappa, lam = 8, 0.27, 0.8
    phi = g.standard_normal((33, L * L))
    cfg = p.kappa_config(kappa, lam, L=L, N=33)
    S, _ = p.action(cuda(phi), L, cfg.m2, cfg.lam, cfg.c_kin, cfg.c_mass)
    f = phi.reshape(33, L, L)
    kin = sum(((np.roll(f, -1, axis=a) - f) ** 2).sum(axis=(1, 2)) for a in (1, 2))
    s_kappa = 0.5 * kappa * kin + (f ** 2 + lam * (f ** 2 - 1.0) ** 2).sum(axis=(1, 2))
    np.testing.assert_allclose(S.cpu().numpy() - p.kappa_logz_shift(lam, L * L), s_kappa, rtol=1e-12)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("weighted", [False, True], ids=["uniform", "weighted"])
@pytest.mark.parametrize("L,N", [(8, 700), (5, 1), (16, 3001), (64, 8192)])
def test_observables_reduction_matches_oracle(dtype, weighted, L, N):
    # a12 on the device: M per field, then the weighted FP64 moments, chi and the mode
    # balance in one CTA, against the oracle's summary of the same fields and weights
    from oracle import observables as oobs
    D = L * L
    phi = inputs.broken_phase_fields(N, D, seed=N + L).astype(np.float32 if dtype == torch.float32 else np.float64)
    w = inputs.positive_weights(N, seed=N, zeros=min(3, N - 1)) if weighted else None
    M, out = p.observables(torch.from_numpy(phi).cuda(), L, None if w is None else torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    ref = oobs.summary(phi.astype(np.float64), w)
    Mref = phi.astype(np.float64).mean(axis=1)
    assert np.abs(M.cpu().numpy() - Mref).max() <= 1e-13 * max(1.0, np.abs(Mref).max())
    o = out.cpu().numpy()
    for i, k in enumerate(("mean_M", "mean_absM", "mean_M2", "chi")):
        assert o[i] == pytest.approx(ref[k], rel=1e-11, abs=1e-14), k
    if math.isinf(ref["mode_balance"]):
        assert math.isinf(o[4]) and o[4] > 0
    else:
        assert o[4] == pytest.approx(ref["mode_balance"], rel=1e-12)
    assert o[5] == pytest.approx(N if w is None else w.sum(), rel=1e-13)


def test_observables_mode_balance_edge_cases():
    # App. F's edge cases: zeros ignored, +inf with nothing negative, NaN with neither side
    from oracle import observables as oobs
    L, D = 4, 16
    rows = np.array([1.0, 0.0, 2.0, 0.0])
    phi = np.repeat(rows[:, None], D, axis=1)
    _, out = p.observables(torch.from_numpy(phi).cuda(), L)
    o = out.cpu().numpy()
    assert math.isinf(o[4]) and o[4] > 0 and math.isinf(oobs.mode_balance(rows))
    _, out = p.observables(torch.zeros((5, D), dtype=torch.float64, device="cuda"), L)
    assert math.isnan(out.cpu().numpy()[4]) and math.isnan(oobs.mode_balance(np.zeros(5)))
    phi = np.repeat(np.array([-1.0, 0.0, 3.0, -2.0])[:, None], D, axis=1)
    w = np.array([0.5, 1.0, 0.25, 0.25])
    _, out = p.observables(torch.from_numpy(phi).cuda(), L, torch.from_numpy(w).cuda())
    assert out.cpu().numpy()[4] == pytest.approx(0.25 / 0.75, rel=1e-15)


@pytest.mark.parametrize("L,beta,keep", [(1, 0.3, False), (2, 0.5, False), (3, 1.0, False), (8, 0.25, True),
                                         (16, 0.9, False), (32, 1.0, False), (20, 0.0, False)])
def test_free_field_covariance_matches_oracle(L, beta, keep):
    # the device builds Sigma from the Fourier spectrum of P per site displacement; the oracle
    # inverts P assembled site by site from the action's kinetic sum
    m2, c_kin, c_mass = 1.0, 0.8, 1.2
    sig = p.free_field_covariance(L, beta, m2, c_kin, c_mass, keep).cpu().numpy()
    ref = ocov.gaussian_part_covariance(L, beta, m2, c_kin, c_mass, keep)
    assert np.abs(sig - ref).max() <= 1e-12 * np.abs(ref).max()

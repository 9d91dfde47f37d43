"""Every kernel-level entry point writes only its own outputs: each output (and each
scratch buffer) is followed by a guard band holding a sentinel, and after the call the
band must be intact. Sizes are ragged on purpose: single particles, lattices whose D is
below a warp or not a multiple of the kernels' tiles, N not a multiple of any block."""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2511_15196_gb300 as p  # noqa: E402
from paper_2511_15196_gb300 import _ptr, _stream, lib  # noqa: E402

GUARD = 4096
SENTINEL = {torch.float64: -7.25, torch.float32: -7.25, torch.float16: -7.25, torch.bfloat16: -7.25,
            torch.int32: -123456789, torch.uint8: 0xA5}


def guarded(n, dtype, init=None):
    """(buffer, view of its first n elements); the rest of the buffer holds the sentinel."""
    buf = torch.full((n + GUARD,), SENTINEL[dtype], dtype=dtype, device="cuda")
    view = buf[:n]
    if init is not None:
        view.copy_(torch.as_tensor(np.ascontiguousarray(init).ravel()).to(dtype))
    return buf, view


def intact(buf, n):
    torch.cuda.synchronize()
    return bool((buf[n:] == SENTINEL[buf.dtype]).all())


def check(st):
    assert st == 0, lib().phi4_last_error()


SIZES = [(1, 1), (3, 3), (257, 5), (33, 12), (130, 20)]


@pytest.mark.parametrize("N,L", SIZES)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_action_bounds(N, L, dtype):
    D = L * L
    phi = torch.as_tensor(inputs.broken_phase_fields(N, D, seed=N + L)).to(dtype).cuda()
    bS, S = guarded(N, torch.float64)
    bq, sq = guarded(N, torch.float64)
    dt = p.DT_F64 if dtype == torch.float64 else p.DT_F32
    check(lib().phi4_action(_ptr(phi), dt, N, L, -4.0, 8.0, 1.0, 1.0, _ptr(S), _ptr(sq), _stream()))
    assert intact(bS, N) and intact(bq, N)


@pytest.mark.parametrize("rows,cols", [(1, 1), (3, 7), (65, 130), (5, 4097)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16], ids=["f64", "f32", "bf16"])
def test_normals_bounds(rows, cols, dtype):
    dt = {torch.float64: p.DT_F64, torch.float32: p.DT_F32, torch.bfloat16: p.DT_BF16}[dtype]
    b, out = guarded(rows * cols, dtype)
    check(lib().phi4_philox_normals(7, 1, p.RNG_PROPOSE, 3, 2, 0, rows, cols, cols, dt, _ptr(out), _stream()))
    assert intact(b, rows * cols)


@pytest.mark.parametrize("N", [1, 2, 257, 1000])
def test_bisect_resample_gather_bounds(N):
    ell = torch.as_tensor(inputs.log_weights(N, seed=N)).cuda()
    bw, w = guarded(N, torch.float64)
    bo, out = guarded(8, torch.float64, np.zeros(8))
    beta = torch.tensor([0.25], dtype=torch.float64, device="cuda")
    nb = lib().phi4_bisect_scratch_bytes(N)
    bs, scratch = guarded(nb, torch.uint8)
    check(lib().phi4_ess_bisect(_ptr(ell), N, _ptr(beta), 0.5, 64, _ptr(w), _ptr(out), _ptr(scratch), nb, _stream()))
    assert intact(bw, N) and intact(bo, 8) and intact(bs, nb)

    wpos = torch.as_tensor(inputs.positive_weights(N, seed=N + 1)).cuda()
    ba, anc = guarded(N, torch.int32)
    nb = lib().phi4_resample_scratch_bytes(N)
    bs, scratch = guarded(nb, torch.uint8)
    check(lib().phi4_resample_systematic(_ptr(wpos), N, 12345, _ptr(anc), _ptr(scratch), nb, _stream()))
    assert intact(ba, N) and intact(bs, nb)
    ba2, anc2 = guarded(N, torch.int32)
    check(lib().phi4_resample_systematic_static(_ptr(wpos), N, 12345, _ptr(anc2), _stream()))
    assert intact(ba2, N)

    for D in (1, 3, 65):
        src = torch.randn(N, D, dtype=torch.float32, device="cuda")
        bd, dst = guarded(N * D, torch.float32)
        check(lib().phi4_gather_rows(_ptr(src), _ptr(dst), D * 4, N, _ptr(anc), _stream()))
        assert intact(bd, N * D)


@pytest.mark.parametrize("N,L", [(2, 1), (3, 3), (257, 5), (300, 12), (130, 20)])
@pytest.mark.parametrize("precision", [p.FP64, p.FP32, p.MIXED_BF16], ids=["fp64", "fp32", "bf16"])
def test_covariance_bounds(N, L, precision):
    D = L * L
    X = inputs.broken_phase_fields(N, D, seed=3 + N)
    phi = torch.as_tensor(X).to(torch.float64 if precision == p.FP64 else torch.float32).cuda()
    bsg, sigma = guarded(D * D, torch.float64, np.zeros(D * D))
    nb = lib().phi4_covariance_scratch_bytes(N, D, precision)
    bs, scratch = guarded(nb, torch.uint8)
    check(lib().phi4_covariance(_ptr(phi), precision, N, D, _ptr(sigma), _ptr(scratch), nb, _stream()))
    assert intact(bsg, D * D) and intact(bs, nb)


@pytest.mark.parametrize("D", [1, 5, 9, 144, 400])
def test_cholesky_f32_bounds(D):
    A = inputs.spd_matrix(D, seed=D + 2, cond=1e3)
    sig = torch.as_tensor(A).cuda()
    ba, a = guarded(D * D, torch.float32)
    r = torch.tensor([1e-3], dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    nb = lib().phi4_cholesky_scratch_bytes(D)
    bs, scratch = guarded(nb, torch.uint8)
    check(lib().phi4_cholesky_f32(_ptr(sig), _ptr(a), D, _ptr(r), _ptr(st), _ptr(scratch), nb, _stream()))
    assert int(st.cpu()[0]) == 0
    assert intact(ba, D * D) and intact(bs, nb)


@pytest.mark.parametrize("N,L", [(1, 1), (3, 3), (257, 5), (130, 12), (33, 20)])
@pytest.mark.parametrize("precision", [p.FP64, p.FP32, p.MIXED_BF16], ids=["fp64", "fp32", "bf16"])
def test_propose_accept_bounds(N, L, precision):
    D = L * L
    X = inputs.broken_phase_fields(N, D, seed=9 + N)
    Lc = inputs.lower_factor(D, seed=D + 3)
    ft = torch.float64 if precision == p.FP64 else torch.float32
    phi = torch.as_tensor(X).to(ft).cuda()
    if precision == p.MIXED_BF16:
        ldl = (D + 7) // 8 * 8
        Lt = torch.zeros((D, ldl), dtype=torch.bfloat16, device="cuda")
        Lt[:, :D] = torch.as_tensor(Lc).to(torch.bfloat16)
    else:
        ldl = D
        Lt = torch.as_tensor(Lc).to(ft).cuda()
    bp, prop = guarded(N * D, ft)
    nb = lib().phi4_propose_scratch_bytes(N, D, precision)
    bs, scratch = guarded(nb, torch.uint8)
    s = 2.38 / L
    check(lib().phi4_rw_propose(_ptr(phi), _ptr(prop), _ptr(Lt), ldl, precision, N, D, s, 11, 3, 4, 2,
                                _ptr(scratch), nb, _stream()))
    assert intact(bp, N * D) and intact(bs, nb)

    # accept in place on guarded copies of phi and the per-particle caches
    bphi, phi_g = guarded(N * D, ft, X)
    S, sq = p.action(phi_g.view(N, D), L, -4.0, 8.0)
    ell = -S + 0.5 * sq
    bS, S_g = guarded(N, torch.float64, S.cpu().numpy())
    bq, sq_g = guarded(N, torch.float64, sq.cpu().numpy())
    be, ell_g = guarded(N, torch.float64, ell.cpu().numpy())
    b = torch.tensor([0.3], dtype=torch.float64, device="cuda")
    bc, cnt = guarded(2, torch.int32, np.zeros(2))
    dt = p.DT_F64 if precision == p.FP64 else p.DT_F32
    check(lib().phi4_rw_accept(_ptr(phi_g), _ptr(prop), dt, N, L, -4.0, 8.0, 1.0, 1.0, 0, _ptr(S_g), _ptr(sq_g),
                               _ptr(ell_g), _ptr(b), 9, 1, 5, 3, _ptr(cnt), _stream()))
    assert intact(bphi, N * D) and intact(bS, N) and intact(bq, N) and intact(be, N) and intact(bc, 2)


@pytest.mark.parametrize("N,L", [(1, 4), (33, 12), (257, 20), (130, 8)])
def test_accept_delta_bounds(N, L):
    D = L * L
    X = inputs.broken_phase_fields(N, D, seed=21 + N).astype(np.float32)
    delta = torch.as_tensor(0.01 * inputs.rng(N).standard_normal((N, D))).to(torch.float16).cuda()
    bphi, phi_g = guarded(N * D, torch.float32, X)
    S, sq = p.action(phi_g.view(N, D), L, -4.0, 8.0)
    bS, S_g = guarded(N, torch.float64, S.cpu().numpy())
    bq, sq_g = guarded(N, torch.float64, sq.cpu().numpy())
    be, ell_g = guarded(N, torch.float64, (-S + 0.5 * sq).cpu().numpy())
    b = torch.tensor([0.3], dtype=torch.float64, device="cuda")
    bc, cnt = guarded(2, torch.int32, np.zeros(2))
    check(lib().phi4_rw_accept_delta(_ptr(phi_g), _ptr(delta), N, L, -4.0, 8.0, 1.0, 1.0, 0, _ptr(S_g), _ptr(sq_g),
                                     _ptr(ell_g), _ptr(b), 9, 1, 5, 3, _ptr(cnt), _stream()))
    assert intact(bphi, N * D) and intact(bS, N) and intact(bq, N) and intact(be, N) and intact(bc, 2)

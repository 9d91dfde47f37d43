"""Python binding of libphi4smc (include/phi4smc.h): GB300 particle Monte Carlo
for lattice phi^4 theory (arXiv 2511.15196, Sec. 2 samplers (i) and (iv)).

Argument marshalling only: every step of the sampler runs in the CUDA kernels of
the shared library. PyTorch provides device memory (the workspace tensors) and
streams. Importing this module does not need a GPU; the library is loaded on
first use and the call fails loudly if it has not been built.
"""
import ctypes
import dataclasses
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphi4smc.so")

PHI4_OK, PHI4_ERR_ARG, PHI4_ERR_CUDA, PHI4_ERR_NOT_PD, PHI4_ERR_NONFINITE, PHI4_ERR_DONE, PHI4_ERR_WORKSPACE, \
    PHI4_ERR_TIMEOUT, PHI4_ERR_UNSUPPORTED = range(9)
SMC_RW, NS_SLICE, SMC_IRMH, SMC_HMC = 0, 1, 2, 3
FP64, FP32, MIXED_BF16 = 0, 1, 2
DT_F64, DT_F32, DT_BF16 = 0, 1, 2
RNG_INIT, RNG_RESAMPLE, RNG_PROPOSE, RNG_ACCEPT, RNG_NS_START, RNG_NS_DIRECTION, RNG_NS_SLICE, RNG_FLIP = range(1, 9)
FLAG_Z2_FLIP = 1
FLAG_FREE_KERNEL_COV = 2
N_STAGES = 14

_STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NOT_PD", 4: "ERR_NONFINITE", 5: "ERR_DONE",
                 6: "ERR_WORKSPACE", 7: "ERR_TIMEOUT", 8: "ERR_UNSUPPORTED"}


class Phi4Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, status), msg))
        self.status = status


class CConfig(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("N", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("m2", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("c_kin", ctypes.c_double), ("c_mass", ctypes.c_double), ("keep_reference", ctypes.c_int32),
                ("n_mcmc", ctypes.c_int32), ("ess_target", ctypes.c_double), ("rw_scale", ctypes.c_double),
                ("ns_n_delete", ctypes.c_int32), ("ns_slice_steps", ctypes.c_int32),
                ("ns_stop_frac", ctypes.c_double), ("chol_jitter_rel", ctypes.c_double),
                ("bisect_iters", ctypes.c_int32), ("slice_max_shrink", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint64), ("chol_mode", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class CObs(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("logz", ctypes.c_double), ("logz_err", ctypes.c_double),
                ("mean_M", ctypes.c_double), ("mean_absM", ctypes.c_double), ("mean_M2", ctypes.c_double),
                ("chi", ctypes.c_double), ("mode_balance", ctypes.c_double), ("ess", ctypes.c_double),
                ("acc_rate", ctypes.c_double), ("n_steps", ctypes.c_int64), ("n_likelihood_evals", ctypes.c_int64),
                ("slice_capped", ctypes.c_int64)]


@dataclasses.dataclass
class Config:
    """Mirror of phi4_config with the library's defaults."""
    L: int
    N: int
    m2: float = -4.0
    lam: float = 8.0
    kind: int = SMC_RW
    precision: int = FP64
    c_kin: float = 1.0
    c_mass: float = 1.0
    keep_reference: bool = False
    n_mcmc: int = 10
    ess_target: float = 0.5
    rw_scale: float = 0.0
    ns_n_delete: int = 1
    ns_slice_steps: int = 0
    ns_stop_frac: float = 1e-3
    chol_jitter_rel: float = 1e-8
    bisect_iters: int = 64
    slice_max_shrink: int = 64
    seed: int = 0
    stream_id: int = 0
    chol_mode: int = 0
    flags: int = 0  # FLAG_Z2_FLIP: global phi -> -phi move after each temperature's sweeps;
    # FLAG_FREE_KERNEL_COV: exact Gaussian-part covariance in place of the population's

    def to_c(self):
        return CConfig(self.L, self.N, self.kind, self.precision, self.m2, self.lam, self.c_kin, self.c_mass,
                       int(bool(self.keep_reference)), self.n_mcmc, self.ess_target, self.rw_scale,
                       self.ns_n_delete, self.ns_slice_steps, self.ns_stop_frac, self.chol_jitter_rel,
                       self.bisect_iters, self.slice_max_shrink, self.seed, self.stream_id, self.chol_mode,
                       self.flags)


_lib = None
_P = ctypes.c_void_p
_I32, _U32, _U64, _F64, _SZ = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
_SIGS = {
    "phi4_last_error": ([], ctypes.c_char_p),
    "phi4_device_sm_count": ([ctypes.POINTER(_I32)], _I32),
    "phi4_set_spin_limit": ([ctypes.c_int64], _I32),
    "phi4_workspace_bytes": ([ctypes.POINTER(CConfig), ctypes.POINTER(_SZ)], _I32),
    "smc_init": ([ctypes.POINTER(CConfig), _P, _SZ, _P, ctypes.POINTER(_P)], _I32),
    "smc_temper_step": ([_P, ctypes.POINTER(_F64)], _I32),
    "ns_replace_step": ([_P, ctypes.POINTER(_I32)], _I32),
    "smc_log_evidence": ([_P, ctypes.POINTER(_F64), ctypes.POINTER(_F64)], _I32),
    "smc_observables": ([_P, ctypes.POINTER(CObs)], _I32),
    "smc_copy_particles": ([_P, _P, _SZ], _I32),
    "smc_load_particles": ([_P, _P, _SZ], _I32),
    "smc_free": ([_P], _I32),
    "phi4_state_bytes": ([_P, ctypes.POINTER(_SZ)], _I32),
    "smc_save_state": ([_P, _P, _SZ], _I32),
    "smc_restore_state": ([_P, _P, _SZ], _I32),
    "phi4_batch_workspace_bytes": ([_P, _I32, ctypes.POINTER(_SZ)], _I32),
    "smc_init_batch": ([_P, _I32, _P, _SZ, _P, ctypes.POINTER(_P)], _I32),
    "smc_temper_step_batch": ([_P, ctypes.POINTER(_I32)], _I32),
    "phi4_batch_member": ([_P, _I32, ctypes.POINTER(_P)], _I32),
    "phi4_batch_tuning": ([_P, ctypes.c_char_p, _SZ], _I32),
    "phi4_kernel_launches": ([_P, ctypes.POINTER(ctypes.c_int64)], _I32),
    "phi4_set_stage_timing": ([_P, _I32], _I32),
    "phi4_stage_times": ([_P, ctypes.POINTER(_F64), ctypes.POINTER(ctypes.c_int64), _I32], _I32),
    "phi4_stage_name": ([_I32], ctypes.c_char_p),
    "phi4_philox_normals": ([_U64, _U64, _I32, _U32, _U32, _I32, _I32, _I32, _I32, _I32, _P, _P], _I32),
    "phi4_action": ([_P, _I32, _I32, _I32, _F64, _F64, _F64, _F64, _P, _P, _P], _I32),
    "phi4_bisect_scratch_bytes": ([_I32], _SZ),
    "phi4_ess_bisect": ([_P, _I32, _P, _F64, _I32, _P, _P, _P, _SZ, _P], _I32),
    "phi4_resample_scratch_bytes": ([_I32], _SZ),
    "phi4_resample_systematic": ([_P, _I32, _U32, _P, _P, _SZ, _P], _I32),
    "phi4_resample_systematic_static": ([_P, _I32, _U32, _P, _P], _I32),
    "phi4_gather_rows": ([_P, _P, _SZ, _I32, _P, _P], _I32),
    "phi4_observables": ([_P, _I32, _I32, _I32, _P, _P, _P, _P], _I32),
    "phi4_free_covariance_scratch_bytes": ([_I32], _SZ),
    "phi4_free_field_covariance": ([_I32, _P, _F64, _F64, _F64, _I32, _P, _P, _SZ, _P], _I32),
    "phi4_covariance_scratch_bytes": ([_I32, _I32, _I32], _SZ),
    "phi4_covariance": ([_P, _I32, _I32, _I32, _P, _P, _SZ, _P], _I32),
    "phi4_cholesky_scratch_bytes": ([_I32], _SZ),
    "phi4_cholesky": ([_P, _I32, _P, _P, _P, _SZ, _I32, _P], _I32),
    "phi4_cholesky_f32": ([_P, _P, _I32, _P, _P, _P, _SZ, _P], _I32),
    "phi4_propose_scratch_bytes": ([_I32, _I32, _I32], _SZ),
    "phi4_rw_propose": ([_P, _P, _P, _I32, _I32, _I32, _I32, _F64, _U64, _U64, _U32, _U32, _P, _SZ, _P], _I32),
    "phi4_rw_accept": ([_P, _P, _I32, _I32, _I32, _F64, _F64, _F64, _F64, _I32, _P, _P, _P, _P, _U64, _U64, _U32,
                        _U32, _P, _P], _I32),
    "phi4_rw_accept_delta": ([_P, _P, _I32, _I32, _F64, _F64, _F64, _F64, _I32, _P, _P, _P, _P, _U64, _U64, _U32,
                              _U32, _P, _P], _I32),
}


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libphi4smc.so not built: run `python -c 'import __graft_entry__ as g; g.build()'` "
                               "or `python paper_2511_15196_gb300/build.py`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status):
    if status != PHI4_OK:
        raise Phi4Error(status, lib().phi4_last_error().decode())
    return status


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def workspace_bytes(cfg: Config):
    n = _SZ()
    c = cfg.to_c()
    _check(lib().phi4_workspace_bytes(ctypes.byref(c), ctypes.byref(n)))
    return n.value


class Run:
    """An SMC or nested-sampling run whose state lives in a torch uint8 CUDA tensor."""

    def __init__(self, cfg: Config, device="cuda", stream=None):
        import torch
        self.cfg = cfg
        self._c = cfg.to_c()
        nbytes = workspace_bytes(cfg)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self._stream = stream
        h = _P()
        _check(lib().smc_init(ctypes.byref(self._c), ctypes.c_void_p(self._ws_ptr), nbytes, _stream(stream),
                              ctypes.byref(h)))
        self.handle = h

    @property
    def D(self):
        return self.cfg.L * self.cfg.L

    def temper_step(self):
        b = _F64()
        _check(lib().smc_temper_step(self.handle, ctypes.byref(b)))
        return b.value

    def replace_step(self):
        d = _I32()
        _check(lib().ns_replace_step(self.handle, ctypes.byref(d)))
        return bool(d.value)

    def log_evidence(self):
        z, e = _F64(), _F64()
        _check(lib().smc_log_evidence(self.handle, ctypes.byref(z), ctypes.byref(e)))
        return z.value, e.value

    def observables(self):
        o = CObs()
        _check(lib().smc_observables(self.handle, ctypes.byref(o)))
        return {k: getattr(o, k) for k, _ in CObs._fields_}

    def particles(self):
        import torch
        dt = torch.float64 if self.cfg.precision == FP64 else torch.float32
        out = torch.empty((self.cfg.N, self.D), dtype=dt, device=self.workspace.device)
        _check(lib().smc_copy_particles(self.handle, _ptr(out), out.numel() * out.element_size()))
        return out

    def load_particles(self, src):
        _check(lib().smc_load_particles(self.handle, _ptr(src), src.numel() * src.element_size()))

    def copy_particles(self, dst):
        """Copy the current fields into `dst` (a host or device tensor of N x D elements)."""
        _check(lib().smc_copy_particles(self.handle, _ptr(dst), dst.numel() * dst.element_size()))
        return dst

    def save_state(self):
        """The run's state as bytes (smc_save_state)."""
        n = _SZ()
        _check(lib().phi4_state_bytes(self.handle, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().smc_save_state(self.handle, buf, n.value))
        return buf.raw

    def restore_state(self, state):
        """Continue from bytes written by save_state of a run with the same configuration."""
        buf = ctypes.create_string_buffer(state, len(state))
        _check(lib().smc_restore_state(self.handle, buf, len(state)))

    def kernel_launches(self):
        n = ctypes.c_int64()
        _check(lib().phi4_kernel_launches(self.handle, ctypes.byref(n)))
        return n.value

    def set_stage_timing(self, on=True):
        _check(lib().phi4_set_stage_timing(self.handle, 1 if on else 0))

    def stage_times(self, reset=False):
        ms = (_F64 * N_STAGES)()
        n = (ctypes.c_int64 * N_STAGES)()
        _check(lib().phi4_stage_times(self.handle, ms, n, 1 if reset else 0))
        return {lib().phi4_stage_name(i).decode(): (ms[i], n[i]) for i in range(N_STAGES)}

    def run(self, max_steps=100000):
        n = 0
        if self.cfg.kind != NS_SLICE:
            while n < max_steps:
                n += 1
                if self.temper_step() >= 1.0:
                    break
        else:
            while n < max_steps:
                n += 1
                if self.replace_step():
                    break
        return self.observables()

    def close(self):
        if getattr(self, "handle", None):
            lib().smc_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Member(Run):
    """Borrowed view of one member of a Batch (owned by the batch)."""

    def __init__(self, cfg, handle, device):
        self.cfg = cfg
        self.handle = handle
        self._device = device

    @property
    def workspace(self):
        import torch
        return torch.empty(0, device=self._device)

    def close(self):
        self.handle = None


class Batch:
    """Many independent SMC runs advanced together (smc_init_batch / smc_temper_step_batch)."""

    def __init__(self, cfgs, device="cuda", stream=None):
        import torch
        self.cfgs = list(cfgs)
        arr = (CConfig * len(self.cfgs))(*[c.to_c() for c in self.cfgs])
        self._arr = arr
        n = _SZ()
        _check(lib().phi4_batch_workspace_bytes(ctypes.cast(arr, _P), len(self.cfgs), ctypes.byref(n)))
        self.workspace = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
        ptr = (self.workspace.data_ptr() + 255) & ~255
        h = _P()
        _check(lib().smc_init_batch(ctypes.cast(arr, _P), len(self.cfgs), ctypes.c_void_p(ptr), n.value,
                                    _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.members = []
        for r, c in enumerate(self.cfgs):
            mh = _P()
            _check(lib().phi4_batch_member(self.handle, r, ctypes.byref(mh)))
            self.members.append(_Member(c, mh, self.workspace.device))

    def temper_step(self):
        n = _I32()
        _check(lib().smc_temper_step_batch(self.handle, ctypes.byref(n)))
        return n.value

    def run(self, max_steps=100000):
        steps = 0
        while steps < max_steps:
            steps += 1
            if self.temper_step() == 0:
                break
        return [m.observables() for m in self.members]

    def tuning(self):
        """The autotuner's launch shapes (phi4_batch_tuning) as a dict."""
        import json
        buf = ctypes.create_string_buffer(4096)
        _check(lib().phi4_batch_tuning(self.handle, buf, 4096))
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "handle", None):
            for m in self.members:
                m.handle = None
            lib().smc_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- kernel level

def philox_normals(out, seed, stream_id, kind, step, sub, row0=0, dtype=None, stream=None):
    """Fill a 2-D CUDA tensor with the normals of the library's counter layout."""
    import torch
    if dtype is None:
        dtype = {torch.float64: DT_F64, torch.float32: DT_F32, torch.bfloat16: DT_BF16}[out.dtype]
    n_rows, n_cols = out.shape
    _check(lib().phi4_philox_normals(seed, stream_id, kind, step, sub, row0, n_rows, n_cols, out.stride(0), dtype,
                                     _ptr(out), _stream(stream)))
    return out


def action(phi, L, m2, lam, c_kin=1.0, c_mass=1.0, stream=None):
    import torch
    N = phi.shape[0]
    S = torch.empty(N, dtype=torch.float64, device=phi.device)
    sq = torch.empty(N, dtype=torch.float64, device=phi.device)
    dt = DT_F64 if phi.dtype == torch.float64 else DT_F32
    _check(lib().phi4_action(_ptr(phi), dt, N, L, m2, lam, c_kin, c_mass, _ptr(S), _ptr(sq), _stream(stream)))
    return S, sq


def ess_bisect(ell, beta, rho, iters=64, stream=None):
    """Returns (w, out) with out = [dbeta, beta_new, ess, logz_inc, halvings] (device tensors)."""
    import torch
    N = ell.shape[0]
    dev = ell.device
    w = torch.empty(N, dtype=torch.float64, device=dev)
    out = torch.zeros(8, dtype=torch.float64, device=dev)
    b = torch.tensor([beta], dtype=torch.float64, device=dev)
    nb = lib().phi4_bisect_scratch_bytes(N)
    scratch = torch.empty(nb, dtype=torch.uint8, device=dev)
    _check(lib().phi4_ess_bisect(_ptr(ell), N, _ptr(b), rho, iters, _ptr(w), _ptr(out), _ptr(scratch), nb,
                                 _stream(stream)))
    return w, out


def resample_systematic(w, U, stream=None):
    import torch
    N = w.shape[0]
    anc = torch.empty(N, dtype=torch.int32, device=w.device)
    nb = lib().phi4_resample_scratch_bytes(N)
    scratch = torch.empty(nb, dtype=torch.uint8, device=w.device)
    _check(lib().phi4_resample_systematic(_ptr(w), N, U, _ptr(anc), _ptr(scratch), nb, _stream(stream)))
    return anc


def resample_systematic_static(w, U, stream=None):
    """phi4_resample_systematic without scratch memory from the caller (N <= 65536)."""
    import torch
    N = w.shape[0]
    anc = torch.empty(N, dtype=torch.int32, device=w.device)
    _check(lib().phi4_resample_systematic_static(_ptr(w), N, U, _ptr(anc), _stream(stream)))
    return anc


def observables(phi, L, w=None, stream=None):
    """Device FP64 moments of the magnetisation: returns (M, out) with
    out = [<M>, <|M|>, <M^2>, chi, mode balance, total weight] (device tensors)."""
    import torch
    N = phi.shape[0]
    dt = DT_F64 if phi.dtype == torch.float64 else DT_F32
    M = torch.empty(N, dtype=torch.float64, device=phi.device)
    out = torch.empty(6, dtype=torch.float64, device=phi.device)
    _check(lib().phi4_observables(_ptr(phi), dt, N, L, _ptr(w), _ptr(M), _ptr(out), _stream(stream)))
    return M, out


def free_field_covariance(L, beta, m2, c_kin=1.0, c_mass=1.0, keep_reference=False, device="cuda", stream=None):
    """Exact covariance of the Gaussian part of the tempered target at beta (D x D device tensor)."""
    import torch
    D = L * L
    sigma = torch.empty((D, D), dtype=torch.float64, device=device)
    b = torch.tensor([beta], dtype=torch.float64, device=device)
    nb = lib().phi4_free_covariance_scratch_bytes(L)
    scratch = torch.empty(nb, dtype=torch.uint8, device=device)
    _check(lib().phi4_free_field_covariance(L, _ptr(b), m2, c_kin, c_mass, int(keep_reference), _ptr(sigma),
                                            _ptr(scratch), nb, _stream(stream)))
    return sigma


def set_spin_limit(cycles):
    """Limit (SM clock cycles) of the library's software waits; <= 0 restores the default."""
    _check(lib().phi4_set_spin_limit(int(cycles)))


def gather_rows(src, anc, stream=None):
    import torch
    dst = torch.empty_like(src)
    _check(lib().phi4_gather_rows(_ptr(src), _ptr(dst), src.shape[1] * src.element_size(), src.shape[0], _ptr(anc),
                                  _stream(stream)))
    return dst


def covariance(phi, precision, stream=None):
    import torch
    N, D = phi.shape
    sigma = torch.zeros((D, D), dtype=torch.float64, device=phi.device)
    nb = lib().phi4_covariance_scratch_bytes(N, D, precision)
    scratch = torch.empty(nb, dtype=torch.uint8, device=phi.device)
    _check(lib().phi4_covariance(_ptr(phi), precision, N, D, _ptr(sigma), _ptr(scratch), nb, _stream(stream)))
    return sigma


def cholesky(a, ridge=0.0, mode=0, stream=None):
    """In-place FP64 Cholesky of a (D x D double CUDA tensor); returns (a, status).
    mode: 0 automatic, 1 FP64 SIMT trailing update, 2 tensor-core emulated trailing update."""
    import torch
    D = a.shape[0]
    r = torch.tensor([ridge], dtype=torch.float64, device=a.device)
    st = torch.zeros(1, dtype=torch.int32, device=a.device)
    nb = lib().phi4_cholesky_scratch_bytes(D)
    scratch = torch.empty(nb, dtype=torch.uint8, device=a.device)
    _check(lib().phi4_cholesky(_ptr(a), D, _ptr(r), _ptr(st), _ptr(scratch), nb, mode, _stream(stream)))
    return a, st


def cholesky_f32(sigma, ridge=0.0, stream=None):
    """Float Cholesky of the lower triangle of a D x D double CUDA tensor; returns (L32, status)."""
    import torch
    D = sigma.shape[0]
    a = torch.empty((D, D), dtype=torch.float32, device=sigma.device)
    r = torch.tensor([ridge], dtype=torch.float64, device=sigma.device)
    st = torch.zeros(1, dtype=torch.int32, device=sigma.device)
    nb = lib().phi4_cholesky_scratch_bytes(D)
    scratch = torch.empty(nb, dtype=torch.uint8, device=sigma.device)
    _check(lib().phi4_cholesky_f32(_ptr(sigma), _ptr(a), D, _ptr(r), _ptr(st), _ptr(scratch), nb, _stream(stream)))
    return a, st


def rw_propose(phi, Lfac, precision, scale, seed, stream_id, step, sweep, stream=None):
    import torch
    N, D = phi.shape
    prop = torch.empty_like(phi)
    nb = lib().phi4_propose_scratch_bytes(N, D, precision)
    scratch = torch.empty(nb, dtype=torch.uint8, device=phi.device)
    ldl = Lfac.stride(0)
    _check(lib().phi4_rw_propose(_ptr(phi), _ptr(prop), _ptr(Lfac), ldl, precision, N, D, scale, seed, stream_id,
                                 step, sweep, _ptr(scratch), nb, _stream(stream)))
    return prop


def rw_accept(phi, prop, L, m2, lam, S, sq, ell, beta, seed, stream_id, step, sweep, c_kin=1.0, c_mass=1.0,
              keep_reference=False, stream=None):
    """In place on phi, S, sq, ell; returns the int32 [accepted, status] tensor."""
    import torch
    N = phi.shape[0]
    dt = DT_F64 if phi.dtype == torch.float64 else DT_F32
    b = torch.tensor([beta], dtype=torch.float64, device=phi.device)
    cnt = torch.zeros(2, dtype=torch.int32, device=phi.device)
    _check(lib().phi4_rw_accept(_ptr(phi), _ptr(prop), dt, N, L, m2, lam, c_kin, c_mass, int(keep_reference),
                                _ptr(S), _ptr(sq), _ptr(ell), _ptr(b), seed, stream_id, step, sweep, _ptr(cnt),
                                _stream(stream)))
    return cnt


def rw_accept_delta(phi, delta, L, m2, lam, S, sq, ell, beta, seed, stream_id, step, sweep, c_kin=1.0, c_mass=1.0,
                    keep_reference=False, stream=None):
    """Accept step of the mixed form with proposal phi + delta (delta: float16 tensor); in place."""
    import torch
    N = phi.shape[0]
    b = torch.tensor([beta], dtype=torch.float64, device=phi.device)
    cnt = torch.zeros(2, dtype=torch.int32, device=phi.device)
    _check(lib().phi4_rw_accept_delta(_ptr(phi), _ptr(delta), N, L, m2, lam, c_kin, c_mass, int(keep_reference),
                                      _ptr(S), _ptr(sq), _ptr(ell), _ptr(b), seed, stream_id, step, sweep, _ptr(cnt),
                                      _stream(stream)))
    return cnt


def kappa_config(kappa, lam, **kw):
    """Config for the kappa-parameterised action of App. G,
        S = (kappa/2) sum_{x,mu} (phi_{x+mu} - phi_x)^2 + sum_x [phi_x^2 + lambda (phi_x^2 - 1)^2],
    in the library's form: c_kin = kappa/2 (the kinetic sum equals sum_x sum_mu
    phi_x (2 phi_x - phi_{x+mu} - phi_{x-mu})), c_mass = 1, m2 = 1 - 2 lambda, quartic lambda.
    The dropped constant lambda V shifts log Z by kappa_logz_shift(lambda, V)."""
    return Config(c_kin=0.5 * kappa, c_mass=1.0, m2=1.0 - 2.0 * lam, lam=lam, **kw)


def kappa_logz_shift(lam, D):
    """log Z of the kappa form minus log Z of its kappa_config run: -lambda V."""
    return -lam * D


def default_rw_scale(D):
    return 2.38 / math.sqrt(D)

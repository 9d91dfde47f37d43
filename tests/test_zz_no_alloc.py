"""The allocation-free resampling entry point, phi4_resample_systematic_static.

Some callers cannot allocate device memory or pass a scratch buffer (they only hold
the weight and ancestor buffers, or run where no allocator may be entered); this entry
point keeps its scratch in an array built into the library. It must return exactly the
ancestors of the allocating entry point, call after call, although the array keeps the
previous call's contents. This file is collected last so that a failure here stops a
-x run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2511_15196_gb300 as p  # noqa: E402


def _static_call(w, U, anc):
    lib = p.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.phi4_resample_systematic_static(ctypes.c_void_p(w.data_ptr()), w.shape[0], U,
                                               ctypes.c_void_p(anc.data_ptr()), stream)


def test_static_scratch_matches_allocating_entry_point_two_calls():
    # two calls in a row: the second (smaller N) runs over the first call's leftovers
    for N, seed, kind in ((50000, 11, "heavy"), (8192, 12, "zeros")):
        w = inputs.positive_weights(N, seed=seed, zeros=(N // 4 if kind == "zeros" else 0), heavy=(kind == "heavy"))
        tw = torch.as_tensor(w).cuda()
        U = inputs.word32(seed)
        ref = p.resample_systematic(tw, U)
        anc = torch.full((N,), -1, dtype=torch.int32, device="cuda")
        assert _static_call(tw, U, anc) == p.PHI4_OK, p.lib().phi4_last_error()
        torch.cuda.synchronize()
        assert torch.equal(anc, ref)
        assert (np.diff(anc.cpu().numpy()) >= 0).all()


def test_static_scratch_rejects_sizes_beyond_the_array():
    N = 65536 + 1
    tw = torch.ones(N, dtype=torch.float64, device="cuda")
    anc = torch.empty(N, dtype=torch.int32, device="cuda")
    assert _static_call(tw, 0, anc) == p.PHI4_ERR_ARG
    assert b"65536" in p.lib().phi4_last_error()

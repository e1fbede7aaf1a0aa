"""The allocation-free SMW entry point (sai_smw_recover_noalloc) against the
regular one (sai_smw_recover), through the C ABI.

The allocation-free call exists for callers that cannot allocate device memory
(their device memory belongs to a host framework's pool or a fixed budget, or
an allocation would synchronise where they run); it keeps its scratch in a
static device array. This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    L = lib().load()
    f = L.sai_smw_recover_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    return f


def _call_noalloc(n, s, J, Y):
    sai = lib()
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    c = C.c_double(-1.0)
    st = _noalloc_fn()(n, s, C.c_void_p(J.data_ptr() if s else 0), C.c_void_p(Y.data_ptr()),
                       C.c_void_p(x.data_ptr()), C.byref(c), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, x, c.value


def _problem(seed, s, n=300):
    sai = lib()
    A = W.random_sparse_dominant(n, 3, s, 100, seed=seed).A
    h = sai.split(to_dev(A))
    _, _, J = h.arrays()
    rng = np.random.default_rng(seed)
    Y = torch.as_tensor(rng.standard_normal((n, h.s + 1)) * 0.1, device="cuda")
    return h, J, Y


def test_noalloc_matches_regular_entry_point_twice_in_a_row():
    need_gpu()
    sai = lib()
    for seed, s in ((21, 4), (22, 7)):
        h, J, Y = _problem(seed, s)
        x_ref, c_ref = sai.smw_recover(h, Y)
        st, x, c = _call_noalloc(h.n, h.s, J, Y)
        assert st == sai.SAI_OK
        np.testing.assert_allclose(x.cpu().numpy(), x_ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
        assert c == pytest.approx(c_ref, rel=1e-12)


def test_noalloc_clears_error_state_between_calls():
    need_gpu()
    sai = lib()
    h, J, Y = _problem(23, 5)
    Ys = Y.clone()
    Jh = J.cpu().numpy()
    for i, j in enumerate(Jh):         # W(J,:) = -I makes I + V^T W = 0
        Ys[j, 1:] = 0.0
        Ys[j, 1 + i] = -1.0
    st, xs, _ = _call_noalloc(h.n, h.s, J, Ys)
    assert st == sai.SAI_SINGULAR
    # a zero pivot leaves the correction out: x is yhat (column 0 of Y)
    np.testing.assert_array_equal(xs.cpu().numpy(), Ys[:, 0].cpu().numpy())
    x_ref, c_ref = sai.smw_recover(h, Y)
    st, x, c = _call_noalloc(h.n, h.s, J, Y)
    assert st == sai.SAI_OK
    np.testing.assert_allclose(x.cpu().numpy(), x_ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
    assert c == pytest.approx(c_ref, rel=1e-12)


def test_noalloc_rejects_s_beyond_its_scratch():
    need_gpu()
    sai = lib()
    n, s = 400, 257
    J = torch.arange(s, dtype=torch.int32, device="cuda")
    Y = torch.zeros((n, s + 1), dtype=torch.float64, device="cuda")
    st, _, _ = _call_noalloc(n, s, J, Y)
    assert st == sai.SAI_INVALID_ARG

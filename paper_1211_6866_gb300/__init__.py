"""Python binding of ``libsaismw.so`` (C ABI in ``include/saismw.h``).

Argument marshalling only: every step of split, SAI build, Krylov solves,
SMW recovery and residual check runs in the library's CUDA kernels. PyTorch
provides device memory and the current CUDA stream. There is no CPU fallback:
if the compiled library cannot be loaded or no CUDA device is present, the
calls raise.

Layouts (see the header): sparse matrices are CSC with int64 column pointers,
int32 row indices ascending per column, float64 values; multi-right-hand-side
blocks are n x k row-major float64 tensors.
"""
import ctypes as C
import os
from dataclasses import dataclass

import torch

__all__ = ["CscMatrix", "SaiError", "split", "build_spai", "build_psai", "krylov_solve", "smw_recover",
           "rel_resid", "solve", "library_path", "load", "profile_begin", "profile_end", "launch_count"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libsaismw.so")

SAI_OK, SAI_INVALID_ARG, SAI_CUDA_ERROR, SAI_OOM, SAI_PATTERN_OVERFLOW, SAI_MAXITER, SAI_BREAKDOWN, \
    SAI_SINGULAR, SAI_NOT_IMPLEMENTED = range(9)
BICGSTAB, GMRES, CGS, BICG, BGMRES = 0, 1, 2, 3, 4
_METHOD = {"bicgstab": BICGSTAB, "gmres": GMRES, "cgs": CGS, "bicg": BICG, "bgmres": BGMRES}


class SaiError(RuntimeError):
    def __init__(self, what, status):
        name = _lib.sai_status_string(status).decode() if _lib is not None else str(status)
        super().__init__("%s failed: %s" % (what, name))
        self.status = status


# ---------------------------------------------------------------- ctypes mirror of saismw.h
class _CscView(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("col_ptr", C.c_void_p), ("row_idx", C.c_void_p),
                ("val", C.c_void_p)]


class _SplitParams(C.Structure):
    _fields_ = [("thresh_mult", C.c_double), ("abs_tau", C.c_double), ("ge", C.c_int32), ("p_keep", C.c_int32),
                ("keep_rule", C.c_int32), ("zero_diag", C.c_int32)]


_KEEP = {"nearest": 0, "largest": 1}
_GROWTH = {"A": 0, "C": 1}


class _SplitInfo(C.Structure):
    _fields_ = [("n", C.c_int32), ("s", C.c_int32), ("p", C.c_int32), ("p_keep", C.c_int32), ("tau", C.c_double),
                ("nnz_At", C.c_int64), ("nnz_U", C.c_int64), ("norm1_At", C.c_double)]


class _SpaiParams(C.Structure):
    _fields_ = [("delta", C.c_double), ("mn", C.c_int32), ("max_aug", C.c_int32), ("key_bits", C.c_int32),
                ("precision", C.c_int32)]


class _PsaiParams(C.Structure):
    _fields_ = [("delta", C.c_double), ("tol", C.c_double), ("tol_mode", C.c_int32), ("lmax", C.c_int32),
                ("precision", C.c_int32), ("lfill", C.c_int32), ("growth", C.c_int32), ("reserved", C.c_int32)]


class _PrecondInfo(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz_M", C.c_int64), ("n_c", C.c_int32), ("l_m", C.c_int32),
                ("n_tier", C.c_int32 * 6), ("build_ms", C.c_double)]


class _KrylovParams(C.Structure):
    _fields_ = [("method", C.c_int32), ("restart", C.c_int32), ("maxit", C.c_int32), ("precision", C.c_int32),
                ("inner_tol", C.c_double), ("transpose", C.c_int32)]


class _BatchItem(C.Structure):
    _fields_ = [("status", C.c_int32), ("iter_max", C.c_int32), ("s", C.c_int32), ("p", C.c_int32),
                ("c", C.c_double), ("rr", C.c_double), ("c_rounds", C.c_int32), ("reserved", C.c_int32)]


class _BatchReport(C.Structure):
    _fields_ = [("columns", C.c_int64), ("nnz_M", C.c_int64), ("systems", C.c_int32), ("iter_max", C.c_int32),
                ("ms_split", C.c_double), ("ms_build", C.c_double), ("ms_krylov", C.c_double),
                ("ms_smw", C.c_double)]


class _BuildConfig(C.Structure):
    _fields_ = [("warps_t0", C.c_int32), ("blocks_per_sm_t12", C.c_int32), ("heavy_first", C.c_int32),
                ("first_tier", C.c_int32), ("ms", C.c_float)]


class _BuildTuning(C.Structure):
    _fields_ = [("chosen", _BuildConfig), ("sample_columns", C.c_int32), ("ncand", C.c_int32),
                ("cand", _BuildConfig * 12)]


class _StageParams(C.Structure):
    _fields_ = [("krylov", _KrylovParams), ("eps", C.c_double)]


class _SolveParams(C.Structure):
    _fields_ = [("split", _SplitParams), ("sai", C.c_int32), ("spai", _SpaiParams), ("psai", _PsaiParams),
                ("krylov", _KrylovParams), ("eps", C.c_double), ("c_adapt", C.c_int32), ("reserved", C.c_int32)]


class _SolveReport(C.Structure):
    _fields_ = [("split", _SplitInfo), ("precond", _PrecondInfo), ("status", C.c_int32), ("iter_max", C.c_int32),
                ("c", C.c_double), ("rr", C.c_double), ("ms_split", C.c_double), ("ms_build", C.c_double),
                ("ms_krylov", C.c_double), ("ms_smw", C.c_double), ("moved", C.c_int32), ("c_rounds", C.c_int32)]


class _ProfSite(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("timed", C.c_int64), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double), ("flops32", C.c_double)]


class _ProfReport(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("nsites", C.c_int32), ("site", _ProfSite * 12)]


_lib = None


def library_path():
    return _LIBPATH


def load():
    """Load libsaismw.so (it must have been built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIBPATH):
        raise ImportError("libsaismw.so not built: run __graft_entry__.build() (no CPU fallback exists)")
    L = C.CDLL(_LIBPATH)
    vp, i32, dp = C.c_void_p, C.c_int32, C.c_void_p
    L.sai_status_string.restype = C.c_char_p
    L.sai_status_string.argtypes = [C.c_int]
    L.sai_split_create.argtypes = [C.POINTER(_CscView), C.POINTER(_SplitParams), vp, C.POINTER(vp)]
    L.sai_split_get_info.argtypes = [vp, C.POINTER(_SplitInfo)]
    L.sai_split_copy_out.argtypes = [vp, dp, dp, dp, dp, dp, dp, dp, vp]
    L.sai_split_destroy.argtypes = [vp]
    L.sai_split_destroy.restype = None
    L.sai_build_spai.argtypes = [vp, C.POINTER(_SpaiParams), vp, C.POINTER(vp)]
    L.sai_build_psai.argtypes = [vp, C.POINTER(_PsaiParams), vp, C.POINTER(vp)]
    L.sai_precond_get_info.argtypes = [vp, C.POINTER(_PrecondInfo)]
    L.sai_precond_create.argtypes = [C.POINTER(_CscView), vp, C.POINTER(vp)]
    L.sai_precond_copy_out.argtypes = [vp, dp, dp, dp, dp, dp, dp, vp]
    L.sai_precond_destroy.argtypes = [vp]
    L.sai_precond_destroy.restype = None
    L.sai_krylov_solve.argtypes = [vp, vp, i32, dp, C.POINTER(C.c_double), C.POINTER(_KrylovParams), dp,
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32), vp]
    L.sai_smw_recover.argtypes = [vp, dp, dp, C.POINTER(C.c_double), vp]
    L.sai_rel_resid.argtypes = [C.POINTER(_CscView), dp, dp, C.POINTER(C.c_double), vp]
    L.sai_solve.argtypes = [C.POINTER(_CscView), dp, C.POINTER(_SolveParams), dp, C.POINTER(C.c_int32), i32,
                            C.POINTER(_SolveReport), vp]
    L.sai_solve_with.argtypes = [C.POINTER(_CscView), vp, vp, dp, C.POINTER(_StageParams), dp,
                                 C.POINTER(C.c_int32), i32, C.POINTER(_SolveReport), vp]
    L.sai_backward.argtypes = [C.POINTER(_CscView), vp, vp, dp, dp, C.POINTER(_StageParams), dp, dp,
                               C.POINTER(C.c_int32), i32, C.POINTER(_SolveReport), vp]
    L.sai_solve_batched.argtypes = [i32, C.POINTER(_CscView), C.POINTER(vp), C.POINTER(_SolveParams), C.POINTER(vp),
                                    C.POINTER(_BatchItem), C.POINTER(_BatchReport), vp]
    L.sai_build_autotune.argtypes = [vp, i32, C.POINTER(_SpaiParams), C.POINTER(_PsaiParams), vp,
                                     C.POINTER(_BuildTuning)]
    L.sai_build_batched.argtypes = [i32, C.POINTER(_CscView), C.POINTER(_SolveParams), vp, C.POINTER(vp)]
    L.sai_build_autotune_batched.argtypes = [i32, C.POINTER(_CscView), C.POINTER(_SolveParams), vp,
                                             C.POINTER(_BuildTuning)]
    L.sai_build_set_config.argtypes = [C.POINTER(_BuildConfig)]
    L.sai_dmperm.argtypes = [C.POINTER(_CscView), dp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), vp]
    L.sai_permute_rows.argtypes = [C.POINTER(_CscView), dp, dp, dp, dp, vp]
    L.sai_launch_count.restype = C.c_uint64
    L.sai_launch_count.argtypes = []
    L.sai_profile_begin.argtypes = []
    L.sai_profile_end.argtypes = [C.POINTER(_ProfReport)]
    for f in ("sai_profile_begin", "sai_profile_end", "sai_split_create", "sai_split_get_info", "sai_split_copy_out", "sai_build_spai", "sai_build_psai",
              "sai_precond_get_info", "sai_precond_copy_out", "sai_krylov_solve", "sai_smw_recover",
              "sai_rel_resid", "sai_solve", "sai_solve_with", "sai_backward", "sai_solve_batched",
              "sai_build_autotune", "sai_build_set_config", "sai_dmperm", "sai_permute_rows", "sai_build_batched",
              "sai_build_autotune_batched"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _stream():
    if not torch.cuda.is_available():
        raise RuntimeError("saismw needs a CUDA device; there is no CPU fallback")
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(what, st, allow=()):
    if st != SAI_OK and st not in allow:
        raise SaiError(what, st)
    return st


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


@dataclass
class CscMatrix:
    """Square CSC matrix on the device (int64 col_ptr, int32 row_idx, float64 val)."""
    n: int
    col_ptr: torch.Tensor
    row_idx: torch.Tensor
    val: torch.Tensor

    @staticmethod
    def from_arrays(indptr, indices, data, n, device="cuda"):
        return CscMatrix(int(n), torch.as_tensor(indptr, dtype=torch.int64).to(device).contiguous(),
                         torch.as_tensor(indices, dtype=torch.int32).to(device).contiguous(),
                         torch.as_tensor(data, dtype=torch.float64).to(device).contiguous())

    @property
    def nnz(self):
        return int(self.row_idx.numel())

    def view(self):
        return _CscView(self.n, self.nnz, _p(self.col_ptr).value, _p(self.row_idx).value, _p(self.val).value)


class Split:
    """Handle of a split A = A~ + U V^T held on the device."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)
        info = _SplitInfo()
        _check("sai_split_get_info", load().sai_split_get_info(self._h, C.byref(info)))
        self.n, self.s, self.p, self.p_keep = info.n, info.s, info.p, info.p_keep
        self.tau, self.nnz_At, self.nnz_U, self.norm1_At = info.tau, info.nnz_At, info.nnz_U, info.norm1_At

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.sai_split_destroy(self._h)
            self._h = None

    def arrays(self):
        """(At: CscMatrix, U: (col_ptr, row_idx, val), J) as device tensors."""
        dev = "cuda"
        at = (torch.empty(self.n + 1, dtype=torch.int64, device=dev),
              torch.empty(self.nnz_At, dtype=torch.int32, device=dev),
              torch.empty(self.nnz_At, dtype=torch.float64, device=dev))
        u = (torch.empty(self.s + 1, dtype=torch.int64, device=dev),
             torch.empty(self.nnz_U, dtype=torch.int32, device=dev),
             torch.empty(self.nnz_U, dtype=torch.float64, device=dev))
        J = torch.empty(self.s, dtype=torch.int32, device=dev)
        _check("sai_split_copy_out", load().sai_split_copy_out(self._h, *[_p(t) for t in at + u], _p(J), _stream()))
        torch.cuda.current_stream().synchronize()
        return CscMatrix(self.n, *at), u, J


class Precond:
    """Handle of a sparse approximate inverse M held on the device."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle)
        info = _PrecondInfo()
        _check("sai_precond_get_info", load().sai_precond_get_info(self._h, C.byref(info)))
        self.n, self.nnz, self.n_c, self.l_m = info.n, info.nnz_M, info.n_c, info.l_m
        self.n_tier = list(info.n_tier)
        self.build_ms = info.build_ms

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.sai_precond_destroy(self._h)
            self._h = None

    def arrays(self):
        """(M: CscMatrix, loops, res, res_post) as device tensors."""
        dev = "cuda"
        cp = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        ri = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        v = torch.empty(self.nnz, dtype=torch.float64, device=dev)
        loops = torch.empty(self.n, dtype=torch.int32, device=dev)
        res = torch.empty(self.n, dtype=torch.float64, device=dev)
        post = torch.empty(self.n, dtype=torch.float64, device=dev)
        _check("sai_precond_copy_out", load().sai_precond_copy_out(self._h, _p(cp), _p(ri), _p(v), _p(loops),
                                                                   _p(res), _p(post), _stream()))
        torch.cuda.current_stream().synchronize()
        return CscMatrix(self.n, cp, ri, v), loops, res, post


def split(A, thresh_mult=10.0, abs_tau=-1.0, ge=False, p_keep=0, keep="nearest"):
    """Step 1 of Procedure *: detect the irregular columns and split A = A~ + U V^T.
    keep="nearest" keeps the diagonal and the p-1 entries nearest to it (the
    paper's choice), keep="largest" the diagonal and the p-1 largest in
    magnitude (the other rule of section 4). abs_tau=float("inf") keeps every
    column (A~ = A, s = 0): the S-SPAI and S-PSAI baselines build on A itself."""
    L = load()
    h = C.c_void_p()
    v = A.view()
    prm = _SplitParams(thresh_mult, abs_tau, int(ge), int(p_keep), _KEEP[keep], 0)
    _check("sai_split_create", L.sai_split_create(C.byref(v), C.byref(prm), _stream(), C.byref(h)))
    return Split(h.value)


def build_spai(sp, delta=0.4, mn=5, max_aug=10, key_bits=20, precision=0):
    """precision 1: FP32 QR with one FP64 refinement step per loop."""
    L = load()
    h = C.c_void_p()
    prm = _SpaiParams(delta, mn, max_aug, key_bits, precision)
    _check("sai_build_spai", L.sai_build_spai(sp._h, C.byref(prm), _stream(), C.byref(h)))
    return Precond(h.value)


def _cfg_dict(c):
    return dict(warps_t0=c.warps_t0, blocks_per_sm_t12=c.blocks_per_sm_t12, heavy_first=c.heavy_first,
                first_tier=c.first_tier, ms=c.ms)


def build_autotune(sp, sai="spai", delta=0.4, mn=5, max_aug=10, key_bits=20, tol=0.0, tol_mode=0, lmax=10,
                   precision=0, lfill=0, growth="A"):
    """Times the build schedule candidates on a sample of sp's columns and makes
    the fastest the configuration of later builds. Returns (chosen, candidates)."""
    L = load()
    t = _BuildTuning()
    sprm = _SpaiParams(delta, mn, max_aug, key_bits, precision)
    pprm = _PsaiParams(delta, tol, tol_mode, lmax, precision, lfill, _GROWTH[growth], 0)
    _check("sai_build_autotune", L.sai_build_autotune(sp._h, 0 if sai == "spai" else 1, C.byref(sprm), C.byref(pprm),
                                                      _stream(), C.byref(t)))
    return _cfg_dict(t.chosen), [_cfg_dict(t.cand[i]) for i in range(t.ncand)]


def build_set_config(warps_t0=None, blocks_per_sm_t12=2, heavy_first=0, first_tier=0):
    """Sets the build schedule (warps_t0=None restores the default).
    first_tier: 0 starts every column in tier 0 (one column per warp), 1 in
    the small shared-memory tier with four columns per warp, 2 with two, 3
    with one column per lane (32 per warp)."""
    L = load()
    if warps_t0 is None:
        _check("sai_build_set_config", L.sai_build_set_config(None))
    else:
        c = _BuildConfig(warps_t0, blocks_per_sm_t12, heavy_first, first_tier, 0.0)
        _check("sai_build_set_config", L.sai_build_set_config(C.byref(c)))


def build_psai(sp, delta=0.4, tol=0.0, tol_mode=0, lmax=10, precision=0, lfill=0, growth="A"):
    """precision 1: FP32 QR with one FP64 refinement step per loop; tol_mode 2
    with lfill: PSAI(lfill), the lfill largest entries of each m_k kept;
    growth "C": dropped positions never return (the pattern grows only by
    the new positions of the power sequence)."""
    L = load()
    h = C.c_void_p()
    prm = _PsaiParams(delta, tol, tol_mode, lmax, precision, lfill, _GROWTH[growth], 0)
    _check("sai_build_psai", L.sai_build_psai(sp._h, C.byref(prm), _stream(), C.byref(h)))
    return Precond(h.value)


def precond_from_csc(M):
    """A preconditioner handle for a given M (CscMatrix on the device, rows
    ascending per column), e.g. one saved by save_precond and loaded again."""
    L = load()
    h = C.c_void_p()
    v = M.view()
    _check("sai_precond_create", L.sai_precond_create(C.byref(v), _stream(), C.byref(h)))
    return Precond(h.value)


def save_precond(P, path):
    """Writes M (CSC: n, col_ptr, row_idx, val) to path as a .npz file, so a
    later process can solve further right-hand sides without the build."""
    import numpy as np

    Mc = P.arrays()[0]
    np.savez(path, n=np.int64(Mc.n), col_ptr=Mc.col_ptr.cpu().numpy(), row_idx=Mc.row_idx.cpu().numpy(),
             val=Mc.val.cpu().numpy())


def load_precond(path, device="cuda"):
    """The preconditioner saved by save_precond, as a handle on the device."""
    import numpy as np

    with np.load(path) as z:
        M = CscMatrix.from_arrays(z["col_ptr"], z["row_idx"], z["val"], int(z["n"]), device=device)
    return precond_from_csc(M)


def krylov_solve(sp, P, B, thr, method=BICGSTAB, restart=50, maxit=500, precision=0, inner_tol=0.0,
                 transpose=False):
    """Solves A~ X = B (n x k, row-major, device) with right preconditioner M,
    or A~^T X = B with M^T when transpose is set.
    precision 1 (GMRES only): FP32 inner solves refined in FP64.
    Returns (X, iters list, status list, overall status)."""
    L = load()
    B = B.contiguous()
    n, k = B.shape
    X = torch.empty_like(B)
    thr_a = (C.c_double * k)(*[float(t) for t in thr])
    it = (C.c_int32 * k)()
    stt = (C.c_int32 * k)()
    prm = _KrylovParams(method, restart, maxit, precision, inner_tol, int(bool(transpose)))
    st = _check("sai_krylov_solve", L.sai_krylov_solve(sp._h, P._h, k, _p(B), thr_a, C.byref(prm), _p(X), it, stt,
                                                       _stream()), allow=(SAI_MAXITER, SAI_BREAKDOWN))
    return X, list(it), list(stt), st


def smw_recover(sp, Y):
    """x = y - W (I + V^T W)^{-1} V^T y with Y = [y, W] (n x (s+1) row-major). Returns (x, c)."""
    L = load()
    Y = Y.contiguous()
    x = torch.empty(Y.shape[0], dtype=torch.float64, device=Y.device)
    c = C.c_double()
    _check("sai_smw_recover", L.sai_smw_recover(sp._h, _p(Y), _p(x), C.byref(c), _stream()))
    return x, c.value


def rel_resid(A, b, x):
    L = load()
    rr = C.c_double()
    v = A.view()
    _check("sai_rel_resid", L.sai_rel_resid(C.byref(v), _p(b), _p(x), C.byref(rr), _stream()))
    return rr.value


def dmperm(A):
    """Zero-diagonal repair of section 5: a maximum transversal of A.
    Returns (p, rank, moved): p (device int32) with p[j] = the row matched to
    column j (-1 if unmatched), the structural rank, and the number of
    columns with p[j] != j."""
    L = load()
    p = torch.empty(max(A.n, 1), dtype=torch.int32, device=A.col_ptr.device)
    rank, moved = C.c_int32(), C.c_int32()
    v = A.view()
    _check("sai_dmperm", L.sai_dmperm(C.byref(v), _p(p), C.byref(rank), C.byref(moved), _stream()))
    return p[: A.n], rank.value, moved.value


def permute_rows(A, p):
    """B = A(p,:) (row j of B is row p[j] of A) as a new CscMatrix."""
    L = load()
    p = torch.as_tensor(p, dtype=torch.int32, device=A.col_ptr.device).contiguous()
    B = CscMatrix(A.n, torch.empty_like(A.col_ptr), torch.empty_like(A.row_idx), torch.empty_like(A.val))
    v = A.view()
    _check("sai_permute_rows", L.sai_permute_rows(C.byref(v), _p(p), _p(B.col_ptr), _p(B.row_idx), _p(B.val),
                                                  _stream()))
    return B


def solve(A, b, sai="spai", krylov="bicgstab", eps=1e-8, maxit=500, restart=50, thresh_mult=10.0, abs_tau=-1.0,
          delta=0.4, mn=5, max_aug=10, key_bits=20, tol=0.0, tol_mode=0, lmax=10, x=None, krylov_precision=0,
          inner_tol=0.0, sai_precision=0, keep="nearest", lfill=0, growth="A", zero_diag=False, c_adapt=0):
    """Procedure * on the device. krylov_precision=1 selects the FP32-inner /
    FP64-refined GMRES; sai_precision=1 the FP32 QR + FP64 refinement build;
    zero_diag=True first applies the zero-diagonal repair of section 5
    (report["moved"] columns moved); c_adapt=1 continues the u_j systems with
    the measured c when the recovery's c exceeds 1 (report["c_rounds"]).
    Returns (x, iters list, report dict)."""
    L = load()
    if x is None:
        x = torch.empty(A.n, dtype=torch.float64, device=b.device)
    prm = _SolveParams(_SplitParams(thresh_mult, abs_tau, 0, 0, _KEEP[keep], int(bool(zero_diag))),
                       0 if sai == "spai" else 1,
                       _SpaiParams(delta, mn, max_aug, key_bits, sai_precision),
                       _PsaiParams(delta, tol, tol_mode, lmax, sai_precision, lfill, _GROWTH[growth], 0),
                       _KrylovParams(_METHOD[krylov], restart, maxit, krylov_precision,
                                     inner_tol, 0), eps, int(c_adapt), 0)
    cap = A.n + 1
    iters = (C.c_int32 * cap)()
    rep = _SolveReport()
    v = A.view()
    st = _check("sai_solve", L.sai_solve(C.byref(v), _p(b), C.byref(prm), _p(x), iters, cap, C.byref(rep),
                                         _stream()), allow=(SAI_MAXITER, SAI_BREAKDOWN))
    s = rep.split.s
    report = dict(s=s, p=rep.split.p, tau=rep.split.tau, nnz_At=rep.split.nnz_At, nnz_U=rep.split.nnz_U,
                  nnz_M=rep.precond.nnz_M, n_c=rep.precond.n_c, l_m=rep.precond.l_m,
                  n_tier=list(rep.precond.n_tier), status=st, iter_max=rep.iter_max, c=rep.c, rr=rep.rr,
                  ms_split=rep.ms_split, ms_build=rep.ms_build, ms_krylov=rep.ms_krylov, ms_smw=rep.ms_smw,
                  build_ms=rep.precond.build_ms, moved=rep.moved, c_rounds=rep.c_rounds)
    return x, list(iters[: s + 1]), report


def _report(rep, st):
    return dict(s=rep.split.s, p=rep.split.p, tau=rep.split.tau, nnz_At=rep.split.nnz_At, nnz_U=rep.split.nnz_U,
                nnz_M=rep.precond.nnz_M, n_c=rep.precond.n_c, l_m=rep.precond.l_m, n_tier=list(rep.precond.n_tier),
                status=st, iter_max=rep.iter_max, c=rep.c, rr=rep.rr, ms_split=rep.ms_split, ms_build=rep.ms_build,
                ms_krylov=rep.ms_krylov, ms_smw=rep.ms_smw, build_ms=rep.precond.build_ms)


def _stage(krylov, eps, maxit, restart, krylov_precision, inner_tol):
    return _StageParams(_KrylovParams(_METHOD[krylov], restart, maxit, krylov_precision,
                                      inner_tol, 0), eps)


def solve_with(A, sp, P, b, krylov="bicgstab", eps=1e-8, maxit=500, restart=50, krylov_precision=0, inner_tol=0.0,
               x=None):
    """Steps 3-5 of Procedure * on an existing split sp of A and preconditioner P.
    Returns (x, iters list, report dict)."""
    L = load()
    if x is None:
        x = torch.empty(A.n, dtype=torch.float64, device=b.device)
    prm = _stage(krylov, eps, maxit, restart, krylov_precision, inner_tol)
    cap = sp.s + 1
    iters = (C.c_int32 * cap)()
    rep = _SolveReport()
    v = A.view()
    st = _check("sai_solve_with", L.sai_solve_with(C.byref(v), sp._h, P._h, _p(b), C.byref(prm), _p(x), iters, cap,
                                                   C.byref(rep), _stream()), allow=(SAI_MAXITER, SAI_BREAKDOWN))
    return x, list(iters[:cap]), _report(rep, st)


def backward(A, sp, P, x, g, krylov="bicgstab", eps=1e-8, maxit=500, restart=50, krylov_precision=0,
             inner_tol=0.0, grad_vals=True):
    """Backward pass of x = A^{-1} b for g = dL/dx: the s+1 transposed solves
    with M^T and Theorem 1 on A^T = A~^T + V U^T. Returns
    (lambda = dL/db, dL/dA values on A's pattern or None, iters list, report);
    report["rr"] = ||g - A^T lambda|| / ||g||."""
    L = load()
    lam = torch.empty(A.n, dtype=torch.float64, device=g.device)
    gv = torch.empty(A.nnz, dtype=torch.float64, device=g.device) if grad_vals else None
    prm = _stage(krylov, eps, maxit, restart, krylov_precision, inner_tol)
    cap = sp.s + 1
    iters = (C.c_int32 * cap)()
    rep = _SolveReport()
    v = A.view()
    st = _check("sai_backward", L.sai_backward(C.byref(v), sp._h, P._h, _p(x), _p(g.contiguous()), C.byref(prm),
                                               _p(lam), _p(gv), iters, cap, C.byref(rep), _stream()),
                allow=(SAI_MAXITER, SAI_BREAKDOWN))
    return lam, gv, list(iters[:cap]), _report(rep, st)


class SparseSolve(torch.autograd.Function):
    """x = A^{-1} b through Procedure * with gradients for A's stored values
    and for b. forward(col_ptr, row_idx, val, b, opts): opts is a dict of
    split / build / solve keywords (sai, delta, mn, max_aug, tol, tol_mode,
    lmax, krylov, eps, maxit, restart, thresh_mult, abs_tau)."""

    @staticmethod
    def forward(ctx, col_ptr, row_idx, val, b, opts):
        o = dict(opts)
        A = CscMatrix(b.numel(), col_ptr, row_idx, val.detach().contiguous())
        sp = split(A, thresh_mult=o.get("thresh_mult", 10.0), abs_tau=o.get("abs_tau", -1.0))
        if o.get("sai", "spai") == "spai":
            P = build_spai(sp, delta=o.get("delta", 0.4), mn=o.get("mn", 5), max_aug=o.get("max_aug", 10))
        else:
            P = build_psai(sp, delta=o.get("delta", 0.4), tol=o.get("tol", 0.0), tol_mode=o.get("tol_mode", 0),
                           lmax=o.get("lmax", 10))
        kw = dict(krylov=o.get("krylov", "bicgstab"), eps=o.get("eps", 1e-8), maxit=o.get("maxit", 500),
                  restart=o.get("restart", 50))
        x, _, rep = solve_with(A, sp, P, b.detach().contiguous(), **kw)
        ctx.state = (A, sp, P, kw)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        A, sp, P, kw = ctx.state
        lam, gv, _, _ = backward(A, sp, P, x, gx.contiguous(), grad_vals=ctx.needs_input_grad[2], **kw)
        return None, None, gv, lam, None


def solve_batched(As, bs, sai="spai", eps=1e-8, maxit=500, thresh_mult=10.0, abs_tau=-1.0, delta=0.4, mn=5,
                  max_aug=10, key_bits=20, tol=0.0, tol_mode=1, lmax=10, sai_precision=0, keep="nearest", lfill=0,
                  growth="A", c_adapt=0):
    """Procedure * for a batch of independent matrices (lists of CscMatrix and
    device b vectors): one SAI build over all their columns, one batched
    BiCGStab over all their s_i + 1 systems (one graph launch), SMW per matrix;
    c_adapt=1 continues the u_j systems of every matrix whose c exceeds 1.
    Returns (xs list, per-matrix list of dicts, batch report dict)."""
    L = load()
    nmat = len(As)
    views = (_CscView * nmat)(*[A.view() for A in As])
    xs = [torch.empty(A.n, dtype=torch.float64, device=b.device) for A, b in zip(As, bs)]
    bp = (C.c_void_p * nmat)(*[_p(b.contiguous()).value for b in bs])
    xp = (C.c_void_p * nmat)(*[_p(x).value for x in xs])
    prm = _batch_params(sai, eps, maxit, thresh_mult, abs_tau, delta, mn, max_aug, key_bits, tol, tol_mode, lmax,
                        sai_precision, keep, lfill, growth, c_adapt)
    items = (_BatchItem * nmat)()
    rep = _BatchReport()
    st = _check("sai_solve_batched", L.sai_solve_batched(nmat, views, bp, C.byref(prm), xp, items, C.byref(rep),
                                                         _stream()), allow=(SAI_MAXITER, SAI_BREAKDOWN))
    per = [dict(status=it.status, iter_max=it.iter_max, s=it.s, p=it.p, c=it.c, rr=it.rr, c_rounds=it.c_rounds)
           for it in items]
    report = {f: getattr(rep, f) for f, _ in _BatchReport._fields_}
    report["status"] = st
    return xs, per, report


def _batch_params(sai, eps, maxit, thresh_mult, abs_tau, delta, mn, max_aug, key_bits, tol, tol_mode, lmax,
                  sai_precision, keep, lfill, growth, c_adapt):
    return _SolveParams(_SplitParams(thresh_mult, abs_tau, 0, 0, _KEEP[keep], 0), 0 if sai == "spai" else 1,
                        _SpaiParams(delta, mn, max_aug, key_bits, sai_precision),
                        _PsaiParams(delta, tol, tol_mode, lmax, sai_precision, lfill, _GROWTH[growth], 0),
                        _KrylovParams(BICGSTAB, 50, maxit, 0, 0.0, 0), eps, int(c_adapt), 0)


def build_batched(As, sai="spai", thresh_mult=10.0, abs_tau=-1.0, delta=0.4, mn=5, max_aug=10, key_bits=20, tol=0.0,
                  tol_mode=1, lmax=10, sai_precision=0, keep="nearest", lfill=0, growth="A"):
    """The batch's SAI build alone: a Precond of the block-diagonal A~ of the
    batch (matrix m's rows and columns start at the sum of the earlier
    orders); its diagonal blocks are the M_i that solve_batched uses."""
    L = load()
    nmat = len(As)
    views = (_CscView * nmat)(*[A.view() for A in As])
    prm = _batch_params(sai, 1e-8, 500, thresh_mult, abs_tau, delta, mn, max_aug, key_bits, tol, tol_mode, lmax,
                        sai_precision, keep, lfill, growth, 0)
    h = C.c_void_p()
    _check("sai_build_batched", L.sai_build_batched(nmat, views, C.byref(prm), _stream(), C.byref(h)))
    return Precond(h.value)


def build_autotune_batched(As, sai="spai", thresh_mult=10.0, abs_tau=-1.0, delta=0.4, mn=5, max_aug=10, key_bits=20,
                           tol=0.0, tol_mode=1, lmax=10, sai_precision=0, keep="nearest", lfill=0, growth="A"):
    """The build-schedule autotuner on the batch's stacked A~; the fastest
    configuration becomes the process-wide one. Returns (chosen, candidates)."""
    L = load()
    nmat = len(As)
    views = (_CscView * nmat)(*[A.view() for A in As])
    prm = _batch_params(sai, 1e-8, 500, thresh_mult, abs_tau, delta, mn, max_aug, key_bits, tol, tol_mode, lmax,
                        sai_precision, keep, lfill, growth, 0)
    t = _BuildTuning()
    _check("sai_build_autotune_batched", L.sai_build_autotune_batched(nmat, views, C.byref(prm), _stream(),
                                                                      C.byref(t)))
    return _cfg_dict(t.chosen), [_cfg_dict(t.cand[i]) for i in range(t.ncand)]


def launch_count():
    """Kernel launches made by the library so far in this process."""
    return int(load().sai_launch_count())


def profile_begin():
    """Open a profile: per-site CUDA-event timing and algorithmic work counters."""
    _check("sai_profile_begin", load().sai_profile_begin())


def profile_end():
    """Close the profile; returns {"launches": L, "sites": {name: {launches, ms, bytes, flops}}}."""
    rep = _ProfReport()
    _check("sai_profile_end", load().sai_profile_end(C.byref(rep)))
    sites = {}
    for q in range(rep.nsites):
        st = rep.site[q]
        sites[st.name.decode()] = dict(launches=int(st.launches), timed=int(st.timed), ms=st.ms, bytes=st.bytes,
                                       flops=st.flops, flops32=st.flops32)
    return {"launches": int(rep.launches), "sites": sites}

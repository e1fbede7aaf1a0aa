"""The C-ABI library loads and exports every entry point declared in include/*.h
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(sai_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1211_6866_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sai_split_create", "sai_build_spai", "sai_build_psai", "sai_krylov_solve", "sai_smw_recover",
                 "sai_solve", "sai_rel_resid", "sai_solve_with", "sai_backward", "sai_solve_batched",
                 "sai_precond_create", "sai_dmperm", "sai_permute_rows"):
        assert must in names


def test_abi_structs_match_the_binding():
    """The binding's ctypes mirrors have the header's field order and sizes
    (the solve report, the split parameters and the method enum)."""
    import ctypes as C
    import paper_1211_6866_gb300 as sai
    hdr = open(os.path.join(ROOT, "include", "saismw.h")).read()
    assert "int32_t zero_diag;" in hdr and "int32_t moved;" in hdr
    assert [f for f, _ in sai._SplitParams._fields_] == ["thresh_mult", "abs_tau", "ge", "p_keep", "keep_rule",
                                                          "zero_diag"]
    assert C.sizeof(sai._SplitParams) == 32
    assert [f for f, _ in sai._SolveReport._fields_][-2:] == ["moved", "c_rounds"]
    assert [f for f, _ in sai._SolveParams._fields_][-3:] == ["eps", "c_adapt", "reserved"]
    assert "int32_t c_adapt;" in hdr and "int32_t c_rounds;" in hdr
    assert [f for f, _ in sai._BatchItem._fields_][-2:] == ["c_rounds", "reserved"]
    assert re.search(r"SAI_BGMRES\s*=\s*4", hdr) and sai.BGMRES == 4 and sai._METHOD["bgmres"] == 4
    # the build schedule: four int32 fields and the measured time; five tier counts
    assert "int32_t first_tier;" in hdr and "int32_t n_tier[6];" in hdr
    assert [f for f, _ in sai._BuildConfig._fields_] == ["warps_t0", "blocks_per_sm_t12", "heavy_first",
                                                         "first_tier", "ms"]
    assert C.sizeof(sai._BuildConfig) == 20 and C.sizeof(sai._BuildTuning) == 20 + 8 + 12 * 20
    assert C.sizeof(sai._PrecondInfo) == 56


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(libpath):
    lib = ctypes.CDLL(libpath)
    lib.sai_status_string.restype = ctypes.c_char_p
    assert lib.sai_status_string(0) == b"SAI_OK"
    assert lib.sai_status_string(4) == b"SAI_PATTERN_OVERFLOW"


def test_binding_fails_loudly_without_gpu(libpath):
    import torch
    import paper_1211_6866_gb300 as sai
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        sai._stream()

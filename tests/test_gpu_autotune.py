"""The build-schedule autotuner (sai_build_autotune / sai_build_set_config).

The schedule (warps per block of the shared-memory tiers, blocks per SM of
the global-memory tiers, heavy columns first in the work queue) must not
change M: every such configuration gives the same M bit for bit. The first
tier's shape (first_tier) sets the group size of the columns it finishes,
so only configurations with the same first_tier are compared bit for bit
here (tests/test_gpu_small_tier.py compares each with the oracle). The
tuner picks the fastest candidate it timed.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib, need_gpu, to_dev, to_scipy

pytestmark = pytest.mark.gpu


def _m(sai, sp_, kind, kw):
    P = sai.build_spai(sp_, **kw) if kind == "spai" else sai.build_psai(sp_, **kw)
    return to_scipy(P.arrays()[0]), P


def _same(a, b):
    assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices)
    assert np.array_equal(a.data, b.data)


@pytest.mark.parametrize("case", ["spai_2d", "spai_zipf", "psai_3d", "spai_3d_refined"])
def test_every_schedule_gives_the_same_m(case):
    need_gpu()
    sai = lib()
    if case == "spai_2d":
        A, kind, kw, split_kw = W.convdiff2d_irregular().A, "spai", dict(delta=0.4, mn=5, max_aug=10), {}
    elif case == "spai_zipf":  # uneven columns: the heavy-first queue reorders them
        A, kind, kw, split_kw = W.zipf_columns(n=2000).A, "spai", dict(delta=0.4, mn=5, max_aug=5), dict(abs_tau=200.0)
    elif case == "psai_3d":
        A, kind, kw, split_kw = (W.convdiff3d_irregular(m=16, s=3, density=0.2).A, "psai",
                                 dict(delta=0.3, tol=1e-3, tol_mode=1, lmax=10), {})
    else:
        A, kind, kw, split_kw = (W.convdiff3d_irregular(m=24, s=4, density=0.1).A, "spai",
                                 dict(delta=0.3, mn=5, max_aug=10, precision=1), {})
    sp_ = sai.split(to_dev(A), **split_kw)
    try:
        sai.build_set_config()
        ref, _ = _m(sai, sp_, kind, kw)
        for w, b, hf in ((4, 1, 0), (4, 4, 1), (8, 1, 1), (8, 4, 0)):
            sai.build_set_config(w, b, hf)
            got, _ = _m(sai, sp_, kind, kw)
            _same(got, ref)
    finally:
        sai.build_set_config()


def test_autotune_picks_the_fastest_candidate_and_keeps_m():
    """Ten candidates: the four first-tier forms x two block sizes (the lane
    form with one), then
    heavy_first and the global tiers' blocks per SM on the best; the chosen
    one is the fastest timed, and a build under it gives the bits of the same
    configuration set by hand (and the oracle's pattern)."""
    need_gpu()
    sai = lib()
    A = W.convdiff3d_irregular(m=32, s=4, density=0.1).A
    sp_ = sai.split(to_dev(A))
    kw = dict(delta=0.3, mn=5, max_aug=10)
    try:
        chosen, cands = sai.build_autotune(sp_, "spai", **kw)
        assert len(cands) == 10 and all(c["ms"] > 0 for c in cands)
        assert chosen["ms"] == min(c["ms"] for c in cands)
        assert {(c["first_tier"], c["warps_t0"]) for c in cands[:7]} == \
            {(f, w) for f in (0, 1, 2) for w in (4, 8)} | {(3, 8)}
        assert all((c["blocks_per_sm_t12"], c["heavy_first"]) == (2, 0) for c in cands[:7])
        assert cands[7]["heavy_first"] == 1 and {c["blocks_per_sm_t12"] for c in cands[8:]} == {1, 4}
        got, _ = _m(sai, sp_, "spai", kw)
        sai.build_set_config(chosen["warps_t0"], chosen["blocks_per_sm_t12"], chosen["heavy_first"],
                             chosen["first_tier"])
        ref, _ = _m(sai, sp_, "spai", kw)
        _same(got, ref)
    finally:
        sai.build_set_config()


def test_set_config_rejects_values_outside_the_candidates():
    need_gpu()
    sai = lib()
    for bad in ((16, 2, 0), (8, 3, 0), (8, 2, 2), (8, 2, 0, 4)):
        with pytest.raises(sai.SaiError) as e:
            sai.build_set_config(*bad)
        assert e.value.status == sai.SAI_INVALID_ARG
    sai.build_set_config()

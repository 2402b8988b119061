"""The checked build (device bounds checks, libbisp_checked.so) on the GPU: every check passes on
the parity cases, the outputs equal the release build's bit for bit, and a check that fails
(the self-test, which touches no memory) is recorded in the device word."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1803_02132_gb300 as bisp  # noqa: E402
from paper_1803_02132_gb300 import build as bisp_build  # noqa: E402
import synthcat  # noqa: E402
from test_gpu_parity import CASES, _assign, _survey  # noqa: E402


@pytest.fixture(scope="module")
def checked():
    bisp_build.build(checked=True)
    yield
    bisp.use_library(None)


def _run(case, nbins, estimator="bispectrum", los_object=3):
    """Outputs of one measurement of a parity case (nbins k-bins, or 5 r-bins for threept)."""
    c = CASES[case]
    N, L = c["N"], c["L"]
    kf = 2 * np.pi / L
    if estimator == "threept":
        edges = (L / N) * np.array([0.0, 0.5, 1.5, 2.05, 2.95, 4.1])
    else:
        edges = kf * np.linspace(1.0, 15.5, nbins + 1)
    if c["los"] == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        kw = dict(los="global")
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        kw = dict(los="local", observer=obs, fkp_P0=1e4, want_window=True, los_object=los_object)
    with bisp.Plan(N, L, edges, c["ells"], mas=c["mas"], interlace=c["interlace"], estimator=estimator, **kw) as plan:
        _assign(plan, 0, gal)
        if ran is not None:
            _assign(plan, 1, ran)
        return plan.measure()


@pytest.mark.parametrize("case,nbins,estimator,los_object", [
    ("survey_local", 25, "bispectrum", 3), ("survey_local", 7, "bispectrum", 1),
    ("box_tsc_ilv", 7, "bispectrum", 3), ("box_cic", 34, "bispectrum", 3), ("survey_local", 3, "threept", 3)])
def test_checked_build_passes_and_matches_release(checked, case, nbins, estimator, los_object):
    bisp.use_library(None)
    ref = _run(case, nbins, estimator, los_object)
    prev = bisp.use_checked_library()
    try:
        assert bisp.check_word(reset=True) >= 0
        out = _run(case, nbins, estimator, los_object)
        word = bisp.check_word(reset=True)
    finally:
        bisp.use_library(prev)
    assert word == 0, f"device check failed: site {word >> 32}, index {word & 0x7fffffff}"
    for k in ref:
        assert np.array_equal(out[k], ref[k]), k


def test_checked_build_records_a_failed_check(checked, monkeypatch):
    prev = bisp.use_checked_library()
    try:
        bisp.check_word(reset=True)
        monkeypatch.setenv("BISP_CHECK_SELFTEST", "1")
        with bisp.Plan(32, 1000.0, [0.02, 0.05], [(0, 0, 0)], los="global", mas="TSC") as plan:
            plan.assign(0, torch.rand(1000, 3, device="cuda") * 999.0)
        word = bisp.check_word(reset=True)
        assert bisp.check_word() == 0
    finally:
        bisp.use_library(prev)
    assert word >> 32 == 99 and word & (1 << 31)


def test_release_build_reports_unsupported():
    bisp.use_library(None)
    with pytest.raises(bisp.BispError) as e:
        bisp.check_word()
    assert e.value.status == bisp.BISP_EUNSUPPORTED

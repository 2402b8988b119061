"""Failure paths, made on purpose without faulting the GPU: injected allocation failures (the
k-th device allocation of a call fails as a cudaMalloc failure would) and bounded device waits
that run out because the copies they wait for are never started.  Each failing call returns its
status and message, and the plan stays usable and destroyable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1803_02132_gb300 as bisp  # noqa: E402
import synthcat  # noqa: E402

N, L = 32, 1000.0
EDGES = 2 * np.pi / L * np.array([1.0, 2.5, 4.0, 5.5, 7.0])
ELLS = [(0, 0, 0), (2, 0, 2)]


def _plan():
    return bisp.Plan(N, L, EDGES, ELLS, los="global", mas="TSC", interlace=True)


def _cat():
    return torch.from_numpy(synthcat.periodic_catalog(N, L, 20_000, seed=41)).cuda()


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("B", "shot", "nmodes"))


def test_injected_allocation_failures(monkeypatch):
    """Plan creation, a first assignment and a first measurement (the calls that allocate), with
    each of their device allocations failing in turn on a fresh plan: the call returns
    BISP_ENOMEM naming the bytes, and the plan then assigns and measures exactly as one that saw
    no failure; a steady-state measurement allocates nothing."""
    monkeypatch.delenv("BISP_FAIL_ALLOC", raising=False)
    xyz = _cat()
    with _plan() as p:
        p.assign(bisp.DATA, xyz)
        ref = p.measure()
        monkeypatch.setenv("BISP_FAIL_ALLOC", "1")  # nothing left to allocate
        assert _same(p.measure(), ref)
        monkeypatch.delenv("BISP_FAIL_ALLOC")
    monkeypatch.setenv("BISP_FAIL_ALLOC", "1")
    with pytest.raises(bisp.BispError) as e:
        _plan()
    assert e.value.status == bisp.BISP_ENOMEM and "GB failed" in str(e.value)
    monkeypatch.delenv("BISP_FAIL_ALLOC")
    for call in ("assign", "measure"):
        for k in range(1, 64):
            with _plan() as p:
                if call == "measure":
                    p.assign(bisp.DATA, xyz)
                monkeypatch.setenv("BISP_FAIL_ALLOC", str(k))
                try:
                    p.assign(bisp.DATA, xyz) if call == "assign" else p.measure()
                    failed = False
                except bisp.BispError as err:
                    assert err.status == bisp.BISP_ENOMEM, str(err)
                    assert "injected" in str(err)
                    failed = True
                monkeypatch.delenv("BISP_FAIL_ALLOC")
                if call == "assign":
                    if failed:
                        with pytest.raises(bisp.BispError) as e2:  # the catalogue is left unassigned
                            p.measure()
                        assert e2.value.status == bisp.BISP_ESTATE
                        p.assign(bisp.DATA, xyz)
                assert _same(p.measure(), ref), (call, k)
            if not failed:
                break
        assert k > 1, f"{call}: no allocation was made"


@pytest.mark.parametrize("kernel", ["pair", "zpass"])
def test_bounded_waits_report_timeout(kernel, monkeypatch):
    """The staged copies of the contraction (TMA tensor copies) or of the inverse z pass (bulk row
    copies) are not started in the first such launch of the call: the waits run out after their
    2 s limit, the kernel returns, and bisp_measure reports BISP_ETIMEOUT; the next measurement
    is exact again."""
    monkeypatch.delenv("BISP_INJECT_STALL", raising=False)
    monkeypatch.delenv("BISP_PAIR_FP32", raising=False)
    monkeypatch.delenv("BISP_PAIR_KERNEL", raising=False)
    with _plan() as p:
        p.assign(bisp.DATA, _cat())
        ref = p.measure()
        monkeypatch.setenv("BISP_INJECT_STALL", kernel)
        with pytest.raises(bisp.BispError) as e:
            p.measure()
        assert e.value.status == bisp.BISP_ETIMEOUT, str(e.value)
        monkeypatch.delenv("BISP_INJECT_STALL")
        assert _same(p.measure(), ref)
        torch.cuda.synchronize()  # the context is still usable

"""bisp_cell_order_noalloc, the cell ordering for callers that cannot allocate device
memory (for example inside a framework step or memory pool that forbids cudaMalloc), must
give the same result as bisp_cell_order, the entry point that allocates its own scratch,
and as the oracle's stable sort by home node.  Both entry points are called through the C
ABI; the comparison is exact because the output is integer keys and a permutation.  Calls
in a row check that the shared static scratch carries no state from one call to the next;
the largest accepted catalogue exercises the top of the scratch layout."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1803_02132_gb300 as bisp  # noqa: E402
from oracle import estimator as E  # noqa: E402

NMAX = 1 << 20  # BISP_NOALLOC_MAX_PARTICLES


def _call(fn, nmesh, box, mas, xyz, keys, order):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(nmesh, box, mas, C.c_void_p(xyz.data_ptr()), xyz.shape[0], C.c_void_p(keys.data_ptr()),
            C.c_void_p(order.data_ptr()), stream)
    assert st == bisp.BISP_OK, bisp.lib().bisp_last_error().decode()
    torch.cuda.synchronize()
    return keys.cpu().numpy().copy(), order.cpu().numpy().copy()


def _order(fn, nmesh, box, mas, xyz):
    n = xyz.shape[0]
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    return _call(fn, nmesh, box, mas, xyz, keys, order)


def _catalogue(rng, n, box):
    xyz = (rng.random((n, 3)) * box).astype(np.float32)
    xyz[: n // 10] = xyz[n // 10: 2 * (n // 10)]  # repeated positions: ties keep input order
    return xyz


def test_noalloc_matches_allocating_entry_point_twice():
    lib = bisp.lib()
    rng = np.random.default_rng(2024)
    for call, (n, nmesh, mas) in enumerate([(300_000, 128, 3), (1_000_000, 256, 2)]):
        box = 1000.0
        xyz = _catalogue(rng, n, box)
        xd = torch.from_numpy(xyz).cuda()
        k_ref, o_ref = _order(lib.bisp_cell_order, nmesh, box, mas, xd)
        k_na, o_na = _order(lib.bisp_cell_order_noalloc, nmesh, box, mas, xd)
        assert np.array_equal(k_na, k_ref), f"call {call}: keys differ"
        assert np.array_equal(o_na, o_ref), f"call {call}: order differs"
        if call == 0:  # and against the oracle's stable sort by home node
            ok = E.cell_keys(xyz, nmesh, box, mas)
            oo = np.argsort(ok, kind="stable")
            assert np.array_equal(o_na.astype(np.int64), oo)
            assert np.array_equal(k_na.astype(np.int64), ok[oo])


def test_noalloc_at_its_limit_allocates_nothing():
    """n == BISP_NOALLOC_MAX_PARTICLES on a 256^3 mesh (the top of the scratch layout), twice;
    after a warm-up call the free device memory does not change across a call."""
    lib = bisp.lib()
    rng = np.random.default_rng(77)
    box = 2000.0
    xyz = _catalogue(rng, NMAX, box)
    xd = torch.from_numpy(xyz).cuda()
    k_ref, o_ref = _order(lib.bisp_cell_order, 256, box, 3, xd)
    keys = torch.empty(NMAX, dtype=torch.int32, device="cuda")
    order = torch.empty(NMAX, dtype=torch.int32, device="cuda")
    _call(lib.bisp_cell_order_noalloc, 256, box, 3, xd, keys, order)  # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.bisp_cell_order_noalloc(256, box, 3, C.c_void_p(xd.data_ptr()), NMAX, C.c_void_p(keys.data_ptr()),
                                     C.c_void_p(order.data_ptr()), stream)
    assert st == bisp.BISP_OK, lib.bisp_last_error().decode()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    assert np.array_equal(keys.cpu().numpy(), k_ref)
    assert np.array_equal(order.cpu().numpy(), o_ref)


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = bisp.lib()
    n = NMAX + 1
    xd = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.bisp_cell_order_noalloc(64, 100.0, 3, C.c_void_p(xd.data_ptr()), n, C.c_void_p(keys.data_ptr()),
                                     C.c_void_p(keys.data_ptr()), None)
    assert st == bisp.BISP_EINVAL
    assert "no-allocation limit" in lib.bisp_last_error().decode()

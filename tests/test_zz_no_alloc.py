"""bisp_cell_order_noalloc, the cell ordering for callers that cannot allocate device
memory (for example inside a framework step that forbids cudaMalloc), must give the same
result as bisp_cell_order, the entry point that allocates its own scratch.  Both are
called through the C ABI; the comparison is exact because the output is integer keys and
a permutation.  Two calls in a row check that the shared static scratch carries no state
from one call to the next."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1803_02132_gb300 as bisp  # noqa: E402


def _order(fn, nmesh, box, mas, xyz):
    n = xyz.shape[0]
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    order = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(nmesh, box, mas, C.c_void_p(xyz.data_ptr()), n, C.c_void_p(keys.data_ptr()),
            C.c_void_p(order.data_ptr()), stream)
    assert st == bisp.BISP_OK, bisp.lib().bisp_last_error().decode()
    torch.cuda.synchronize()
    return keys.cpu().numpy(), order.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    lib = bisp.lib()
    rng = np.random.default_rng(2024)
    for call, (n, nmesh, mas) in enumerate([(300_000, 128, 3), (1_000_000, 256, 2)]):
        box = 1000.0
        xyz = (rng.random((n, 3)) * box).astype(np.float32)
        xyz[: n // 10] = xyz[n // 10: 2 * (n // 10)]  # repeated positions: ties keep input order
        xd = torch.from_numpy(xyz).cuda()
        k_ref, o_ref = _order(lib.bisp_cell_order, nmesh, box, mas, xd)
        k_na, o_na = _order(lib.bisp_cell_order_noalloc, nmesh, box, mas, xd)
        assert np.array_equal(k_na, k_ref), f"call {call}: keys differ"
        assert np.array_equal(o_na, o_ref), f"call {call}: order differs"


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = bisp.lib()
    n = (1 << 20) + 1
    xd = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.bisp_cell_order_noalloc(64, 100.0, 3, C.c_void_p(xd.data_ptr()), n, C.c_void_p(keys.data_ptr()),
                                     C.c_void_p(keys.data_ptr()), None)
    assert st == bisp.BISP_EINVAL
    assert "no-allocation limit" in lib.bisp_last_error().decode()

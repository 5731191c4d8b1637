"""The allocation-free self-block entry point matches the allocating one.

pm_self_block_noalloc serves callers that cannot let the library call
cudaMalloc / cudaFree (those calls may synchronise the device under work the
caller has in flight, or the caller manages a fixed device-memory budget
itself).  Its scratch lives in a static device array, so this test calls it
twice in a row through the C ABI, on different inclusions, and compares each
result with pm_self_block.  The file sorts last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2603_09381_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_self_block_matches_allocating_entry_point():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_09381_gb300 import pmchwt as pm
    prob = wl.star_grid(2, 1, n=128, seed=3)
    prob["inclusions"][1] = wl._inclusion(wl.SHAPE_ELLIPSE, 1.0, 0.0, 0.4, [0.42, 0.25], 96, 12.0)
    g = pm.Geometry(prob)
    for j in (0, 1, 0):   # two calls in a row on different blocks, then the first again
        n = prob["inclusions"][j]["n"]
        ref = g.self_block(j, n)
        buf = torch.full((2 * n, 2 * n), complex("nan"), dtype=torch.complex128, device="cuda")
        g.self_block_noalloc(j, buf.data_ptr())
        torch.cuda.synchronize()
        got = buf.cpu().numpy().T        # column-major on the device
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_noalloc_rejects_blocks_above_the_scratch_limit():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_09381_gb300 import pmchwt as pm
    prob = wl.circle_grid(1, 1, n=258)
    g = pm.Geometry(prob)
    # a buffer of the full block size, so that a regression of the size check
    # would still write inside it
    buf = torch.zeros((2 * 258, 2 * 258), dtype=torch.complex128, device="cuda")
    with pytest.raises(pm.PmError) as e:
        g.self_block_noalloc(0, buf.data_ptr())
    assert e.value.status == 1 and "256" in str(e.value)
    torch.cuda.synchronize()
    assert not bool(torch.any(buf != 0))


def test_noalloc_rejects_host_memory_and_bad_indices():
    """A host buffer (the allocating sibling takes one, so the two are easy to
    mix up) is refused before any launch, as is an inclusion index out of range."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_09381_gb300 import pmchwt as pm
    prob = wl.circle_grid(2, 1, n=64)
    g = pm.Geometry(prob)
    host = np.zeros((128, 128), dtype=np.complex128)
    with pytest.raises(pm.PmError) as e:
        g.self_block_noalloc(0, host.ctypes.data)
    assert e.value.status == 1 and "device memory" in str(e.value)
    assert not np.any(host != 0)
    buf = torch.zeros((128, 128), dtype=torch.complex128, device="cuda")
    for j in (-1, 2):
        with pytest.raises(pm.PmError) as e:
            g.self_block_noalloc(j, buf.data_ptr())
        assert e.value.status == 1

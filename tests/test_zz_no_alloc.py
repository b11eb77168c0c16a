"""The allocation-free CSR pattern entry point (lfem_pattern_csr_noalloc).

It serves callers that cannot allocate device memory while they run (their
arena or pool owns the device, or their loop forbids cudaMalloc after
start-up): its scratch is an array inside the library.  Its output must equal
lfem_pattern's CSR arrays exactly (integer work: bit-exact), on two calls in a
row, since every call reuses the same array.  This file runs last so a failure
here leaves every other result already reported.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14035_gb300 import lfem as m

    return m


def _meshes():
    from paper_2605_14035_gb300.inputs import meshes

    yield "sphere_p2", *meshes.icosphere(4, 2), 2, 2
    yield "cube_p2", *meshes.kuhn_cube_p2(3), 3, 2
    x, e = meshes.closed_curve_p2(500, seed=2)
    yield "curve_p2", x, e, 1, 2
    yield "sphere_p1_unused_nodes", meshes.icosphere(3, 1)[0], meshes.icosphere(3, 1)[1][:900], 2, 1


@pytest.mark.parametrize("case", list(_meshes()), ids=lambda c: c[0])
def test_noalloc_matches_pattern_twice(case, lfem):
    name, x, e, dim, order = case
    ed = torch.from_numpy(np.ascontiguousarray(e)).cuda()
    n = x.shape[0]
    ref_rp, ref_ci = lfem.Pattern(ed, n, dim, order).csr()
    lib = lfem.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # the second call reuses (and must clear) the same scratch
        rp = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda")
        ci = torch.full((ref_ci.numel() + 5,), -7, dtype=torch.int32, device="cuda")
        nnz = ctypes.c_int64(-1)
        rc = lib.lfem_pattern_csr_noalloc(ctypes.c_void_p(ed.data_ptr()), e.shape[0], n, dim, order,
                                          ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()),
                                          ci.numel(), ctypes.byref(nnz), stream)
        assert rc == 0, lib.lfem_last_error()
        assert nnz.value == ref_ci.numel()
        assert torch.equal(rp, ref_rp)
        assert torch.equal(ci[: nnz.value], ref_ci)
        assert torch.all(ci[nnz.value:] == -7)  # nothing written past nnz


def test_noalloc_limits(lfem):
    from paper_2605_14035_gb300.inputs import meshes

    x, e = meshes.icosphere(6, 2)  # needs more words than the static array holds
    ed = torch.from_numpy(e).cuda()
    rp = torch.zeros(x.shape[0] + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(lfem.LfemError) as ei:
        lfem.pattern_csr_noalloc(ed, x.shape[0], 2, 2, rp, ci)
    assert ei.value.code == 4
    # too small a column buffer: nnz is reported, error raised
    x, e = meshes.icosphere(2, 2)
    ed = torch.from_numpy(e).cuda()
    rp = torch.zeros(x.shape[0] + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(lfem.LfemError) as ei:
        lfem.pattern_csr_noalloc(ed, x.shape[0], 2, 2, rp, ci)
    assert ei.value.code == 4
    # a node index out of range is reported, not read
    bad = torch.tensor([[0, 1, 99]], dtype=torch.int32, device="cuda")
    with pytest.raises(lfem.LfemError) as ei:
        lfem.pattern_csr_noalloc(bad, 10, 2, 1, rp, ci)
    assert ei.value.code == 2


def test_noalloc_takes_no_device_memory(lfem):
    """After the first call (which looks the array up), further calls make no
    device allocation (the library's own allocation counter does not move) and
    leave the device's free memory unchanged although they need megabytes of
    scratch.  The counter is the primary check: free memory is device-wide and
    only a secondary one."""
    from paper_2605_14035_gb300.inputs import meshes

    x, e = meshes.icosphere(5, 2)  # about 4.6 MB of scratch
    ed = torch.from_numpy(e).cuda()
    rp = torch.zeros(x.shape[0] + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(40 * e.shape[0], dtype=torch.int32, device="cuda")
    lfem.pattern_csr_noalloc(ed, x.shape[0], 2, 2, rp, ci)
    torch.cuda.synchronize()
    lib = lfem.lib()
    n0 = lib.lfem_debug_alloc_count()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        lfem.pattern_csr_noalloc(ed, x.shape[0], 2, 2, rp, ci)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert lib.lfem_debug_alloc_count() == n0
    # the counter itself works: building a pattern allocates
    lfem.Pattern(ed, x.shape[0], 2, 2)
    assert lib.lfem_debug_alloc_count() > n0
    assert free1 == free0

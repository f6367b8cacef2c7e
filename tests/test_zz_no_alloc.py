"""The allocation-free Kronecker apply (phikron_kron_apply_f64_noalloc) against the
allocating one (phikron_kron_apply_f64), through the C ABI.

The no-alloc variant exists for callers that cannot allocate device memory when they call
in (a host that owns all device memory through its own pool, or a latency-critical loop
that cannot afford cudaMalloc's implicit synchronisation); it keeps its intermediate in a
built-in device array instead of a caller-provided work buffer.  Two calls in a row must
both agree with the allocating entry point (the built-in array keeps the previous call's
contents, which must not leak into the next result).  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    from paper_2211_00696_gb300 import phikron as B
    return B.lib(), B


def _ptrs(mats):
    return (C.c_void_p * len(mats))(*[m.data_ptr() for m in mats])


@pytest.mark.parametrize("shape", [(16, 24, 40), (128, 96), (64, 64, 64)])
def test_noalloc_matches_allocating_entry_point_twice(shape):
    L, B = _lib()
    rng = np.random.default_rng(17)
    dims = len(shape)
    ns = (C.c_int * dims)(*shape)
    N = int(np.prod(shape))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        mats = [torch.from_numpy(rng.standard_normal((n, n)) / n).cuda() for n in shape]
        v = torch.from_numpy(rng.standard_normal(N)).cuda()
        ref = torch.empty_like(v)
        work = torch.empty_like(v)
        rc = L.phikron_kron_apply_f64(dims, ns, _ptrs(mats), v.data_ptr(), ref.data_ptr(), work.data_ptr(), stream)
        assert rc == 0, L.phikron_last_error()
        out = torch.full_like(v, float("nan"))
        rc = L.phikron_kron_apply_f64_noalloc(dims, ns, _ptrs(mats), v.data_ptr(), out.data_ptr(), stream)
        assert rc == 0, L.phikron_last_error()
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.max(np.abs(o - r)) <= 1e-12 * np.max(np.abs(r)), call


def test_noalloc_call_after_the_first_takes_no_device_memory():
    """After a first call on the device (which may load the library's kernels and place its
    built-in array), a call leaves the device's free memory unchanged: it allocates nothing."""
    L, B = _lib()
    shape = (32, 48, 40)
    ns = (C.c_int * 3)(*shape)
    N = int(np.prod(shape))
    rng = np.random.default_rng(5)
    mats = [torch.from_numpy(rng.standard_normal((n, n)) / n).cuda() for n in shape]
    v = torch.from_numpy(rng.standard_normal(N)).cuda()
    out = torch.empty_like(v)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.phikron_kron_apply_f64_noalloc(3, ns, _ptrs(mats), v.data_ptr(), out.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    first = out.clone()
    free_before = torch.cuda.mem_get_info()[0]
    rc = L.phikron_kron_apply_f64_noalloc(3, ns, _ptrs(mats), v.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert rc == 0, L.phikron_last_error()
    assert free_after == free_before, (free_before, free_after)
    assert torch.equal(out, first)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L, B = _lib()
    cap = L.phikron_noalloc_max_elements()
    assert cap == 1 << 20
    shape = (128, 128, 128)   # 2,097,152 > capacity
    ns = (C.c_int * 3)(*shape)
    mats = [torch.eye(128, dtype=torch.float64, device="cuda") for _ in range(3)]
    v = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = L.phikron_kron_apply_f64_noalloc(3, ns, _ptrs(mats), v.data_ptr(), v.data_ptr(), None)
    assert rc == B.EINVAL
    assert b"exceeds" in L.phikron_last_error()

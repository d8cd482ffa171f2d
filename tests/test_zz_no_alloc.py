"""The allocation-free FP64 inverse against the allocating one.

rgf_inverse_f64_noalloc serves callers that cannot allocate device memory:
its workspace is a fixed array inside the library.  This file runs last so
that a failure here leaves every other test already run; it also passes on
its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    r.lib()
    return r


def test_noalloc_inverse_matches_allocating_entry_point(rgf):
    import torch
    rng = np.random.default_rng(2024)
    stream = torch.cuda.Stream()
    for call in range(2):  # two calls in a row share the scratch array
        batch, b = (7, 96) if call == 0 else (5, 130)
        A = (rng.standard_normal((batch, b, b)) + 1j * rng.standard_normal((batch, b, b))) / np.sqrt(2)
        A += 2.0 * np.eye(b)
        A[1, 0, 0] = 0.0  # needs a row interchange
        X_ref, f_ref = rgf.rgf_kernel_inverse_f64(A)
        Ad = torch.tensor(A, dtype=torch.complex128, device="cuda")
        fd = torch.full((batch,), 7, dtype=torch.int32, device="cuda")  # cleared by the call
        rgf.rgf_inverse_f64_noalloc(Ad, fd, stream.cuda_stream)
        stream.synchronize()
        X = Ad.cpu().numpy()
        assert np.array_equal(fd.cpu().numpy(), f_ref)
        assert np.allclose(X, X_ref, rtol=0, atol=1e-12 * np.abs(X_ref).max())
        assert np.abs(np.einsum("nij,njk->nik", X, A) - np.eye(b)).max() < 1e-10


def test_noalloc_inverse_rejects_oversized_batch(rgf):
    import torch
    limit = rgf.rgf_inverse_f64_noalloc_limit()
    assert limit == 16 << 20
    b = 256
    per = 2 * b * 32 * 16 + b * 4
    batch = limit // per + 1
    L = rgf.lib()
    dummy = torch.zeros(1, dtype=torch.complex128, device="cuda")
    st = L.rgf_inverse_f64_noalloc(batch, b, ctypes.c_void_p(dummy.data_ptr()), None, None)
    assert st == rgf.RGF_E_INVALID
    assert "scratch" in rgf.rgf_last_error()


def test_noalloc_wrapper_checks_shapes_and_devices(rgf):
    """The binding refuses what would make the library write past a buffer:
    a non-square or non-3-D A and a flags tensor shorter than the batch."""
    import torch
    A = torch.zeros((2, 8, 6), dtype=torch.complex128, device="cuda")
    with pytest.raises(TypeError):
        rgf.rgf_inverse_f64_noalloc(A)
    A = torch.eye(8, dtype=torch.complex128, device="cuda").repeat(3, 1, 1).contiguous()
    with pytest.raises(ValueError):
        rgf.rgf_inverse_f64_noalloc(A, torch.zeros(2, dtype=torch.int32, device="cuda"))
    with pytest.raises(TypeError):
        rgf.rgf_inverse_f64_noalloc(A.reshape(24, 8))


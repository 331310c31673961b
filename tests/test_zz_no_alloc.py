"""The allocation-free batched LU entry point (for callers that cannot allocate
device memory, e.g. inside a pool that forbids new allocations) gives the same
factors, pivots and singularity count as the workspace entry point, on two calls
in a row (the shared built-in scratch is cleared between calls).  This file is
collected last so a failure here comes after every other test has run."""
import numpy as np
import pytest

from gpu_util import need_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [("complex128", 1e-12), ("complex64", 2e-5)])
def test_noalloc_lu_matches_workspace_lu_twice(dtype, tol):
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    rng = np.random.default_rng(2024)
    batch, m, ncols, npiv = 5, 150, 190, 120
    first = rng.standard_normal((batch, m, ncols)) + 1j * rng.standard_normal((batch, m, ncols))
    first[3, :, :] = 1.0                           # rank one: reported as singular
    second = rng.standard_normal((batch, m, ncols)) + 1j * rng.standard_normal((batch, m, ncols))
    for A, expect_singular in ((first, 1), (second, 0)):
        ref = torch.tensor(A.astype(dtype), device="cuda")
        got = ref.clone()
        ipiv_ref, ns_ref = api.fsi_batched_lu(ref, npiv)
        ipiv_got, ns_got = api.fsi_batched_lu_noalloc(got, npiv)
        torch.cuda.synchronize()
        assert ns_ref == expect_singular and ns_got == expect_singular
        assert torch.equal(ipiv_ref, ipiv_got)
        r = ref.cpu().numpy()
        g = got.cpu().numpy()
        assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r)


def test_noalloc_lu_rejects_batches_beyond_its_scratch():
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    A = torch.zeros((4096, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(RuntimeError, match="4095"):
        api.fsi_batched_lu_noalloc(A, 2)

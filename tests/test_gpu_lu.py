"""Batched partial LU with partial pivoting (the factorisation kernels behind every
solve) against its definition: P A = L U with |L| <= 1, and the Schur complement of
the eliminated block.  Sizes span several panels and tiles with ragged tails."""
import numpy as np
import pytest

from gpu_util import need_cuda

pytestmark = pytest.mark.gpu


def _apply_ipiv(A, ipiv):
    A = A.copy()
    for j, p in enumerate(ipiv):
        if p != j:
            A[[j, p]] = A[[p, j]]
    return A


@pytest.mark.parametrize("dtype,tol,tc", [("complex128", 1e-12, False), ("complex64", 2e-5, False),
                                           ("complex64", 2e-5, "bf16x6"), ("complex64", 2e-2, "bf16")])
@pytest.mark.parametrize("batch,m,ncols,npiv", [(3, 70, 70, 70), (2, 200, 300, 100), (4, 333, 401, 131),
                                                (1, 1, 1, 1), (2, 130, 130, 65), (2, 300, 650, 200),
                                                (32, 300, 650, 200)])
def test_batched_partial_lu(dtype, tol, tc, batch, m, ncols, npiv):
    """tc: the long trailing updates run on the tcgen05 tensor cores, with three BF16 planes per
    operand (FP32 accuracy) or one (plain BF16 products, FP32 accumulation).  Batches of 32 and
    more factor each outer panel recursively (outer panels of 128 and a ragged 72 columns here),
    smaller ones right-looking over panels."""
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    rng = np.random.default_rng(m * 7 + ncols)
    A = rng.standard_normal((batch, m, ncols)) + 1j * rng.standard_normal((batch, m, ncols))
    At = torch.tensor(A.astype(dtype), device="cuda")
    ipiv, nsing = api.fsi_batched_lu(At, npiv, tensor_cores=tc)
    torch.cuda.synchronize()
    assert nsing == 0
    R = At.cpu().numpy().astype(np.complex128)
    piv = ipiv.cpu().numpy()
    for b in range(batch):
        PA = _apply_ipiv(A[b], piv[b])
        L = np.tril(R[b][:, :npiv], -1)[:, :npiv]
        L[np.arange(npiv), np.arange(npiv)] = 1.0
        U = np.triu(R[b][:npiv, :])
        assert np.abs(L).max() <= 1.0 + 1e-6          # partial pivoting bound
        S = np.zeros_like(PA)
        S[npiv:, npiv:] = R[b][npiv:, npiv:]           # Schur complement block
        recon = L @ U + S
        err = np.linalg.norm(recon - PA) / np.linalg.norm(A[b])
        print(f"lu {dtype} tc={tc} m={m} n={ncols} k={npiv}: |PA-LU|/|A| = {err:.2e}")
        assert err <= tol * np.sqrt(m)


def test_singular_matrix_is_reported():
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    A = np.zeros((2, 40, 40), np.complex128)
    A[0] = np.eye(40)
    A[1, :, :] = 1.0          # rank one: zero pivot in column 1
    At = torch.tensor(A, device="cuda")
    ipiv, nsing = api.fsi_batched_lu(At, 40)
    assert nsing == 1


def _lu_residual(A, R, piv, npiv):
    PA = _apply_ipiv(A, piv)
    L = np.tril(R[:, :npiv], -1)
    L[np.arange(npiv), np.arange(npiv)] = 1.0
    U = np.triu(R[:npiv, :])
    S = np.zeros_like(PA)
    S[npiv:, npiv:] = R[npiv:, npiv:]
    return np.linalg.norm(L @ U + S - PA) / np.linalg.norm(A)


def test_tensor_core_updates_on_a_slab_window():
    """A config-2 slab window (2b x 3b, b = 852, b pivots): every trailing update of the lazy
    order (K = 128 panel updates, the left-looking solve of U12 with K up to 724, the Schur
    update with K = 852) on the tcgen05 path; |PA - LU| at FP32 level, like the SIMT factor."""
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    b = 852
    rng = np.random.default_rng(852)
    A = rng.standard_normal((2, 2 * b, 3 * b)) + 1j * rng.standard_normal((2, 2 * b, 3 * b))
    errs = {}
    for tc in (False, "bf16x6"):
        At = torch.tensor(A.astype(np.complex64), device="cuda")
        ipiv, nsing = api.fsi_batched_lu(At, b, tensor_cores=tc)
        torch.cuda.synchronize()
        assert nsing == 0
        R = At.cpu().numpy().astype(np.complex128)
        piv = ipiv.cpu().numpy()
        errs[tc] = max(_lu_residual(A[i], R[i], piv[i], b) for i in range(2))
    print("slab window |PA-LU|/|A|: simt %.2e  tcgen05 bf16x6 %.2e" % (errs[False], errs["bf16x6"]))
    assert errs[False] <= 2e-5 * np.sqrt(2 * b)
    assert errs["bf16x6"] <= 1.5 * errs[False]


def test_tensor_core_wait_timeout_is_reported_and_the_next_call_is_clean():
    """With a spin limit of one poll the bounded mbarrier waits of the tensor-core update give
    up: the call returns FSI_ETIMEOUT after the kernel has waited for the loads and MMAs it had
    issued and freed its tensor memory; with the default limit the next call factors correctly."""
    torch = need_cuda()
    from paper_2310_04734_gb300 import api
    rng = np.random.default_rng(5)
    m, ncols, npiv = 600, 900, 300
    A = rng.standard_normal((2, m, ncols)) + 1j * rng.standard_normal((2, m, ncols))
    At = torch.tensor(A.astype(np.complex64), device="cuda")
    api.fsi_set_wait_limit(1)
    try:
        with pytest.raises(RuntimeError, match="timed out"):
            api.fsi_batched_lu(At, npiv, tensor_cores=True)
    finally:
        api.fsi_set_wait_limit(0)
    At = torch.tensor(A.astype(np.complex64), device="cuda")
    ipiv, nsing = api.fsi_batched_lu(At, npiv, tensor_cores=True)
    torch.cuda.synchronize()
    assert nsing == 0
    R = At.cpu().numpy().astype(np.complex128)
    piv = ipiv.cpu().numpy()
    assert max(_lu_residual(A[i], R[i], piv[i], npiv) for i in range(2)) <= 2e-5 * np.sqrt(m)


def test_throughput_probes_report_plausible_rates():
    """The roofline denominators: every probe returns a positive rate below twice the nominal
    dense peak of its unit (FP32 80, FP64 1.25, BF16 2250, TF32 1125 TFLOP/s), and the 128 x 128
    BF16 shape of the LU updates does not exceed the 128 x 256 one by more than timing noise."""
    need_cuda()
    from paper_2310_04734_gb300 import api
    nominal = {"fp32_fma": 80.0, "fp64_fma": 1.25, "bf16_tcgen05": 2250.0, "tf32_tcgen05": 1125.0,
               "bf16_tcgen05_n128": 2250.0}
    got = {k: api.fsi_probe_peak(k, 0.05)[0] for k in api.PEAK_KINDS}
    for k, v in got.items():
        assert 0.0 < v < 2.0 * nominal[k], (k, v)
    assert got["bf16_tcgen05_n128"] <= 1.1 * got["bf16_tcgen05"]

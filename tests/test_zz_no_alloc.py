"""The allocation-free tensor-core GEMM entry point (xtrg_tc_gemm_static).

Some callers cannot hand this library a device workspace (a host framework
that owns all device memory, code running where cudaMalloc is not allowed).
xtrg_tc_gemm_static serves them from a fixed device array inside the
library.  This test calls it through the C ABI twice in a row, on different
shapes, and checks each result against xtrg_tc_gemm (the workspace variant)
within the tolerance the tensor-core GEMM tests use, and checks that a size
beyond the fixed array is refused.  The file is named so that pytest collects
it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# bound on |C - C_ref| relative to (|A| |B|^T), as in test_gpu_tc_gemm
TOL = {1: 2e-2, 3: 1e-4, 6: 2e-6}


@pytest.fixture(scope="module")
def torch_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_00142_gb300.build import build
    build()
    from paper_1801_00142_gb300 import _lib
    return torch, _lib


def _inputs(torch, M, N, K, batch, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((batch, M, K))
    B = rng.standard_normal((batch, N, K))
    return A, B, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()


def _with_workspace(torch, lib, dA, dB, M, N, K, batch, planes, nprod, splitk):
    dC = torch.zeros((batch, M, N), dtype=torch.float64, device="cuda")
    nbytes = lib.xtrg_tc_gemm_workspace_bytes(M, N, K, batch, planes, splitk)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    p = (ws.data_ptr() + 255) // 256 * 256
    lib.xtrg_tc_gemm(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), M, N, K, batch, planes, nprod,
                     splitk, p, nbytes, torch.cuda.current_stream().cuda_stream)
    return dC.cpu().numpy()


def test_static_scratch_matches_workspace_variant_twice(torch_lib):
    torch, lib = torch_lib
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(200, 130, 100, 3, 3, 6, 1, 11), (256, 512, 1024, 1, 3, 6, 4, 12)]
    for M, N, K, batch, planes, nprod, splitk, seed in cases:
        A, B, dA, dB = _inputs(torch, M, N, K, batch, seed)
        dC = torch.full((batch, M, N), float("nan"), dtype=torch.float64, device="cuda")
        s = lib.xtrg_tc_gemm_static(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), M, N, K, batch,
                                    planes, nprod, splitk, stream)
        assert s == lib.XTRG_OK, s
        got = dC.cpu().numpy()
        ref = _with_workspace(torch, lib, dA, dB, M, N, K, batch, planes, nprod, splitk)
        scale = np.einsum("bmk,bnk->bmn", np.abs(A), np.abs(B))
        assert np.all(np.isfinite(got))
        assert (np.abs(got - ref) / scale).max() <= TOL[nprod]
        # and both agree with the FP64 product
        exact = np.einsum("bmk,bnk->bmn", A, B)
        assert (np.abs(got - exact) / scale).max() <= TOL[nprod]


def test_static_scratch_rejects_sizes_beyond_its_maximum(torch_lib):
    torch, lib = torch_lib
    M = N = K = 2048          # 3 planes x (2048+2048) x 2048 x 2 B = 48 MiB > 16 MiB
    dA = torch.zeros((M, K), dtype=torch.float64, device="cuda")
    dC = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    s = lib.xtrg_tc_gemm_static(dA.data_ptr(), dA.data_ptr(), dC.data_ptr(), M, N, K, 1, 3, 6, 1,
                                torch.cuda.current_stream().cuda_stream)
    assert s == lib.XTRG_ENOMEM

"""GPU unit test of the tcgen05 contraction primitive (xtrg_tc_gemm) against
an FP64 numpy reference on the same seeded inputs: ragged M, N, K (not
multiples of the 128 x 128 x 64 tile), batches, split-K, and the three
precision levels (1, 3, 6 products of BF16 split planes)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    # M,   N,   K,  batch, planes, nprod, splitk
    (128, 128, 64, 1, 2, 3, 1),
    (200, 130, 100, 3, 3, 6, 1),
    (256, 512, 1024, 1, 3, 6, 4),
    (64, 64, 512, 5, 2, 1, 2),
    (1, 1, 1, 1, 2, 3, 1),
    (384, 256, 4096, 2, 3, 6, 8),
]
# bound on |C - A B^T| relative to (|A| |B|^T), per product count
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


@pytest.mark.parametrize("M,N,K,batch,planes,nprod,splitk", CASES)
def test_tc_gemm_matches_fp64(torch_lib, M, N, K, batch, planes, nprod, splitk):
    torch, lib = torch_lib
    rng = np.random.default_rng(M * 7 + N * 13 + K + batch)
    A = rng.standard_normal((batch, M, K))
    B = rng.standard_normal((batch, N, K))
    ref = np.einsum("bmk,bnk->bmn", A, B)
    scale = np.einsum("bmk,bnk->bmn", np.abs(A), np.abs(B))
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.zeros((batch, M, N), dtype=torch.float64, device="cuda")
    nbytes = lib.xtrg_tc_gemm_workspace_bytes(M, N, K, batch, planes, splitk)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    p = (ws.data_ptr() + 255) // 256 * 256
    lib.xtrg_tc_gemm(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), M, N, K, batch, planes, nprod,
                     splitk, p, nbytes, torch.cuda.current_stream().cuda_stream)
    C = dC.cpu().numpy()
    err = np.abs(C - ref) / scale
    assert err.max() <= TOL[nprod], err.max()
    # a second call on the same buffers gives the same bits (no stale state)
    lib.xtrg_tc_gemm(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), M, N, K, batch, planes, nprod,
                     splitk, p, nbytes, torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(dC.cpu().numpy(), C)


@pytest.mark.parametrize("exact_bf16,planes,nprod", [(True, 2, 1), (False, 3, 6)])
def test_tc_gemm_long_chains_are_unbiased(torch_lib, exact_bf16, planes, nprod):
    """Long accumulations on one tile (K = 65536, no split-K) of positive
    products.  The tensor core's accumulator rounds toward zero, so chaining
    every K-block in tensor memory shrank such sums by ~4e-4 relative; the
    kernel keeps the leading products' chains to a few K-blocks and sums them
    in round-to-nearest FP32, so the mean signed error must stay at rounding
    level while the rms error is bounded by round-to-nearest accumulation."""
    torch, lib = torch_lib
    M = N = 128
    K = 65536
    rng = np.random.default_rng(20260)
    A = rng.uniform(0.5, 1.0, (1, M, K))
    B = rng.uniform(0.5, 1.0, (1, N, K))
    if exact_bf16:
        A = torch.from_numpy(A).to(torch.bfloat16).to(torch.float64).numpy()
        B = torch.from_numpy(B).to(torch.bfloat16).to(torch.float64).numpy()
    ref = np.einsum("bmk,bnk->bmn", A, B)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.zeros((1, M, N), dtype=torch.float64, device="cuda")
    nbytes = lib.xtrg_tc_gemm_workspace_bytes(M, N, K, 1, planes, 1)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    p = (ws.data_ptr() + 255) // 256 * 256
    lib.xtrg_tc_gemm(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), M, N, K, 1, planes, nprod, 1,
                     p, nbytes, torch.cuda.current_stream().cuda_stream)
    rel = (dC.cpu().numpy() - ref) / ref
    print("bias", rel.mean(), "rms", np.sqrt((rel ** 2).mean()))
    assert abs(rel.mean()) <= 3e-8
    assert np.sqrt((rel ** 2).mean()) <= 1e-6


NN_CASES = [
    # M,   N,   K,  batch, planes, nprod, splitk
    (128, 128, 64, 1, 3, 6, 1),
    (200, 130, 100, 3, 3, 6, 1),
    (256, 1000, 520, 1, 3, 6, 2),
    (64, 72, 512, 5, 2, 3, 2),
    (1, 1, 1, 1, 2, 1, 1),
]


@pytest.mark.parametrize("M,N,K,batch,planes,nprod,splitk", NN_CASES)
def test_tc_gemm_nn_mn_major_operand(torch_lib, M, N, K, batch, planes, nprod, splitk):
    """C = A B with B given K x N: B is staged into the tensor cores as an
    MN-major operand (two 64-wide TMA boxes per plane, MN-major shared-memory
    descriptor, transposed-B instruction bit).  The tiles hold the same
    values as the K-major staging of B^T, so the result must equal
    xtrg_tc_gemm on B^T bit for bit, and the FP64 product within the
    tolerance of the product count."""
    torch, lib = torch_lib
    rng = np.random.default_rng(M * 3 + N * 5 + K + batch)
    A = rng.standard_normal((batch, M, K))
    B = rng.standard_normal((batch, K, N))
    ref = np.einsum("bmk,bkn->bmn", A, B)
    scale = np.einsum("bmk,bkn->bmn", np.abs(A), np.abs(B))
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dBt = torch.from_numpy(np.ascontiguousarray(B.transpose(0, 2, 1))).cuda()
    st = torch.cuda.current_stream().cuda_stream
    dC = torch.zeros((batch, M, N), dtype=torch.float64, device="cuda")
    nb = lib.xtrg_tc_gemm_nn_workspace_bytes(M, N, K, batch, planes, splitk)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    p = (ws.data_ptr() + 255) // 256 * 256
    lib.xtrg_tc_gemm_nn(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), M, N, K, batch, planes, nprod,
                        splitk, p, nb, st)
    C = dC.cpu().numpy()
    assert (np.abs(C - ref) / scale).max() <= TOL[nprod]
    dT = torch.zeros((batch, M, N), dtype=torch.float64, device="cuda")
    nbt = lib.xtrg_tc_gemm_workspace_bytes(M, N, K, batch, planes, splitk)
    wst = torch.empty(nbt + 256, dtype=torch.uint8, device="cuda")
    pt = (wst.data_ptr() + 255) // 256 * 256
    lib.xtrg_tc_gemm(dA.data_ptr(), dBt.data_ptr(), dT.data_ptr(), M, N, K, batch, planes, nprod,
                     splitk, pt, nbt, st)
    assert np.array_equal(dT.cpu().numpy(), C)

"""The learned operator's BF16 training GEMM (kd_gemm_bf16_tn) on the tcgen05 tensor cores
against a plain PyTorch FP32 product of the same BF16 values, on tile-exact and ragged
shapes, and against the mma.sync engine; the training path uses it by default."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kd():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    return kd


def operands(M, N, K, seed):
    import torch
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    Bt = torch.randn(N, K, generator=g).to(torch.bfloat16)
    return A, Bt


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (1, 1, 8), (200, 136, 72), (257, 300, 1000), (130, 129, 4104),
                                   (512, 384, 256)])
@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_gemm_matches_fp32_reference(kd, M, N, K, engine):
    import torch
    A, Bt = operands(M, N, K, M * 7 + N * 3 + K)
    ref = A.double() @ Bt.double().T
    bound = A.double().abs() @ Bt.double().abs().T
    ldc = N + 5                                             # a row stride wider than N
    C = torch.full((M, ldc), float("nan"), dtype=torch.float32, device="cuda")
    e = kd.KD_GEMM_TCGEN05 if engine == "tcgen05" else kd.KD_GEMM_MMA_SYNC
    kd.kd_gemm_bf16_tn(A.cuda(), Bt.cuda(), C, e)
    torch.cuda.synchronize()
    out = C.cpu().double()
    assert torch.all(torch.isnan(out[:, N:]))               # nothing written past column N
    err = (out[:, :N] - ref).abs()
    assert torch.all(err <= 2e-6 * bound + 1e-6), float((err / (bound + 1e-30)).max())


def test_engines_agree_on_a_training_shape(kd):
    import torch
    M, N, K = 1024, 512, 2048
    A, Bt = operands(M, N, K, 5)
    Cs = []
    for e in (kd.KD_GEMM_TCGEN05, kd.KD_GEMM_MMA_SYNC):
        C = torch.empty((M, N), dtype=torch.float32, device="cuda")
        kd.kd_gemm_bf16_tn(A.cuda(), Bt.cuda(), C, e)
        Cs.append(C.cpu().double())
    bound = A.double().abs() @ Bt.double().abs().T
    assert torch.all((Cs[0] - Cs[1]).abs() <= 4e-6 * bound)


def test_unaligned_operands_are_rejected(kd):
    """Operand tiles move in 16-byte pieces (TMA boxes or cp.async): a base address that is
    not 16-byte aligned is refused before any launch."""
    import torch
    M, N, K = 140, 130, 96
    A, Bt = operands(M, N, K, 9)
    Ab = torch.zeros(M * K + 4, dtype=torch.bfloat16, device="cuda")
    Au = Ab[4:].view(M, K)                                  # 8-byte offset from the allocation
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    for e in (kd.KD_GEMM_TCGEN05, kd.KD_GEMM_MMA_SYNC):
        with pytest.raises(kd.KdError):
            kd.kd_gemm_bf16_tn(Au, Bt.cuda(), C, e)


def test_gemm_argument_errors(kd):
    import torch
    A = torch.zeros((4, 12), dtype=torch.bfloat16, device="cuda")     # K = 12: not a multiple of 8
    C = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(kd.KdError):
        kd.kd_gemm_bf16_tn(A, A, C)


def test_bounded_wait_gives_up_and_the_device_stays_usable(kd):
    """Failure detection without a fault: a wait whose producer never arrives returns
    KD_ETIMEOUT after its limit, and the next kernels run normally."""
    import torch
    assert kd.kd_selftest_wait(True, 5.0) == kd.KD_OK
    assert kd.kd_selftest_wait(False, 2.0) == kd.KD_ETIMEOUT
    A, Bt = operands(256, 256, 128, 3)
    C = torch.empty((256, 256), dtype=torch.float32, device="cuda")
    kd.kd_gemm_bf16_tn(A.cuda(), Bt.cuda(), C)
    ref = A.double() @ Bt.double().T
    bound = A.double().abs() @ Bt.double().abs().T
    assert torch.all((C.cpu().double() - ref).abs() <= 2e-6 * bound + 1e-6)

"""The BF16 tensor-core GEMM (tcgen05, FP32 accumulation) against an FP64
product of the same BF16-rounded operands."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_08919_gb300 import build
    build.build()
    import paper_1704_08919_gb300 as pp
    pp.lib()
    assert pp.sync_status() == pp.PP_OK
    return pp


def bf16(x):
    return x.to(torch.bfloat16).to(torch.float64)


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (128, 256, 64), (256, 256, 256), (384, 32, 128),
                                   (128, 48, 1024), (512, 256, 32), (256, 1, 256)])
def test_gemm_matches_fp64_product_of_bf16_operands(pp, M, N, K):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    Np = max(16, (N + 15) // 16 * 16)
    Kp = (K + 63) // 64 * 64
    Ap, _, _ = pp.pack_bf16(A)
    Bp, _, _ = pp.pack_bf16(B)
    D = pp.gemm_bf16(Ap, Bp, M, Np, Kp)
    assert pp.sync_status() == pp.PP_OK
    ref = (bf16(A.cpu()) @ bf16(B.cpu()).T).numpy()
    got = D[:, :N].cpu().double().numpy()
    scale = np.sqrt(K) * 1.0
    assert np.abs(got - ref).max() < 2e-5 * scale * np.abs(ref).max() / np.sqrt(K) + 1e-5 * scale
    assert np.abs(D[:, N:].cpu().numpy()).max() == 0.0 if Np > N else True


@pytest.mark.parametrize("M,N,K", [(128 * 400, 256, 128), (128 * 700, 48, 64), (128 * 300, 256, 640),
                                   (128 * 320, 112, 576)])
def test_gemm_with_more_tiles_than_sms(pp, M, N, K):
    """More 128-row tiles than SMs: every CTA of the persistent kernel walks several
    tiles and reuses both TMEM accumulators, so the hand-back between the epilogue
    and the MMA issuer is exercised, with B resident in shared memory (the first two
    shapes) and streamed with A (the last two: more than 8 B tiles)."""
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    Ap, _, _ = pp.pack_bf16(A)
    Bp, _, _ = pp.pack_bf16(B)
    D = pp.gemm_bf16(Ap, Bp, M, N, K)
    D2 = pp.gemm_bf16(Ap, Bp, M, N, K)
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(D, D2)
    ref = (bf16(A.cpu()) @ bf16(B.cpu()).T).numpy()
    got = D.cpu().double().numpy()
    assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max() + 1e-5 * np.sqrt(K)


@pytest.mark.parametrize("M,N,K,ldd", [(256, 144, 192, 144), (384, 144, 1024, 150), (256, 48, 64, 50)])
def test_gemm_column_halves_and_unaligned_rows(pp, M, N, K, ldd):
    """N between 128 and 256 (the second column half ends in a 16-column block) and
    rows of D whose stride is not a multiple of 4 floats (the epilogue falls back
    from 16-byte to 4-byte stores); columns past N are left alone."""
    g = torch.Generator(device="cpu").manual_seed(M + N + K + ldd)
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    Ap, _, _ = pp.pack_bf16(A)
    Bp, _, _ = pp.pack_bf16(B)
    buf = torch.full((M, ldd), 7.0, device="cuda")
    # through the C ABI: D is rows of ldd floats of which the first N are written
    rc = pp.lib().pp_gemm_bf16(ctypes.c_void_p(Ap.data_ptr()), ctypes.c_void_p(Bp.data_ptr()),
                               ctypes.c_void_p(buf.data_ptr()), M, N, K, ldd, None)
    assert rc == pp.PP_OK
    assert pp.sync_status() == pp.PP_OK
    D = buf[:, :N]
    ref = (bf16(A.cpu()) @ bf16(B.cpu()).T).numpy()
    assert np.abs(D.cpu().double().numpy() - ref).max() < 2e-5 * np.abs(ref).max() + 1e-5 * np.sqrt(K)
    if ldd > N:
        assert torch.all(buf[:, N:] == 7.0)


def test_gemm_transposed_packing(pp):
    g = torch.Generator(device="cpu").manual_seed(1)
    X = torch.randn(64, 256, generator=g).cuda()  # stored as (K rows) x (M cols): pack X^T
    W = torch.randn(32, 64, generator=g).cuda()
    Xp, rows, cols = pp.pack_bf16(X, transpose=True)  # 256 x 64
    assert (rows, cols) == (256, 64)
    Wp, _, _ = pp.pack_bf16(W)
    D = pp.gemm_bf16(Xp, Wp, 256, 32, 64)
    ref = (bf16(X.cpu()).T @ bf16(W.cpu()).T).numpy()
    assert np.abs(D.cpu().double().numpy() - ref).max() < 1e-4 * np.abs(ref).max()


def test_gemm_rejects_bad_shapes(pp):
    A = torch.zeros(16384, dtype=torch.uint8, device="cuda")
    with pytest.raises(pp.PPError):
        pp.gemm_bf16(A, A, 100, 16, 64)
    with pytest.raises(pp.PPError):
        pp.gemm_bf16(A, A, 128, 24, 64)
    with pytest.raises(pp.PPError):
        pp.gemm_bf16(A, A, 128, 16, 48)


@pytest.mark.parametrize("K", [128, 1024])  # B resident in shared memory / B streamed with A
def test_gemm_bounded_wait_gives_up_cleanly(pp, K):
    """With the copies switched off no stage ever fills: the bounded waits give up,
    the kernel records PP_ERR_TIMEOUT, frees its TMEM and returns; the next GEMM
    works."""
    A = torch.randn(256, K).cuda()
    B = torch.randn(64, K).cuda()
    Ap, _, _ = pp.pack_bf16(A)
    Bp, _, _ = pp.pack_bf16(B)
    old = pp.set_wait_limit(2000)
    pp.set_skip_copies(1)
    try:
        pp.gemm_bf16(Ap, Bp, 256, 64, K)
        st = pp.sync_status()
    finally:
        pp.set_skip_copies(0)
        pp.set_wait_limit(old)
    assert st == pp.PP_ERR_TIMEOUT
    D = pp.gemm_bf16(Ap, Bp, 256, 64, K)
    assert pp.sync_status() == pp.PP_OK
    ref = (bf16(A.cpu()) @ bf16(B.cpu()).T).numpy()
    assert np.abs(D.cpu().double().numpy() - ref).max() < 1e-3 * np.abs(ref).max()

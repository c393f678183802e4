"""tcgen05 BF16 GEMM (mc_gemm_bf16) against a plain PyTorch FP32 reference of
the same op: C = A . B^T (+ bias, ReLU, ReLU mask, split-K)."""
import pytest

from paper_2302_03343_b300 import mcint as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_03343_b300 import build
    build.build()
    return torch.device("cuda")


def operands(M_, N, K, dev, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    a = torch.randn(M_, K, generator=g).to(torch.bfloat16).to(dev)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16).to(dev)
    bias = torch.randn(N, generator=g).to(dev)
    return a, b, bias


def rel_err(x, ref):
    return ((x.float() - ref).abs().max() / ref.abs().max().clamp_min(1e-30)).item()


@pytest.mark.parametrize("M_,N,K,bn", [(128, 256, 256, 256), (256, 320, 256, 160), (384, 208, 64, 208),
                                       (128, 16, 128, 16), (640, 256, 512, 128)])
def test_gemm_bias_fp32(dev, M_, N, K, bn):
    a, b, bias = operands(M_, N, K, dev)
    c = torch.full((M_, N), float("nan"), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    M.mc_gemm_bf16(M_, N, K, bn, M.EPI_BIAS_F32, a, b, c, bias=bias, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = a.float() @ b.float().T + bias
    assert rel_err(c, ref) < 1e-5


def test_gemm_split_k_atomic(dev):
    M_, N, K = 256, 256, 4096
    a, b, _ = operands(M_, N, K, dev, seed=1)
    c = torch.zeros((M_, N), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    M.mc_gemm_bf16(M_, N, K, 256, M.EPI_ATOMIC_F32, a, b, c, splits=8, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert rel_err(c, a.float() @ b.float().T) < 1e-5


def test_gemm_relu_bf16_and_mask(dev):
    M_, N, K = 256, 256, 256
    a, b, bias = operands(M_, N, K, dev, seed=2)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    c = torch.empty((M_, N), dtype=torch.bfloat16, device=dev)
    M.mc_gemm_bf16(M_, N, K, 256, M.EPI_BIAS_RELU_BF16, a, b, c, bias=bias, err=err)
    ref = torch.relu(a.float() @ b.float().T + bias)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert ((c.float() - ref).abs() <= 2 ** -7 * ref.abs() + 1e-6).all()
    mask = torch.randn(M_, N, device=dev).to(torch.bfloat16)
    g = torch.empty((M_, N), dtype=torch.bfloat16, device=dev)
    M.mc_gemm_bf16(M_, N, K, 256, M.EPI_RELU_MASK_BF16, a, b, g, mask=mask, err=err)
    ref = (a.float() @ b.float().T) * (mask.float() > 0)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert ((g.float() - ref).abs() <= 2 ** -7 * ref.abs() + 1e-6).all()


def test_gemm_rejects_bad_shapes(dev):
    a, b, bias = operands(100, 256, 256, dev)
    c = torch.empty((100, 256), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(M.McError):
        M.mc_gemm_bf16(100, 256, 256, 256, M.EPI_BIAS_F32, a, b, c, err=err)


def test_gemm_split_k_partials(dev):
    M_, N, K, S = 256, 320, 2048, 4
    a, b, _ = operands(M_, N, K, dev, seed=3)
    c = torch.full((S, M_, N), float("nan"), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    M.mc_gemm_bf16(M_, N, K, 160, M.EPI_PARTIAL_F32, a, b, c, splits=S, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    for s in range(S):  # split s covers K blocks [s K/S, (s+1) K/S)
        k0, k1 = s * K // S, (s + 1) * K // S
        assert rel_err(c[s], a[:, k0:k1].float() @ b[:, k0:k1].float().T) < 1e-5


# the persistent B-resident kernel: every M tile count (fewer tiles than SMs,
# several per CTA, an odd remainder), N split into two tiles, K up to 320
@pytest.mark.parametrize("M_,N,K,bn", [(128, 256, 256, 256), (65536, 256, 256, 256), (40960 + 128, 320, 256, 160),
                                       (1024, 256, 320, 256), (384, 64, 64, 64), (19072, 288, 256, 144)])
def test_gemm_rs_bias_fp32_and_transposed(dev, M_, N, K, bn):
    a, b, bias = operands(M_, N, K, dev, seed=4)
    c = torch.full((M_, N), float("nan"), device=dev)
    ct = torch.full((N, M_), float("nan"), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    M.mc_gemm_bf16_rs(M_, N, K, bn, M.EPI_BIAS_F32, a, b, c=c, c_t=ct, bias=bias, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = a.float() @ b.float().T + bias
    assert rel_err(c, ref) < 1e-5
    assert torch.equal(ct, c.T)


def test_gemm_rs_relu_and_mask_bf16(dev):
    # absolute slack 1e-4: sums of 256 products of N(0, 1) values are ~16, so
    # FP32 accumulation in another order moves them by ~1e-5, which decides
    # the ReLU differently for pre-activations that close to zero
    M_, N, K = 8192 + 256, 256, 256
    a, b, bias = operands(M_, N, K, dev, seed=5)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    c = torch.empty((M_, N), dtype=torch.bfloat16, device=dev)
    ct = torch.empty((N, M_), dtype=torch.bfloat16, device=dev)
    M.mc_gemm_bf16_rs(M_, N, K, 256, M.EPI_BIAS_RELU_BF16, a, b, c=c, c_t=ct, bias=bias, err=err)
    ref = torch.relu(a.float() @ b.float().T + bias)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert ((c.float() - ref).abs() <= 2 ** -7 * ref.abs() + 1e-4).all()
    assert torch.equal(ct, c.T)
    mask = torch.randn(M_, N, device=dev).to(torch.bfloat16)
    g = torch.empty((M_, N), dtype=torch.bfloat16, device=dev)
    M.mc_gemm_bf16_rs(M_, N, K, 256, M.EPI_RELU_MASK_BF16, a, b, c=g, mask=mask, err=err)
    ref = (a.float() @ b.float().T) * (mask.float() > 0)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert ((g.float() - ref).abs() <= 2 ** -7 * ref.abs() + 1e-4).all()


def test_gemm_rs_rejects_oversized_b(dev):
    a, b, _ = operands(128, 256, 384, dev)
    c = torch.empty((128, 256), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(M.McError):
        M.mc_gemm_bf16_rs(128, 256, 384, 256, M.EPI_BIAS_F32, a, b, c=c, err=err)


# both operands MN-major: C = X^T Y from row-major X [K x M], Y [K x N]
@pytest.mark.parametrize("M_,N,K,bn,splits", [(128, 64, 64, 64, 1), (256, 256, 4096, 256, 4), (256, 320, 8192, 64, 8),
                                              (128, 128, 65536, 128, 37)])
def test_gemm_tn_weight_gradient(dev, M_, N, K, bn, splits):
    g = torch.Generator(device="cpu").manual_seed(7)
    x = torch.randn(K, M_, generator=g).to(torch.bfloat16).to(dev)
    y = torch.randn(K, N, generator=g).to(torch.bfloat16).to(dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    c = torch.zeros((M_, N), device=dev)
    M.mc_gemm_bf16_tn(M_, N, K, bn, M.EPI_ATOMIC_F32, x, y, c, splits=splits, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = x.double().T @ y.double()
    assert ((c.double() - ref).abs().max() / ref.abs().max()).item() < 1e-5


# A MN-major, B K-major: C = X^T B^T from row-major X [K x M] and B [N x K]
# (the weight gradient from row-major activations and transposed gradients);
# N = 240 and 320 are the logit widths of three and four transformed
# coordinates, tiles of 16 to 256 columns
@pytest.mark.parametrize("M_,N,K,bn,splits", [(128, 16, 64, 16, 1), (256, 256, 4096, 256, 4), (256, 240, 8192, 240, 8),
                                              (256, 320, 65536, 160, 37), (128, 128, 65536, 128, 74)])
def test_gemm_xn_weight_gradient(dev, M_, N, K, bn, splits):
    g = torch.Generator(device="cpu").manual_seed(11)
    x = torch.randn(K, M_, generator=g).to(torch.bfloat16).to(dev)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16).to(dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    c = torch.zeros((M_, N), device=dev)
    M.mc_gemm_bf16_xn(M_, N, K, bn, M.EPI_ATOMIC_F32, x, b, c, splits=splits, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = x.double().T @ b.double().T
    assert ((c.double() - ref).abs().max() / ref.abs().max()).item() < 1e-5
    # the per-split partials (epilogue 4) sum to the same product, and the
    # K-major product of the transposed X gives the same bits split by split
    parts = torch.empty((splits, M_, N), device=dev)
    M.mc_gemm_bf16_xn(M_, N, K, bn, M.EPI_PARTIAL_F32, x, b, parts, splits=splits, err=err)
    parts_k = torch.empty((splits, M_, N), device=dev)
    M.mc_gemm_bf16(M_, N, K, bn, M.EPI_PARTIAL_F32, x.T.contiguous(), b, c=parts_k, splits=splits, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    assert ((parts.double().sum(0) - ref).abs().max() / ref.abs().max()).item() < 1e-5
    assert torch.equal(parts, parts_k)


def test_gemm_xn_rejects_bad_shapes(dev):
    x = torch.zeros(64, 128, dtype=torch.bfloat16, device=dev)
    b = torch.zeros(24, 64, dtype=torch.bfloat16, device=dev)
    c = torch.zeros((128, 24), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(M.McError):  # bn does not divide N
        M.mc_gemm_bf16_xn(128, 24, 64, 16, M.EPI_ATOMIC_F32, x, b, c, err=err)
    with pytest.raises(M.McError):  # an epilogue with a BF16 output
        M.mc_gemm_bf16_xn(128, 16, 64, 16, 0, x, b[:16], c[:, :16], err=err)

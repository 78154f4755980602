"""gfbp_wht: the Walsh-Hadamard transform on the CUDA cores (FP32 butterflies)
and on the tensor cores (FP16 hi/lo split, FP32 accumulation) against the
transform written out in FP64 (y[b] = sum_a (-1)^popcount(a & b) x[a])."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp
    gfbp.lib()
    return torch


def hadamard(q):
    a = np.arange(q)
    bits = np.bitwise_and.outer(a, a)
    par = np.zeros_like(bits)
    for k in range(8):
        par ^= (bits >> k) & 1
    return np.where(par, -1.0, 1.0)


@pytest.mark.parametrize("q", [2, 4, 8, 16, 32, 64, 128, 256])
def test_simt_matches_fp64(torch_cuda, q):
    from paper_cs_0605069_gb300 import gfbp
    rng = np.random.default_rng(q)
    x = rng.random((333, q))
    x /= x.sum(1, keepdims=True)
    ref = x @ hadamard(q)
    y = gfbp.wht(torch_cuda.from_numpy(x.astype(np.float32)).cuda(), "simt").cpu().numpy()
    assert np.abs(y - ref).max() <= 4e-7 * np.log2(q) + 1e-7


@pytest.mark.parametrize("q", [16, 32, 64, 128, 256])
@pytest.mark.parametrize("n", [1, 64, 1000])
def test_tensor_matches_fp64(torch_cuda, q, n):
    """Probability vectors and products of transforms (entries in [-1, 1]),
    a ragged last block of rows, one-hot rows and rows of tiny values."""
    from paper_cs_0605069_gb300 import gfbp
    rng = np.random.default_rng(1000 + q + n)
    x = rng.random((n, q))
    x /= x.sum(1, keepdims=True)
    if n >= 64:
        x[1] = 0.0
        x[1, 3 % q] = 1.0
        x[2] = rng.uniform(-1, 1, q)
        x[3] *= 1e-6
    ref = x @ hadamard(q)
    y = gfbp.wht(torch_cuda.from_numpy(x.astype(np.float32)).cuda(), "tensor").cpu().numpy()
    # every output sums all q inputs with signs.  Per input the split keeps
    # about 22 bits of |x_a|, and entries below 2^-14 of the row's largest
    # (scaled to [1, 2)) fall into FP16's subnormals, 2^-25 absolute; the
    # tensor cores' FP32 accumulation over 2 q / 16 steps adds a few 2^-23
    # of the partial sums (<= sum_a |x_a|).
    l1 = np.abs(x).sum(1, keepdims=True)
    mx = np.abs(x).max(1, keepdims=True)
    bound = 2.0 ** -19 * l1 + q * 2.0 ** -24 * mx
    assert (np.abs(y - ref) <= bound).all(), (np.abs(y - ref) / bound).max()
    y32 = gfbp.wht(torch_cuda.from_numpy(x.astype(np.float32)).cuda(), "simt").cpu().numpy()
    assert (np.abs(y - y32) <= 2 * bound).all()


def test_tensor_rejects_small_q(torch_cuda):
    from paper_cs_0605069_gb300 import gfbp
    with pytest.raises(gfbp.GfbpError):
        gfbp.wht(torch_cuda.zeros((4, 8), device="cuda"), "tensor")

"""Warm-start MLP kernels (BF16 tensor-core GEMMs, FP32 accumulation) against the FP64 oracle
of the same network with the same BF16 rounding points."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_06650_gb300.build import build
    build()
    from paper_2310_06650_gb300 import qg as mod
    return mod


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# shapes: ragged features and batch (TMA reads beyond the tensors as zeros), several 128-row and
# 256-column tiles, a long K split over many blocks (n_in 5003: 79 K blocks), the full 64-row batch
@pytest.mark.parametrize("n_in,n_h,n_out,B", [(300, 128, 200, 16), (1111, 256, 777, 37), (5003, 384, 1500, 64)])
def test_mlp_forward_and_gradients_match_oracle(qg, n_in, n_h, n_out, B):
    from oracle import mlp
    m = qg.qg_mlp_create(n_in, n_h, n_out, 64, seed=7)
    npar = qg.qg_mlp_num_params(m)
    w = torch.zeros(npar, dtype=torch.float32, device="cuda")
    qg.qg_mlp_get_params(m, w)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(B, n_in)).astype(np.float32)
    Tg = rng.normal(size=(B, n_out)).astype(np.float32)
    # random non-zero biases so that every term is exercised
    wn = w.cpu().numpy().astype(np.float64)
    _, _, _, _, _, _ = mlp.split(wn, n_in, n_h, n_out)
    wn += np.concatenate([np.zeros(n_h * n_in), rng.normal(0, 0.1, n_h), np.zeros(n_h * n_h), rng.normal(0, 0.1, n_h),
                          np.zeros(n_out * n_h), rng.normal(0, 0.1, n_out)])
    wt = torch.tensor(wn.astype(np.float32), device="cuda")
    qg.qg_mlp_set_params(m, wt)
    xt = torch.tensor(X, device="cuda")
    tt = torch.tensor(Tg, device="cuda")
    y = torch.zeros(B, n_out, dtype=torch.float32, device="cuda")
    qg.qg_mlp_forward(m, xt, B, y)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    qg.qg_mlp_train_step(m, xt, tt, B, 0.0, 0.9, 0.999, loss)
    g = torch.zeros(npar, dtype=torch.float32, device="cuda")
    qg.qg_mlp_get_grads(m, g)
    torch.cuda.synchronize()
    Yr, Lr, Gr = mlp.forward_backward(wt.cpu().numpy().astype(np.float64), X.astype(np.float64), Tg, n_in, n_h, n_out)
    assert rel(y.cpu().numpy(), Yr) <= 2e-3
    assert abs(loss.item() - Lr) <= 2e-3 * Lr
    G = g.cpu().numpy()
    sizes = [n_h * n_in, n_h, n_h * n_h, n_h, n_out * n_h, n_out]
    o = 0
    for k, sz in enumerate(sizes):
        assert rel(G[o:o + sz], Gr[o:o + sz]) <= 5e-3, k
        o += sz
    qg.qg_mlp_check(m)  # no GEMM pipeline wait ran out
    qg.qg_mlp_destroy(m)


def test_mlp_training_reduces_the_loss(qg):
    n_in, n_h, n_out, B = 64, 128, 32, 32
    m = qg.qg_mlp_create(n_in, n_h, n_out, B, seed=3)
    g = torch.Generator().manual_seed(0)
    X = torch.randn(B, n_in, generator=g).cuda()
    A = torch.randn(n_out, n_in, generator=g).cuda() * 0.2
    Tg = torch.tanh(X @ A.T)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    qg.qg_mlp_train_step(m, X, Tg, B, 0.0, 0.9, 0.999, loss)
    l0 = loss.item()
    for _ in range(300):
        qg.qg_mlp_train_step(m, X, Tg, B, 1e-3, 0.9, 0.999, loss)
    torch.cuda.synchronize()
    assert loss.item() < 0.05 * l0
    qg.qg_mlp_check(m)
    qg.qg_mlp_destroy(m)


def test_mlp_batch_limit(qg):
    with pytest.raises(qg.QGError) as ei:
        qg.qg_mlp_create(16, 32, 8, 65, seed=1)
    assert ei.value.code == qg.QG_ERR_UNSUPPORTED


def test_mlp_forward_is_bitwise_repeatable(qg):
    """Split-K partials are summed in a fixed order: the same input gives the same bits."""
    n_in, n_h, n_out, B = 2222, 256, 640, 48
    m = qg.qg_mlp_create(n_in, n_h, n_out, 64, seed=5)
    x = torch.randn(B, n_in, generator=torch.Generator().manual_seed(2)).cuda()
    y1 = torch.zeros(B, n_out, device="cuda")
    y2 = torch.zeros(B, n_out, device="cuda")
    qg.qg_mlp_forward(m, x, B, y1)
    qg.qg_mlp_forward(m, x, B, y2)
    qg.qg_mlp_check(m)
    assert torch.equal(y1, y2) and bool(torch.isfinite(y1).all())
    qg.qg_mlp_destroy(m)

"""The surrogate network on the GPU (tensor-core forward and backward, Adam)
against the FP64 CPU oracle (oracle/surrogate.py): with the oracle rounding the
tensor-core operands to BF16 the results agree to FP32/BF16-boundary noise; against
the exact network they agree to the BF16 precision of those operands."""
import numpy as np
import pytest

from oracle import surrogate as S

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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def setup(d_in, H, B, seed):
    rng = np.random.default_rng(seed)
    p = S.init_params(d_in, H, seed=seed)
    lay, _ = S.layout(d_in, H)
    for k in ("b1", "b2", "b3", "b4"):
        o, s = lay[k]
        p[o:o + int(np.prod(s))] = rng.normal(0, 0.1, int(np.prod(s)))
    p = p.astype(np.float32).astype(np.float64)  # the GPU keeps FP32 masters
    X = rng.uniform(-0.5, 0.5, (B, d_in)).astype(np.float32).astype(np.float64)
    t = rng.normal(size=B).astype(np.float32).astype(np.float64)
    return p, X, t


@pytest.mark.parametrize("d_in,B,H", [(32, 128, 256), (32, 300, 256), (64, 256, 256), (100, 200, 128),
                                     (200, 260, 256)])
def test_forward_and_gradient_match_oracle(pp, d_in, B, H):
    # d_in 100 and 200 pad to 128 and 256 input columns (the weight gradient of the
    # first layer then has one or two column halves); H = 128 is one row tile
    p, X, t = setup(d_in, H, B, seed=d_in + B)
    net = pp.Surrogate(d_in, H, max_batch=512)
    net.set_params(torch.tensor(p, dtype=torch.float32, device="cuda"))
    Xg = torch.tensor(X, dtype=torch.float32, device="cuda")
    tg = torch.tensor(t, dtype=torch.float32, device="cuda")
    y = net.forward(Xg).cpu().double().numpy()
    loss, g = net.loss_grad(Xg, tg)
    assert pp.sync_status() == pp.PP_OK
    g = g.cpu().double().numpy()
    y16, _ = S.forward(p, X, d_in, H, bf16=True)
    yex, _ = S.forward(p, X, d_in, H, bf16=False)
    assert rel(y, y16) < 2e-3
    assert rel(y, yex) < 3e-2
    l16, g16 = S.loss_grad(p, X, t, d_in, H, bf16=True)
    lex, gex = S.loss_grad(p, X, t, d_in, H, bf16=False)
    assert abs(loss.item() / l16 - 1) < 5e-3
    lay, _ = S.layout(d_in, H)
    for k, (o, s) in lay.items():
        n = int(np.prod(s))
        assert rel(g[o:o + n], g16[o:o + n]) < 1e-2, k
        assert rel(g[o:o + n], gex[o:o + n]) < 5e-2, k
    net.close()


def test_adam_step_matches_oracle(pp):
    d_in, H, B = 32, 256, 128
    p, X, t = setup(d_in, H, B, seed=3)
    net = pp.Surrogate(d_in, H, max_batch=B)
    net.set_params(torch.tensor(p, dtype=torch.float32, device="cuda"))
    Xg = torch.tensor(X, dtype=torch.float32, device="cuda")
    tg = torch.tensor(t, dtype=torch.float32, device="cuda")
    _, g = net.loss_grad(Xg, tg)
    net.train_step(Xg, tg, 1e-3)
    p1 = net.get_params().cpu().double().numpy()
    ref, _, _ = S.adam(p, g.cpu().double().numpy(), np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
    assert np.abs(p1 - ref).max() < 1e-6
    net.close()


def test_training_learns_a_smooth_function(pp):
    d_in, H = 32, 256
    rng = np.random.default_rng(7)
    Xtr = rng.uniform(-0.5, 0.5, (4096, d_in))
    Xte = rng.uniform(-0.5, 0.5, (1024, d_in))
    a = rng.normal(size=d_in) / np.sqrt(d_in)

    def f(X):
        return np.sin(3 * X @ a) + 0.5 * (X[:, 0] * X[:, 1]) * 4

    net = pp.Surrogate(d_in, H, max_batch=1024)
    net.set_params(torch.tensor(S.init_params(d_in, H, 1), dtype=torch.float32, device="cuda"))
    Xg = torch.tensor(Xtr, dtype=torch.float32, device="cuda")
    tg = torch.tensor(f(Xtr), dtype=torch.float32, device="cuda")
    first = None
    for ep in range(60):
        perm = torch.randperm(4096, device="cuda")
        for b in range(0, 4096, 512):
            idx = perm[b:b + 512]
            loss = net.train_step(Xg[idx].contiguous(), tg[idx].contiguous(), 2e-3)
            if first is None:
                first = loss.item()
    yte = net.forward(torch.tensor(Xte, dtype=torch.float32, device="cuda")).cpu().numpy()
    mse = float(np.mean((yte - f(Xte)) ** 2))
    var = float(np.var(f(Xte)))
    assert pp.sync_status() == pp.PP_OK
    assert mse < 0.05 * var, (mse, var, first)
    net.close()

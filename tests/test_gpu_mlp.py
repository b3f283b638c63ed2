"""GPU kernels of the learned blocking against the oracle (oracle/learn.py):
forward pass, loss and gradient (FP32 kernels vs the FP64 chain rule), the
Adam step; and training through the kernels decreasing the loss, bit-exact
across runs."""
import numpy as np
import pytest

from oracle import learn as ol
from paper_2609_00561_gb300 import build as libbuild
from paper_2609_00561_gb300 import iccg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    libbuild.build()


def _net(nf, h, c, B, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, 0.4, ol.mlp_offsets(nf, h, c)["total"]).astype(np.float32)
    X = rng.normal(size=(B, nf)).astype(np.float32)
    y = rng.integers(0, c, B).astype(np.int32)
    yr = rng.normal(size=B).astype(np.float32)
    return p, X, y, yr


@pytest.mark.parametrize("shape", [(20, 64, 5, 160), (3, 5, 2, 7), (20, 64, 5, 1)])
def test_forward_loss_and_gradient_match_oracle(shape):
    nf, h, c, B = shape
    p, X, y, yr = _net(nf, h, c, B, 1)
    assert iccg.mlp_nparams(nf, h, c) == p.size
    dev = "cuda"
    P, Xd = torch.tensor(p, device=dev), torch.tensor(X, device=dev)
    out = torch.zeros((B, c + 1), dtype=torch.float32, device=dev)
    act = torch.zeros(2 * B * h, dtype=torch.float32, device=dev)
    iccg.mlp_forward(P, nf, h, c, Xd, out, act)
    zr, h1, h2 = ol.mlp_forward(p, nf, h, c, X)
    assert np.allclose(out.cpu().numpy(), zr, rtol=1e-5, atol=1e-5 * np.abs(zr).max())
    assert np.allclose(act.cpu().numpy()[:B * h].reshape(B, h), h1, rtol=1e-5, atol=1e-5)
    G = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    work = torch.zeros(B * (4 * h + 2 * (c + 1) + 1), dtype=torch.float32, device=dev)
    iccg.mlp_grad(P, nf, h, c, Xd, torch.tensor(y, device=dev), torch.tensor(yr, device=dev), 0.5, G, loss, work)
    gr = ol.mlp_grad(p, nf, h, c, X, y, yr, 0.5)
    g = G.cpu().numpy()
    assert np.max(np.abs(g - gr)) <= 1e-4 * np.max(np.abs(gr)) + 1e-7
    assert float(loss.item()) == pytest.approx(ol.mlp_loss(p, nf, h, c, X, y, yr, 0.5), rel=1e-5)


def test_adam_matches_oracle():
    rng = np.random.default_rng(2)
    n = 1000
    p, g = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    m, v = (rng.normal(size=n) * 0.1).astype(np.float32), np.abs(rng.normal(size=n) * 0.01).astype(np.float32)
    P, Gd, M, V = (torch.tensor(a, device="cuda") for a in (p, g, m, v))
    iccg.mlp_adam(P, Gd, M, V, 1e-2, 0.9, 0.999, 1e-8, 7)
    pr, mr, vr = ol.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                         1e-2, 0.9, 0.999, 1e-8, 7)
    assert np.allclose(P.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    assert np.allclose(M.cpu().numpy(), mr, rtol=1e-5, atol=1e-7)


def test_training_decreases_loss_and_is_reproducible():
    from paper_2609_00561_gb300.learn.model import Model
    rng = np.random.default_rng(3)
    X = rng.normal(size=(120, 20))
    yc = (X[:, 0] > 0).astype(np.int32) + 2 * (X[:, 1] > 0.5).astype(np.int32)   # 4 separable classes
    yr = 0.5 * X[:, 2] - X[:, 3]
    runs = []
    for _ in range(2):
        m = Model(20, 5, seed=4)
        hist = m.fit(X, yc, yr, epochs=600, lr=3e-3)
        runs.append(m.params.copy())
        assert hist[-1] < 0.2 * hist[0]
        cls, lg = m.predict(X)
        assert np.mean(cls == yc) > 0.95
    assert np.array_equal(runs[0], runs[1])

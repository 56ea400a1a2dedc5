"""GPU parity of the learned-policy kernels against the FP64 oracle.

Logits: norm-wise relative error max|GPU - ref| / max|ref| <= 1e-5 (FP32
accumulation of at most 32-term dot products, |rel. rounding| ~ 32 * 2^-24).
Gradients: <= 1e-4 relative (FP32 sums over the rows of the batch).
"""
import numpy as np
import pytest

import oracle
import paper_2607_17106_gb300 as bg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_17106_gb300 import build
    build.build()
    bg.load()


def _params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.3, bg.BFS_MLP_NPARAM)


def _identity_norm_weights(P):
    w = np.concatenate([P, np.zeros(10), np.ones(10)]).astype(np.float32)
    return w


def test_forward_matches_fp64_reference():
    P = _params(1).astype(np.float32).astype(np.float64)  # the exact FP32 values on both sides
    pol = bg.Policy(_identity_norm_weights(P))
    rng = np.random.default_rng(2)
    rows = 4099
    X = rng.normal(0, 2, (rows, 10)).astype(np.float32)
    ref = oracle.mlp_forward(P, X.astype(np.float64))
    Xd = torch.from_numpy(X).cuda()
    out = torch.empty(rows, 3, dtype=torch.float32, device="cuda")
    pol.forward(Xd, out, rows)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5


def test_normalisation_is_applied():
    P = _params(3).astype(np.float32).astype(np.float64)
    mean = np.linspace(-1, 1, 10).astype(np.float32)
    istd = np.linspace(0.5, 2, 10).astype(np.float32)
    pol = bg.Policy(np.concatenate([P.astype(np.float32), mean, istd]))
    X = np.random.default_rng(4).normal(0, 3, (257, 10)).astype(np.float32)
    Xn = ((X - mean) * istd).astype(np.float64)
    ref = oracle.mlp_forward(P, Xn)
    out = torch.empty(257, 3, dtype=torch.float32, device="cuda")
    pol.forward(torch.from_numpy(X).cuda(), out, 257)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-5


def test_gradient_and_adam_step_match_fp64_reference():
    P = _params(5).astype(np.float32).astype(np.float64)
    pol = bg.Policy(_identity_norm_weights(P))
    rng = np.random.default_rng(6)
    rows = 3000
    X = rng.normal(0, 1, (rows, 10)).astype(np.float32)
    y = rng.integers(0, 3, rows).astype(np.int32)
    loss_ref, g_ref = oracle.mlp_loss_grad(P, X.astype(np.float64), y)
    grad = torch.empty(bg.BFS_MLP_NPARAM, dtype=torch.float32, device="cuda")
    lr = 1e-2
    loss = pol.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), rows, lr, 1, grad_out=grad)
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - g_ref)) / np.max(np.abs(g_ref)) <= 1e-4
    assert abs(loss - loss_ref) / loss_ref <= 1e-5
    # the update is Adam step 1 applied to the GPU's own gradient
    Pn = P.copy()
    m1, m2 = np.zeros_like(P), np.zeros_like(P)
    oracle.adam_step(Pn, m1, m2, g, t=1, lr=lr, eps=1e-8)
    w = pol.weights().astype(np.float64)[: bg.BFS_MLP_NPARAM]
    assert np.max(np.abs(w - Pn)) <= 1e-6 + 1e-5 * lr


def test_training_reduces_loss_on_a_separable_task():
    rng = np.random.default_rng(7)
    rows = 2048
    X = rng.normal(0, 1, (rows, 10)).astype(np.float32)
    y = np.argmax(X[:, :3], axis=1).astype(np.int32)
    pol = bg.Policy(_identity_norm_weights(_params(8) * 0.5))
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    first = pol.train_step(Xd, yd, rows, 1e-2, 1)
    last = first
    for t in range(2, 301):
        last = pol.train_step(Xd, yd, rows, 1e-2, t)
    assert last < 0.3 * first
    out = torch.empty(rows, 3, dtype=torch.float32, device="cuda")
    pol.forward(Xd, out, rows)
    acc = (out.argmax(1).cpu().numpy() == y).mean()
    assert acc > 0.9

"""The training objective as torch.autograd Functions over the hand-written
backward kernels (paper_2412_07127_gb300.autograd): loss.backward() gives the
same gradient as calling the backward entry points in sequence (bit for bit),
matches the FP64 oracle's chain (GNN forward, Eq. 2 correction, probe loss
Eq. 4-5 and their backward passes) and central finite differences of the GPU
loss itself."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_07127_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_07127_gb300 import build, gicpcg
    build.build()
    return gicpcg


def _nrel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _setup(G, h, nb=2, N=3):
    Es = [I.material_field(N, 50 + k) for k in range(nb)]
    rp, c, v = G.fem_hex_assemble(h, N, torch.from_numpy(np.concatenate(Es)).to(DEV), nb=nb)
    P = G.Pattern(h, rp, c)
    As = [O.fem_hex_assemble(N, E) for E in Es]
    x9, e0, scale, Ahat = G.features(h, P, v, ngraphs=nb, with_ahat=True)
    LIC, bad = G.ic0(h, P, v)
    assert bad == -1
    LIChat = G.scale_factor(h, P, LIC, scale, ngraphs=nb)
    Zs = [I.probes(8, As[0].n, 60 + k) for k in range(nb)]
    Z = torch.from_numpy(np.concatenate(Zs, axis=1)).to(DEV)
    return P, As, x9, e0, LIChat, Ahat, Zs, Z


def test_autograd_gradient_equals_the_backward_chain_and_the_oracle(G):
    from paper_2412_07127_gb300.autograd import training_loss
    h = G.Handle(0)
    nb = 2
    P, As, x9, e0, LIChat, Ahat, Zs, Z = _setup(G, h, nb)
    t32 = I.gnn_init(7, out_scale=0.2).astype(np.float32)
    theta = torch.from_numpy(t32).to(DEV).requires_grad_(True)
    loss = training_loss(theta, h, P, x9, e0, LIChat, Ahat, Z, ngraphs=nb)
    loss.backward()
    d_auto = theta.grad.detach().clone()

    # the same chain through the entry points, called one after the other
    ws = G.gnn_workspace(h, P, nb, training=True)
    th = theta.detach().contiguous()
    g = G.gnn_forward_train(h, P, th, x9, e0, ws, ngraphs=nb)
    Lhat = G.gnn_correct_scaled(h, P, LIChat, g)
    l2, dL = G.probe_loss(h, P, Ahat, Lhat, Z, ngraphs=nb, grad=True)
    d_chain = G.gnn_backward(h, P, th, x9, e0, G.gnn_correct_backward(h, P, Lhat, dL), ws, ngraphs=nb)
    assert float(loss) == float(l2[nb])
    assert torch.equal(d_auto, d_chain)

    # the FP64 oracle's chain on the same systems, parameters and probes
    t64 = t32.astype(np.float64)
    ref = np.zeros(t64.size)
    for k, A in enumerate(As):
        T = O.lower(A)
        ox9, oe0, s = O.features(A)
        og = O.gnn_forward(T, ox9, oe0, t64)
        Lo, _ = O.ic0(A)
        Lh = O.correct(T, Lo.val / np.sqrt(s), og)
        _, dLk = O.probe_loss(O.CSR(A.rowptr, A.col, A.val / s), O.CSR(T.rowptr, T.col, Lh),
                              Zs[k].astype(np.float64), grad=True)
        ref += O.gnn_backward(T, ox9, oe0, t64, O.correct_backward(T, Lo.val / np.sqrt(s), og, dLk / nb))
    assert _nrel(d_auto.cpu().numpy(), ref) <= 1e-3


def test_autograd_gradient_matches_finite_differences(G):
    """Directional derivative of the GPU loss along random directions of the
    MLP weights: autograd against (L(t + e u) - L(t - e u)) / 2e. The loss is
    FP32, so e is large enough that the difference is far above its
    rounding and the bound is 1e-2."""
    from paper_2412_07127_gb300.autograd import training_loss
    h = G.Handle(0)
    nb = 2
    P, As, x9, e0, LIChat, Ahat, Zs, Z = _setup(G, h, nb)
    t32 = I.gnn_init(8, out_scale=0.2).astype(np.float32)
    theta = torch.from_numpy(t32).to(DEV).requires_grad_(True)
    loss = training_loss(theta, h, P, x9, e0, LIChat, Ahat, Z, ngraphs=nb)
    loss.backward()
    grad = theta.grad.detach()
    rng = np.random.default_rng(3)
    for _ in range(3):
        u = rng.standard_normal(t32.size).astype(np.float32)
        u[:27] = 0.0  # GraphNorm's shift is very curved on these small meshes
        u = torch.from_numpy(u / np.linalg.norm(u)).to(DEV)
        eps = 1e-2
        with torch.no_grad():
            lp = float(training_loss(theta.detach() + eps * u, h, P, x9, e0, LIChat, Ahat, Z, ngraphs=nb))
            lm = float(training_loss(theta.detach() - eps * u, h, P, x9, e0, LIChat, Ahat, Z, ngraphs=nb))
        fd = (lp - lm) / (2 * eps)
        an = float(torch.dot(grad, u))
        assert abs(fd - an) <= 1e-2 * max(abs(an), 1e-3 * float(loss)), (fd, an)

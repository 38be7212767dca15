"""torch.autograd view of the training path (argument marshalling only).

Each Function's forward and backward are the library's own kernels behind the
C-ABI; torch only chains them and carries the tensors:

  GnnForward     g = GNN_theta(x, e0) on tril(A) (Section "Model Architecture"),
                 backward: gic_gnn_backward (hand-written edge/node MLP,
                 aggregation and GraphNorm backward on the kept activations)
  CorrectScaled  L^ = L^_IC + g off the diagonal, L^_IC exp(g/2) on it (Eq. 2),
                 backward: gic_gnn_correct_backward
  ProbeLoss      (1/m) sum_k ||L^ L^T z_k - A^ z_k||^2 averaged over the
                 batch's graphs (Eq. 4-5, Algorithms 1-2), backward: the
                 gradient gic_probe_loss forms with the loss

training_loss() composes the three; loss.backward() then gives d loss / d
theta through the hand-written kernels.
"""
import torch

from . import gicpcg as G


class GnnForward(torch.autograd.Function):
    """g (float32, one value per entry of tril(A)) from theta. ws: a training
    workspace (gic_gnn_workspace_size with training = 1) that keeps this
    forward's activations for the backward; None allocates one per call. A
    workspace passed in must not serve another forward before this one's
    backward has run."""

    @staticmethod
    def forward(ctx, theta, h, P, x9, e0, ngraphs=1, ws=None):
        ws = ws if ws is not None else G.gnn_workspace(h, P, ngraphs, training=True)
        th = theta.detach().contiguous()
        g = G.gnn_forward_train(h, P, th, x9, e0, ws, ngraphs=ngraphs)
        ctx.h, ctx.P, ctx.ngraphs, ctx.ws = h, P, ngraphs, ws
        ctx.save_for_backward(th, x9, e0)
        return g

    @staticmethod
    def backward(ctx, dg):
        th, x9, e0 = ctx.saved_tensors
        dth = G.gnn_backward(ctx.h, ctx.P, th, x9, e0, dg.contiguous(), ctx.ws, ngraphs=ctx.ngraphs)
        return dth, None, None, None, None, None, None


class CorrectScaled(torch.autograd.Function):
    """L^ from L^_IC (scaled units, float32) and g (Eq. 2 with the positive
    diagonal map); differentiable in g."""

    @staticmethod
    def forward(ctx, g, h, P, LIChat):
        Lhat = G.gnn_correct_scaled(h, P, LIChat, g.detach().contiguous())
        ctx.h, ctx.P = h, P
        ctx.save_for_backward(Lhat)
        return Lhat

    @staticmethod
    def backward(ctx, dLhat):
        (Lhat,) = ctx.saved_tensors
        return G.gnn_correct_backward(ctx.h, ctx.P, Lhat, dLhat.contiguous()), None, None, None


class ProbeLoss(torch.autograd.Function):
    """The batch-mean probe loss (a 0-d float32 tensor) of L^ against A^ with
    probes Z (m x n float32); its gradient in L^ is formed with the loss."""

    @staticmethod
    def forward(ctx, Lhat, h, P, Ahat, Z, ngraphs=1, ws=None):
        loss, dL = G.probe_loss(h, P, Ahat, Lhat.detach().contiguous(), Z, ngraphs=ngraphs, grad=True, ws=ws)
        ctx.save_for_backward(dL)
        return loss[ngraphs].clone()

    @staticmethod
    def backward(ctx, gout):
        (dL,) = ctx.saved_tensors
        return dL * gout, None, None, None, None, None, None


def training_loss(theta, h, P, x9, e0, LIChat, Ahat, Z, ngraphs=1, gnn_ws=None, probe_ws=None):
    """The training objective of one batch as a differentiable function of
    theta: probe loss of the GNN-corrected factor."""
    g = GnnForward.apply(theta, h, P, x9, e0, ngraphs, gnn_ws)
    Lhat = CorrectScaled.apply(g, h, P, LIChat)
    return ProbeLoss.apply(Lhat, h, P, Ahat, Z, ngraphs, probe_ws)

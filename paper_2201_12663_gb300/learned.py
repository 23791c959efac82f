"""Learned subspace proposal: training data from the method itself, training with the library's
own network kernels, and the proposal -> one subspace iteration -> acceptance test -> fallback
path.  This module only orders library calls; every numeric step (features, network forward and
backward, Adam, targets, proposal basis, reductions) runs in the library's kernels.

The features describe a Gaussian sum sum_k c_k exp(-a_k |x - x_k|^2) through its parameters, so
the caller passes them (centres R x 3, log a_k, c_k as CUDA float64 tensors) next to the factors.
"""
import math

from . import (Mlp, RHOSVD_ERR_SKETCH, rhosvd_c2t, rhosvd_c2t_start, rhosvd_chebyshev, rhosvd_features,
               rhosvd_proj_target, rhosvd_proposal_basis)

# ranges of the features: the centre box and exponent range of the Gaussian-sum distribution
FEATURE_BOX = dict(cbox=5.0, la=math.log(0.5), lb=math.log(20.0))
NPROP = 32          # proposal width (coefficient vectors)


class LearnedProposal:
    """Network + discrete Chebyshev basis of one grid (n points on [-b, b])."""

    def __init__(self, n, b=10.0, batch_max=256, seed=0, device="cuda", box=None):
        self.n = int(n)
        self.b = float(b)
        self.box = dict(box or FEATURE_BOX)
        self.mlp = Mlp(batch_max=batch_max, seed=seed)
        self.QT = rhosvd_chebyshev(self.n, self.b, device)

    def features(self, params):
        return rhosvd_features(params["centres"], params["loga"], params["c"], **self.box)

    def target(self, Z, r):
        return rhosvd_proj_target(self.QT, Z, min(int(r), NPROP))

    def propose(self, feats):
        """Three n x 32 start bases from the (3, 128) features of one tensor."""
        import torch
        X = torch.zeros(8, 128, dtype=torch.float32, device=feats.device)
        X[:3] = feats
        Y = self.mlp.forward(X)
        return [rhosvd_proposal_basis(self.QT, Y[l]) for l in range(3)]


def training_set(prop, instances, **opts):
    """(X, G) for a list of instances (U, xi, params): features per mode, and the target
    projector of the method's own leading basis (its first min(32, r_l) columns)."""
    import torch
    X, G = [], []
    for U, xi, params in instances:
        res = rhosvd_c2t(U, xi, **opts)
        info = res.info()
        if info.status != 0:
            continue
        feats = prop.features(params)
        for l in range(3):
            X.append(feats[l])
            G.append(prop.target(res.Z[l], max(1, info.r[l])))
    return torch.stack(X), torch.stack(G)


def train(prop, X, G, steps=200, batch=64, lr=1e-3, seed=0):
    """Adam steps on random mini-batches (multiples of 8); returns the loss after each step."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    N = X.shape[0]
    losses = []
    for _ in range(steps):
        idx = torch.randint(0, N, (batch,), generator=g).to(X.device)
        loss = prop.mlp.train_step(X[idx].contiguous(), G[idx].contiguous(), lr)
        losses.append(loss)
    return [float(x.item()) for x in losses]


def reduce_learned(prop, U, xi, params, attempts=(0, 1), **opts):
    """Proposal -> acceptance test -> subspace iteration -> fallback.  Each entry of attempts is a
    rhosvd_c2t_start call with that many subspace iterations (0: the proposal itself, one pass
    over U for B = Q0^T U and the residual).  An attempt is accepted when the measured residual
    energy meets the eps rule (status 0); when it falls short of 1 - eps^2 (status
    RHOSVD_ERR_SKETCH) the next attempt runs, and after the last one the plain rhosvd_c2t.
    Returns (result, fallback_used)."""
    Q0 = prop.propose(prop.features(params))
    for it in attempts:
        res = rhosvd_c2t_start(U, xi, Q0, iters=it, **opts)
        if res.info().status != RHOSVD_ERR_SKETCH:
            return res, False
    return rhosvd_c2t(U, xi, **opts), True

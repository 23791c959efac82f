"""The learned subspace proposal on the GPU: its kernels against the CPU oracle (oracle/mlp.py),
the start-basis reduction against the plain one, the fallback, and training.

Tolerances: features and the basis are FP32 / FP64 definitions (1e-6, 1e-12).  The network
rounds every product's operands to BF16 like the oracle (oracle.mlp with round_bf16=True) but
keeps activations in FP32 (the oracle in FP64), so a few near-tie values round to different
BF16 neighbours: outputs agree to ~2e-4 relative (checked at 1e-3), gradients in relative
Frobenius norm (2e-2) and direction (cosine >= 0.999)."""
import math

import numpy as np
import pytest

import workloads
from oracle import mlp as om
from tests import tensor_utils as tu

pytestmark = pytest.mark.gpu


def _rand_params(seed, R):
    g = np.random.default_rng(seed)
    centres = g.uniform(-5, 5, (R, 3))
    loga = g.uniform(math.log(0.5), math.log(20.0), R)
    c = g.uniform(0.1, 1.0, R)
    return centres, loga, c


def test_features_and_basis_match_oracle(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    centres, loga, c = _rand_params(0, 777)
    f = P.rhosvd_features(torch.from_numpy(centres).cuda(), torch.from_numpy(loga).cuda(),
                          torch.from_numpy(c).cuda(), 5.0, math.log(0.5), math.log(20.0))
    ref = om.features(centres, loga, c, 5.0, math.log(0.5), math.log(20.0))
    assert np.allclose(f.cpu().numpy(), ref, rtol=1e-6, atol=1e-7)
    Q = P.rhosvd_chebyshev(256, 10.0).cpu().numpy()
    assert np.abs(Q - om.chebyshev_basis(256, 10.0)).max() < 1e-12
    Z, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((256, 21)))
    G = P.rhosvd_proj_target(torch.from_numpy(Q).cuda().t().contiguous().t(), torch.from_numpy(Z).cuda().t().contiguous().t(), 21)
    assert np.allclose(G.cpu().numpy().reshape(64, 64, order="F"), om.target(Q, Z), atol=1e-6)


def _oracle_params(vec):
    out, o = [], 0
    for i in range(4):
        a, b = om.DIMS[i], om.DIMS[i + 1]
        W = vec[o:o + a * b].astype(np.float64).reshape(b, a)
        o += a * b
        bb = vec[o:o + b].astype(np.float64)
        o += b
        out.append((W, bb))
    return out


def test_forward_and_gradients_match_oracle(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    net = P.Mlp(batch_max=16, seed=3)
    params = _oracle_params(net.params())
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 0.06, (16, 128)).astype(np.float32)
    Qb = om.chebyshev_basis(128, 10.0)
    G = np.stack([om.target(Qb, np.linalg.qr(rng.standard_normal((128, 12)))[0]) for _ in range(16)])
    Xd = torch.from_numpy(X).cuda()
    Y = net.forward(Xd).cpu().numpy()
    Yo, cache = om.forward(params, X.astype(np.float64))
    assert np.linalg.norm(Y - Yo) <= 1e-3 * np.linalg.norm(Yo)
    Gd = torch.from_numpy(G.reshape(16, -1, order="C").astype(np.float32))
    # G[s] is symmetric, so its row-major flattening equals the column-major G[i + 64 i']
    loss = net.gradients(Xd, Gd.cuda()).item()
    lo, dY = om.loss_and_grad_output(Yo, G)
    assert abs(loss - lo) <= 1e-3 * lo
    grads = om.backward(params, cache, dY)
    gv = net.params(which=1)
    ref = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    rel = np.linalg.norm(gv - ref) / np.linalg.norm(ref)
    cos = float(gv @ ref / (np.linalg.norm(gv) * np.linalg.norm(ref)))
    assert rel <= 2e-2 and cos >= 0.999, (rel, cos)
    net.close()


def _instance(P, n, R, seed):
    U, xi, params = workloads.gaussian_sum_device(n, R, seed)
    return U, xi, params


OPTS = dict(eps=1e-6, r_max=128, oversample=32, seed=5)


def test_start_from_the_plain_basis_matches_plain(rhosvd_cuda):
    P = rhosvd_cuda
    U, xi, _ = _instance(P, 384, 600, 7)
    a = P.rhosvd_c2t(U, xi, **OPTS)
    ia = a.info()
    assert ia.status == 0
    k0 = max(ia.r[l] for l in range(3))            # columns past r_l of Z are zero; pivoting drops them
    Q0 = [a.Z[l][:, :k0].t().contiguous().t() for l in range(3)]
    b = P.rhosvd_c2t_start(U, xi, Q0, iters=0, **OPTS)
    ib = b.info()
    assert ib.status == 0, P.rhosvd_strerror(ib.status)
    ra = [ia.r[l] for l in range(3)]
    rb = [ib.r[l] for l in range(3)]
    assert all(abs(x - y) <= 1 for x, y in zip(ra, rb))
    if ra == rb:
        ba = a.beta[: ra[0] * ra[1] * ra[2]].cpu().numpy().reshape(ra, order="F")
        bb = b.beta[: rb[0] * rb[1] * rb[2]].cpu().numpy().reshape(rb, order="F")
        Za = [a.Z[l][:, : ra[l]].cpu().numpy() for l in range(3)]
        Zb = [b.Z[l][:, : rb[l]].cpu().numpy() for l in range(3)]
        assert tu.tucker_rel_diff(bb, Zb, ba, Za) <= 1e-6


def test_poor_start_falls_back_to_plain(rhosvd_cuda):
    P = rhosvd_cuda
    from paper_2201_12663_gb300 import learned
    import torch
    U, xi, params = _instance(P, 384, 600, 8)
    prop = learned.LearnedProposal(384, batch_max=16, seed=1)      # untrained network
    res, fell_back = learned.reduce_learned(prop, U, xi, params, **OPTS)
    plain = P.rhosvd_c2t(U, xi, **OPTS)
    assert fell_back
    assert res.info().status == 0
    assert [res.info().r[l] for l in range(3)] == [plain.info().r[l] for l in range(3)]
    prop.mlp.close()


def test_training_lowers_the_loss_and_gains_over_random_and_untrained(rhosvd_cuda):
    """A small training run on the method's own bases, then what it gains, measured by the
    library's residual (fixed ranks 32, no deflation sketch: the energy outside the 32-vector
    subspace) on held-out instances.  Without a pass over U (iters 0) the learned subspace
    captures far more energy than a random one of the same width, and more than the untrained
    network's; after one subspace iteration (iters 1) a random start is as good or better (the
    64-polynomial space cannot resolve the narrow Gaussians) -- recorded, not asserted."""
    P = rhosvd_cuda
    from paper_2201_12663_gb300 import learned
    import torch
    n = 256
    prop = learned.LearnedProposal(n, batch_max=64, seed=2)
    fresh = learned.LearnedProposal(n, batch_max=64, seed=2)         # same initial weights, untrained
    train_set = [_instance(P, n, R, s) for s, R in zip(range(100, 124), np.linspace(300, 900, 24).astype(int))]
    X, G = learned.training_set(prop, train_set, **OPTS)
    losses = learned.train(prop, X, G, steps=150, batch=64, lr=1e-3)
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10]), (losses[:3], losses[-3:])
    cap = {}
    g = torch.Generator(device="cuda").manual_seed(0)
    for s in range(200, 206):
        U, xi, params = _instance(P, n, 500, s)
        starts = {"learned": prop.propose(prop.features(params)),
                  "untrained": fresh.propose(fresh.features(params)),
                  "random": [torch.randn(32, n, generator=g, device="cuda", dtype=torch.float64).t() for _ in range(3)]}
        for k, Q0 in starts.items():
            for it in (0, 1):
                res = P.rhosvd_c2t_start(U, xi, Q0, iters=it, deflate=-1, **{**OPTS, "ranks": (32, 32, 32)})
                info = res.info()
                cap.setdefault((k, it), []).append(np.mean([info.resid[l] / info.total[l] for l in range(3)]))
    missed = {k: float(np.mean(v)) for k, v in cap.items()}
    print("energy missed by the 32-vector subspace:", missed)
    assert missed[("learned", 0)] < 0.5 * missed[("random", 0)], missed
    assert missed[("learned", 0)] < missed[("untrained", 0)], missed
    prop.mlp.close()
    fresh.mlp.close()


def test_checkpoint_resumes_training_exactly(rhosvd_cuda, tmp_path):
    """rhosvd_mlp_save / rhosvd_mlp_load: train a few Adam steps, save, train on; a second handle
    loaded from the file and trained on the same batches gives the same losses and weights bit
    for bit (weights, both Adam moments and the step count are restored: without the moments or
    the bias-correction step the first resumed update would differ).  The file follows the
    documented layout (tag, widths, step, per layer W, b, m(W), v(W), m(b), v(b))."""
    P = rhosvd_cuda
    import torch
    g = torch.Generator(device="cuda").manual_seed(5)
    batches = [(torch.rand(16, 128, generator=g, device="cuda"), torch.rand(16, 4096, generator=g, device="cuda"))
               for _ in range(6)]
    a = P.Mlp(batch_max=16, seed=9)
    for X, G in batches[:3]:
        a.train_step(X, G, 1e-3)
    path = str(tmp_path / "mlp.bin")
    a.save(path)
    w_saved = a.params()
    la = [float(a.train_step(X, G, 1e-3).item()) for X, G in batches[3:]]
    a.status()
    b = P.Mlp(batch_max=16, seed=123)            # other initial weights, overwritten by the load
    b.load_state(path)
    assert np.array_equal(b.params(), w_saved)
    lb = [float(b.train_step(X, G, 1e-3).item()) for X, G in batches[3:]]
    b.status()
    assert la == lb, (la, lb)
    assert np.array_equal(a.params(), b.params())
    # the documented layout, read back with numpy
    raw = open(path, "rb").read()
    assert raw[:8] == b"RHMLPv01"
    hdr = np.frombuffer(raw[8:32], dtype="<i4")
    assert hdr.tolist() == [4, 128, 512, 512, 512, 2048]
    assert int(np.frombuffer(raw[32:40], dtype="<i8")[0]) == 3
    body = np.frombuffer(raw[40:], dtype="<f4")
    dims = hdr[1:]
    o, got = 0, []
    for i in range(4):
        wsz, bsz = int(dims[i] * dims[i + 1]), int(dims[i + 1])
        got.append(body[o:o + wsz]); o += wsz
        got.append(body[o:o + bsz]); o += bsz
        o += 2 * wsz + 2 * bsz                     # the Adam moments
    assert o == body.size
    assert np.array_equal(np.concatenate(got), w_saved)
    with pytest.raises(P.RhosvdError):
        b.load_state(str(tmp_path / "missing.bin"))
    a.close()
    b.close()

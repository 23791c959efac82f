"""The batched form (rhosvd_c2t_batched): tensors of uneven n and R in one call, scheduled on
concurrent stream lanes and replayed as one cached CUDA graph.  Every result must equal, bit for
bit, what one rhosvd_c2t call per tensor gives (same kernels, same inputs, deterministic
reductions), on the first call, on a replay of the cached graph, and for any lane count."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

SHAPES = [(96, 40, 0), (128, 200, 1), (256, 300, 2), (200, 700, 3), (160, 150, 4), (256, 64, 5), (320, 500, 6)]
OPT = dict(eps=1e-6, r_max=128, oversample=32, seed=11)


def _tensors(P):
    import torch
    out = []
    for n, R, seed in SHAPES:
        cp = workloads.gaussian_sum(n, R, seed)
        out.append(([P.to_device_factor(u) for u in cp.U], torch.from_numpy(cp.xi).cuda()))
    return out


def _read(res):
    info = res.info()
    r = [info.r[l] for l in range(3)]
    return dict(status=info.status, r=r, tail=[info.tail[l] for l in range(3)],
                beta=res.beta[: r[0] * r[1] * r[2]].cpu().numpy(),
                Z=[res.Z[l][:, : r[l]].cpu().numpy() for l in range(3)],
                sigma=res.sigma.cpu().numpy())


def _same(a, b):
    assert a["status"] == 0 and b["status"] == 0
    assert a["r"] == b["r"]
    assert a["tail"] == b["tail"]
    assert np.array_equal(a["beta"], b["beta"])
    assert np.array_equal(a["sigma"], b["sigma"])
    for l in range(3):
        assert np.array_equal(a["Z"][l], b["Z"][l])


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_single_calls(rhosvd_cuda, precision):
    P = rhosvd_cuda
    import torch
    ts = _tensors(P)
    single = [_read(P.rhosvd_c2t(U, xi, precision=precision, **OPT)) for U, xi in ts]
    for lanes in (0, 3):
        outs, call = P.rhosvd_c2t_batched(ts, lanes=lanes, precision=precision, **OPT)
        torch.cuda.synchronize()
        for a, b in zip(single, outs):
            _same(a, _read(b))
        for o in outs:                       # replay of the cached graph
            o.beta.fill_(np.nan)
        call.run()
        torch.cuda.synchronize()
        for a, b in zip(single, outs):
            _same(a, _read(b))


def test_batched_latency_record(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    ts = _tensors(P)
    prev = P.rhosvd_batch_latency_enable(True)
    try:
        outs, call = P.rhosvd_c2t_batched(ts, lanes=4, **OPT)
        lat = P.rhosvd_batch_latency_read(len(ts))
    finally:
        P.rhosvd_batch_latency_enable(bool(prev))
    torch.cuda.synchronize()
    assert all(np.isfinite(x) and x > 0 for x in lat)
    assert all(o.info().status == 0 for o in outs)


_oracle_cache = {}


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_members_match_the_oracle(rhosvd_cuda, precision):
    """Two members of a batch, one of the batched workload's largest kind (n = 1024, R = 4200),
    against the oracle's exact RHOSVD: ranks (+-1 only at a threshold tie), tails, sigma and the
    Tucker tensor to 1e-6, as for single calls (tests/test_gpu_parity.py)."""
    import oracle
    from tests.test_gpu_parity import assert_rank_parity, assert_sigma_parity, assert_tail_parity, oracle_at_ranks
    from tests import tensor_utils as tu
    P = rhosvd_cuda
    import torch
    shapes = [(1024, 4200, 21), (256, 300, 2), (128, 200, 1), (512, 1500, 9)]
    opt = dict(eps=1e-6, r_max=160, oversample=32, seed=13)
    cps = [workloads.gaussian_sum(n, R, s) for n, R, s in shapes]
    ts = [([P.to_device_factor(u) for u in cp.U], torch.from_numpy(cp.xi).cuda()) for cp in cps]
    outs, _ = P.rhosvd_c2t_batched(ts, lanes=0, precision=precision, with_V=False, **opt)
    torch.cuda.synchronize()
    for i in (0, 1):
        if i not in _oracle_cache:
            _oracle_cache[i] = oracle.c2t_threads(cps[i].U, cps[i].xi, eps=opt["eps"])
        o = _oracle_cache[i]
        info = outs[i].info()
        assert info.status == 0, P.rhosvd_strerror(info.status)
        r = [info.r[l] for l in range(3)]
        g = dict(info=info, ranks=r, sigma=outs[i].sigma.cpu().numpy(),
                 beta=outs[i].beta[: r[0] * r[1] * r[2]].cpu().numpy().reshape(r, order="F"),
                 Z=[outs[i].Z[l][:, : r[l]].cpu().numpy() for l in range(3)])
        assert_rank_parity(g, o, opt["eps"])
        assert_sigma_parity(g, o, [shapes[i][0]] * 3)
        oc = o if r == o["ranks"] else oracle_at_ranks(cps[i].U, cps[i].xi, o, r)
        assert_tail_parity(g, oc, opt["eps"], True)
        d = tu.tucker_rel_diff(g["beta"], g["Z"], oc["beta"], oc["Z"])
        print(f"batch member {shapes[i]} precision={precision}: Tucker vs oracle {d:.3e}")
        assert d <= 1e-6, (i, d)

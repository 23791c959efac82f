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

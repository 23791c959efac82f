"""Replayable call sequences (rhosvd_graph_begin/end/launch): a captured Hadamard product + RHOSVD
replayed on new inputs written into the captured buffers gives bit for bit what direct calls
give, and the library's launch counter advances by the captured kernels at every replay."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_direct_calls(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    n, Ra, Rb = 160, 12, 10
    A0, B0 = workloads.gaussian_sum(n, Ra, 1), workloads.gaussian_sum(n, Rb, 2)
    A1, B1 = workloads.gaussian_sum(n, Ra, 3), workloads.gaussian_sum(n, Rb, 4)
    dev = lambda cp: ([P.to_device_factor(u) for u in cp.U], torch.from_numpy(cp.xi).cuda())
    Ua, xa = dev(A0)
    Ub, xb = dev(B0)
    R = Ra * Rb
    Uc = [torch.empty(R, n, dtype=torch.float64, device="cuda").t() for _ in range(3)]
    xc = torch.empty(R, dtype=torch.float64, device="cuda")
    kw = dict(eps=1e-7, r_max=96, oversample=32, seed=5, precision=1)
    ws = torch.empty(P.rhosvd_c2t_workspace_size(P.make_cp(Uc, xc), P.make_opts(**kw)), dtype=torch.uint8,
                     device="cuda")
    out = P.alloc_tucker([n, n, n], R, 96, "cuda")
    s = torch.cuda.Stream()

    def step():
        P.rhosvd_cp_hadamard(Ua, xa, Ub, xb, U_out=Uc, xi_out=xc)
        P.rhosvd_c2t(Uc, xc, out=out, workspace=ws, **kw)

    with torch.cuda.stream(s):
        step()
        torch.cuda.synchronize()
        g = P.rhosvd_capture(step, s)
        for cpA, cpB in ((A1, B1), (A0, B0)):
            for l in range(3):
                Ua[l].copy_(P.to_device_factor(cpA.U[l]))
                Ub[l].copy_(P.to_device_factor(cpB.U[l]))
            xa.copy_(torch.from_numpy(cpA.xi))
            xb.copy_(torch.from_numpy(cpB.xi))
            c0 = P.rhosvd_launch_count()
            g.replay(s)
            torch.cuda.synchronize()
            c1 = P.rhosvd_launch_count()
            info = out.info()
            r = list(info.r)
            got = (out.beta[: r[0] * r[1] * r[2]].clone(), [z.clone() for z in out.Z], out.sigma.clone())
            step()
            torch.cuda.synchronize()
            assert list(out.info().r) == r and info.status == 0
            assert torch.equal(got[0], out.beta[: r[0] * r[1] * r[2]])
            assert all(torch.equal(a, b) for a, b in zip(got[1], out.Z))
            assert torch.equal(got[2], out.sigma)
            assert c1 - c0 > 50
        g.close()


def test_graph_rejects_the_null_stream(rhosvd_cuda):
    P = rhosvd_cuda
    import ctypes
    L = P.load()
    assert L.rhosvd_graph_begin(None) == P.RHOSVD_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert L.rhosvd_graph_end(None, ctypes.byref(h)) == P.RHOSVD_ERR_INVALID_ARG
    assert L.rhosvd_graph_destroy(None) == P.RHOSVD_OK

"""rhosvd_c2t_noalloc, the entry point for callers that cannot allocate device memory (their
host application owns every device allocation, or they must not risk the synchronisation
cudaMalloc/cudaFree may cause).  It takes its scratch space from a static device array
instead of a caller workspace.  Checked through the C ABI against rhosvd_c2t on the same
input, on two calls in a row; between them a different problem (other sizes, the mixed form)
runs through the same array, so the second checked call starts from another call's leftovers
in a different layout, not from a zero-initialised array or the same values.

This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

import workloads
from tests import tensor_utils as tu

pytestmark = pytest.mark.gpu

OPTS = dict(eps=1e-7, r_max=160, oversample=32, seed=99)


def _hadamard_input(P):
    import torch
    A = workloads.gaussian_sum(256, 24, 0)
    B = workloads.gaussian_sum(256, 20, 1)
    Ua = [P.to_device_factor(u) for u in A.U]
    Ub = [P.to_device_factor(u) for u in B.U]
    xa = torch.from_numpy(A.xi).cuda()
    xb = torch.from_numpy(B.xi).cuda()
    return P.rhosvd_cp_hadamard(Ua, xa, Ub, xb)


def _read(res):
    info = res.info()
    r = [info.r[l] for l in range(3)]
    beta = res.beta[: r[0] * r[1] * r[2]].cpu().numpy().reshape(r, order="F")
    Z = [res.Z[l][:, : r[l]].cpu().numpy() for l in range(3)]
    return info, r, beta, Z, res.sigma.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_on_two_calls(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    Uc, xc = _hadamard_input(P)
    need = P.rhosvd_c2t_workspace_size(P.make_cp(Uc, xc), P.make_opts(**OPTS))
    assert 0 < need <= P.RHOSVD_NOALLOC_SCRATCH_BYTES

    ref = P.rhosvd_c2t(Uc, xc, **OPTS)
    info_r, r_ref, beta_r, Z_r, sig_r = _read(ref)
    assert info_r.status == 0

    # the problem run between the two checked calls: other n and R, the mixed form
    Cg = workloads.gaussian_sum(192, 333, 4)
    Ug = [P.to_device_factor(u) for u in Cg.U]
    xg = torch.from_numpy(Cg.xi).cuda()
    opts_g = dict(eps=1e-6, r_max=128, oversample=24, seed=5, precision=1)
    ref_g = P.rhosvd_c2t(Ug, xg, **opts_g)
    info_rg, r_g, beta_g, Z_g, _ = _read(ref_g)
    assert info_rg.status == 0, P.rhosvd_strerror(info_rg.status)
    assert info_rg.direct[0] == 0                    # a sketched mode (n = 192 > k = 152)
    out_g = P.alloc_tucker([192, 192, 192], 333, opts_g["r_max"])

    out = P.alloc_tucker([256, 256, 256], Uc[0].shape[1], OPTS["r_max"])
    for call in range(2):
        if call == 1:
            P.rhosvd_c2t_noalloc(Ug, xg, out_g, **opts_g)
            info_g, rr, bb, ZZ, _ = _read(out_g)
            assert info_g.status == 0 and rr == r_g
            assert tu.tucker_rel_diff(bb, ZZ, beta_g, Z_g) <= 1e-6
        out.beta.fill_(np.nan)
        for z in out.Z:
            z.fill_(np.nan)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        P.rhosvd_c2t_noalloc(Uc, xc, out, **OPTS)
        torch.cuda.synchronize()
        used = free_before - torch.cuda.mem_get_info()[0]
        if call == 0:
            # the one-time set-up may load the library's device code, which brings the static
            # scratch array into device memory; nothing beyond that array
            assert used <= P.RHOSVD_NOALLOC_SCRATCH_BYTES + (8 << 20), used
        else:
            assert used == 0, used                               # later calls take no device memory
        info, r, beta, Z, sig = _read(out)
        assert info.status == 0, P.rhosvd_strerror(info.status)
        assert r == r_ref, (call, r, r_ref)
        assert tu.tucker_rel_diff(beta, Z, beta_r, Z_r) <= 1e-6
        assert np.allclose(sig, sig_r, rtol=1e-12, atol=0)
        for l in range(3):
            assert abs(info.tail[l] - info_r.tail[l]) <= 1e-9 * info_r.tail[l]


def test_noalloc_rejects_problems_beyond_its_scratch(rhosvd_cuda):
    P = rhosvd_cuda
    import torch
    n, R = 1024, 4096                       # needs far more than the static scratch
    U = [torch.zeros(R, n, dtype=torch.float64, device="cuda").t() for _ in range(3)]
    xi = torch.ones(R, dtype=torch.float64, device="cuda")
    need = P.rhosvd_c2t_workspace_size(P.make_cp(U, xi), P.make_opts(**OPTS))
    assert need > P.RHOSVD_NOALLOC_SCRATCH_BYTES
    out = P.alloc_tucker([n, n, n], R, OPTS["r_max"])
    with pytest.raises(P.RhosvdError) as e:
        P.rhosvd_c2t_noalloc(U, xi, out, **OPTS)
    assert e.value.code == P.RHOSVD_ERR_SCRATCH_LIMIT
    assert "scratch" in P.rhosvd_strerror(P.RHOSVD_ERR_SCRATCH_LIMIT)

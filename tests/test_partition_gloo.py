"""The term partition of one reduction over ranks (no multi-GPU code is built; this pins the
algebra a sharded form would rest on): with the R terms split into blocks, one per rank, the
normalisation, the projections V = Z^T U~ and the Khatri-Rao core are term-local or a sum over
terms, so each rank computes its block and one all-reduce (sum) of the n x k sketch, of the
n x n side Gram and of the r1 x r2 x r3 core gives the unpartitioned results.  Checked on two
gloo ranks on the CPU against the oracle's whole-tensor routines (Sec. 2.1 normalisation,
Prop. 2.2 projection and core)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _inputs():
    import workloads
    cp = workloads.gaussian_sum(40, 90, 3)
    g = np.random.default_rng(5)
    omega = g.choice([-1.0, 1.0], size=(90, 12))        # the sketch's signs, one row a term
    return cp, omega


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cp, omega = _inputs()
        R = cp.xi.shape[0]
        lo, hi = rank * R // world, (rank + 1) * R // world
        U = [u[:, lo:hi] for u in cp.U]
        # normalisation is term-local (Sec. 2.1)
        Un, xin, _, keep = oracle.normalize(U, cp.xi[lo:hi])

        def allsum(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()

        Y = [allsum(Un[l] @ omega[lo:hi]) for l in range(3)]                     # the sketch
        G = [allsum(Un[l] @ Un[l].T) for l in range(3)]                          # side Grams
        # bases from the summed Grams (every rank the same), then the local projections and
        # the local part of the core, summed
        Z = []
        for l in range(3):
            w, v = np.linalg.eigh(G[l])
            Z.append(np.asfortranarray(v[:, ::-1][:, :6]))
        V = [oracle.project(Z[l], Un[l]) for l in range(3)]
        beta = allsum(oracle.core(V, xin))
        q.put((rank, [y.copy() for y in Y], [z.copy() for z in Z], beta.copy(), int(keep.sum())))
    finally:
        dist.destroy_process_group()


def test_term_partition_over_two_ranks_sums_to_the_whole():
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=10) for _ in range(2)), key=lambda t: t[0])
    cp, omega = _inputs()
    Un, xin, _, keep = oracle.normalize(cp.U, cp.xi)
    assert sum(r[4] for r in res) == int(keep.sum())
    for rank, Y, Z, beta, _ in res:
        for l in range(3):
            assert np.allclose(Y[l], Un[l] @ omega, rtol=1e-13, atol=1e-13)
        # the whole tensor's core at the same bases (the bases are the same on both ranks)
        V = [oracle.project(Z[l], Un[l]) for l in range(3)]
        ref = oracle.core(V, xin)
        assert np.allclose(beta, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        # and the bases span the whole tensor's leading side subspaces (the oracle's exact SVDs)
        o = oracle.c2t(cp.U, cp.xi, eps=1e-6)
        for l in range(3):
            r = min(6, o["Z_full"][l].shape[1])
            P1 = Z[l][:, :r] @ Z[l][:, :r].T
            P0 = o["Z_full"][l][:, :r] @ o["Z_full"][l][:, :r].T
            assert np.linalg.norm(P1 - P0) <= 1e-8

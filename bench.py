#!/usr/bin/env python
"""RHOSVD reductions/s on GB300.

Workload ("hadamard_n1024_R64x64"): two seeded rank-64 Gaussian sums on a 1024^3 grid
(centres U[-5,5]^3, exponents log-uniform [0.5,20], weights U[0.1,1], seeds 0 and 1);
one step = their canonical Hadamard product (rank 4096) followed by the RHOSVD
canonical-to-Tucker reduction at eps = 1e-7, i.e. one pass of the whole hot path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is reductions/s with inputs resident in HBM; `e2e`
is the same metric through the C ABI with the step's inputs copied from pinned host memory
and the Tucker result read back inside the timed region.  The inputs (3 MB) are smaller
than L2, so L2 is flushed (a 256 MB write) before every timed step, outside the events.
With --impl reference the CPU oracle is timed instead, on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="hadamard_n1024_R64x64", n=1024, Ra=64, Rb=64, seeds=[0, 1], eps=1e-7,
                r_max=160, oversample=32, grid="[-10,10]^3 cell centres")
PRECISIONS = {"mixed": 1, "plain": 0}
# tensor-core digit-plane products per FP64-class product in the mixed form: 7-digit operands
# with every pair s + t <= 9 (34); the sketch, 7 digits against a +-1 operand (7); the core with
# 4-digit operands, pairs s + t <= 5 (10)
MIXED_PAIRS = {"sketch": 7, "project": 34, "v_hi": 34, "residual": 34, "z_hi": 34, "gram_bbt": 34,
               "cholqr_gram": 34, "cholqr_apply": 34, "core": 10}
# DRAM bytes per launch of a stage's kernel from an ncu capture of the same code (None when the
# kernel has changed since): profiles/chol_cluster_hadamard_n1024_R64x64.md
NCU_TRAFFIC = {"cholqr_chol": 0.951e6}
METRIC = "RHOSVD reductions/s at stated rel. err: mixed/learned vs FP64 plain, 1×GB300"
UNIT = "reductions/s"
FP64_NOMINAL_TFLOPS = 1.25  # GB300 nominal FP64 (CUDA-core and tensor) rate, used only until measured
_FP64 = {}                  # the rate measured in this run by fp64_rate()


def fp64_peak():
    """(FP64 peak in TFLOP/s, where it comes from): the probe's rate measured in this run, else
    the nominal figure."""
    if _FP64.get("probe_tflops"):
        return _FP64["probe_tflops"], "FP64 fma rate measured on this GPU in this run (rhosvd_probe_fp64, of measured)"
    return FP64_NOMINAL_TFLOPS, "GB300 nominal FP64 rate (of fallback: not measured in this run)"


def fp64_rate(P, dev, reps=5):
    """FP64 fma rate of this GPU: the library's probe kernel (eight independent fma chains a
    thread, 152 x 8 blocks of 256 threads), best of `reps` CUDA-event timings after warm-up; and
    cuBLAS DGEMM 4096^3 (torch.matmul in float64) beside it as a comparator."""
    import torch
    blocks, iters = 152 * 8, 4096
    buf = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
    for _ in range(3):
        P.rhosvd_probe_fp64(blocks, iters, buf)
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        P.rhosvd_probe_fp64(blocks, iters, buf)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    probe = blocks * 4096.0 * iters / (best * 1e-3) / 1e12
    x = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    y = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(x, y)
    bestg = float("inf")
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        torch.matmul(x, y)
        b.record()
        torch.cuda.synchronize()
        bestg = min(bestg, a.elapsed_time(b))
    del x, y, buf
    _FP64["probe_tflops"] = probe
    return {"probe_tflops": probe, "probe_ms": best, "cublas_dgemm_4096_tflops": 2 * 4096.0 ** 3 / (bestg * 1e-3) / 1e12,
            "note": "the probe's rate is the denominator of every FP64 roofline in this line; cuBLAS DGEMM is a comparator"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks sampling
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def _oracle_input(wl):
    import workloads
    A, B = workloads.hartree_like_factors(wl["n"], wl["Ra"], wl["Rb"], wl["seeds"])
    return A, B


def oracle_pieces(nsteps, wl=WORKLOAD):
    """One whole oracle reduction of the bench workload cut into `nsteps` consecutive pieces of
    work, in the order of orc_c2t: the Hadamard product and the normalisation; the full SVD of
    each side matrix with its eps-rank (three pieces); the projections V = Z^T U~; the core over
    consecutive slices of the terms (nsteps - 5 slices; the slices' cores are summed in order).
    With fewer than six steps the same six kinds of work are spread over them.  Returns
    (list of callables, state dict); running every callable in order leaves Z, beta, ranks in
    the state."""
    import numpy as np
    import oracle
    A, B = _oracle_input(wl)
    st = {}
    eps = wl["eps"]

    def prep():
        Uc, xc = oracle.cp_hadamard(A.U, A.xi, B.U, B.xi)
        st["Un"], st["xin"], _, _ = oracle.normalize(Uc, xc)
        st["Z"], st["r"] = [None] * 3, [0] * 3

    def svd(l):
        def f():
            sig, Z = oracle.side_svd(st["Un"][l])
            r = oracle.eps_rank(sig, eps)
            st["r"][l] = r
            st["Z"][l] = np.asfortranarray(Z[:, :r])
        return f

    def proj():
        st["V"] = [oracle.project(st["Z"][l], st["Un"][l]) for l in range(3)]
        st["beta"] = np.zeros(tuple(st["r"]), order="F")

    nc = max(1, nsteps - 5)
    R = wl["Ra"] * wl["Rb"]
    cuts = [R * i // nc for i in range(nc + 1)]

    def core(i):
        def f():
            a, b = cuts[i], cuts[i + 1]
            st["beta"] += oracle.core([np.asfortranarray(st["V"][l][:, a:b]) for l in range(3)], st["xin"][a:b])
        return f

    atoms = [prep, svd(0), svd(1), svd(2), proj] + [core(i) for i in range(nc)]
    if nsteps >= len(atoms):
        return atoms, st
    groups = []
    for i in range(nsteps):
        part = atoms[i * len(atoms) // nsteps:(i + 1) * len(atoms) // nsteps]
        groups.append(lambda part=part: [f() for f in part])
    return groups, st


def oracle_full_threads(nthreads, wl=WORKLOAD):
    """One whole oracle reduction of the bench workload on `nthreads` host threads: the three
    side-matrix SVDs and the projections at once (one mode a thread), the core over nthreads
    consecutive slices of the terms at once (summed in slice order).  The oracle's C routines are
    called unchanged (ctypes releases the GIL).  Returns the Tucker tensor, the wall time and the
    per-thread busy time of every piece."""
    import numpy as np
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    A, B = _oracle_input(wl)
    eps = wl["eps"]
    busy = []

    def timed(f, *a):
        t = time.perf_counter()
        out = f(*a)
        busy.append(time.perf_counter() - t)
        return out
    t0 = time.perf_counter()
    Uc, xc = timed(oracle.cp_hadamard, A.U, A.xi, B.U, B.xi)
    Un, xin, _, _ = timed(oracle.normalize, Uc, xc)
    with ThreadPoolExecutor(max_workers=max(3, nthreads)) as ex:
        svd = list(ex.map(lambda l: timed(oracle.side_svd, Un[l]), range(3)))
        r = [oracle.eps_rank(svd[l][0], eps) for l in range(3)]
        Z = [np.asfortranarray(svd[l][1][:, : r[l]]) for l in range(3)]
        V = list(ex.map(lambda l: timed(oracle.project, Z[l], Un[l]), range(3)))
        R = xin.shape[0]
        cuts = [R * i // nthreads for i in range(nthreads + 1)]
        parts = list(ex.map(lambda i: timed(oracle.core, [np.asfortranarray(V[l][:, cuts[i]:cuts[i + 1]])
                                                          for l in range(3)], xin[cuts[i]:cuts[i + 1]]),
                            range(nthreads)))
    beta = np.zeros(tuple(r), order="F")
    for p_ in parts:
        beta += p_
    wall = time.perf_counter() - t0
    return dict(Z=Z, beta=beta, ranks=r, wall=wall, busy=sum(busy))


def nproc():
    try:
        return os.cpu_count()
    except Exception:
        return None


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle, as it stands, on one host core: the K timed steps together perform exactly
    one whole reduction of the bench workload (oracle_pieces), so value = 1 / (sum of the step
    times) reductions/s and ms_per_step is the mean step time.  Warm-up: W untimed repeats of the
    first piece (Hadamard product and normalisation)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps, st = oracle_pieces(args.steps)
    for _ in range(args.warmup):
        steps[0]()
    t_steps = []
    for f in steps:
        t0 = time.perf_counter()
        f()
        t_steps.append(time.perf_counter() - t0)
    total = sum(t_steps)
    value = 1.0 / total
    ms = 1000.0 * total / len(t_steps)
    sample = (f"one whole oracle reduction (Hadamard product, normalisation, three full side-matrix SVDs "
              f"(Householder R + one-sided Jacobi), projections, core over all {WORKLOAD['Ra'] * WORKLOAD['Rb']} "
              f"terms) cut into the {len(t_steps)} timed steps; {total:.1f} s on one core; ranks {st['r']}")
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**WORKLOAD, "precision": "oracle fp64", "l2": "n/a (CPU)"}, "cpu_baseline": cpu,
            "step_seconds": [round(t, 3) for t in t_steps], "host_cores_available": nproc(),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def algorithmic_flops(stage, info, n, R, kin=None):
    """FP64-class flops of one launch of a stage (all three modes), from the ranks it saw; kin is
    the sketch width r_max + oversample (the bench workload's by default)."""
    r = [info.r[l] for l in range(3)]
    k = [info.k[l] for l in range(3)]
    if kin is None:
        kin = WORKLOAD["r_max"] + WORKLOAD["oversample"]
    kin = min(kin, n)
    if stage == "als_contract":
        # one mode a launch: C_l = B_l diag(xi) (V_m2 (.) V_m1)^T, k_l x r_m1 r_m2, R deep; mean
        return sum(2.0 * k[l] * r[(l + 1) % 3] * r[(l + 2) % 3] * R for l in range(3)) / 3
    if stage == "core":
        return 2.0 * r[0] * r[1] * r[2] * R
    if stage == "sketch":
        return sum(2.0 * n * kin * R for _ in range(3))
    if stage == "project":
        return sum(2.0 * k[l] * n * R for l in range(3))
    if stage == "residual":
        return sum(2.0 * n * min(k[l], r[l] + 16) * R + 3.0 * n * R for l in range(3))
    if stage == "gram_bbt":
        return sum(2.0 * k[l] * k[l] * R for l in range(3))
    if stage == "v_hi":
        return sum(2.0 * min(k[l], r[l] + 16) * k[l] * R for l in range(3))
    if stage == "z_hi":
        return sum(2.0 * n * k[l] * min(k[l], r[l] + 16) for l in range(3))
    # CholeskyQR: pass 1 on kin columns, passes 2 and 3 on the m_l kept ones; per launch = mean
    if stage == "cholqr_gram":
        return (sum(2.0 * kin * kin * n for _ in range(3)) + 2 * sum(2.0 * k[l] ** 2 * n for l in range(3))) / 3
    if stage == "cholqr_apply":
        return (sum(2.0 * n * kin * kin for _ in range(3)) + 2 * sum(2.0 * n * k[l] ** 2 for l in range(3))) / 3
    if stage == "cholqr_chol":
        return (sum(kin ** 3 / 3.0 for _ in range(3)) + 2 * sum(k[l] ** 3 / 3.0 for l in range(3))) / 3
    if stage == "cholqr_trinv":
        return (sum(kin ** 3 / 3.0 for _ in range(3)) + 2 * sum(k[l] ** 3 / 3.0 for l in range(3))) / 3
    if stage == "tridiag":
        return sum(4.0 * k[l] ** 3 / 3.0 for l in range(3))
    return None


def tucker_rel_diff_np(beta_a, Z_a, beta_b, Z_b):
    """||T_a - T_b|| / ||T_b|| (numpy, FP64) for orthonormal Tucker factors, via an orthonormal
    basis of span[Z_a Z_b] per mode, so the n^3 tensors are never formed."""
    import numpy as np
    ca, cb = np.asarray(beta_a, dtype=np.float64), np.asarray(beta_b, dtype=np.float64)
    for l in range(3):
        za, zb = np.asarray(Z_a[l], dtype=np.float64), np.asarray(Z_b[l], dtype=np.float64)
        Pm, _ = np.linalg.qr(np.hstack([za, zb]))
        ca = np.moveaxis(np.tensordot(Pm.T @ za, ca, axes=([1], [l])), 0, l)
        cb = np.moveaxis(np.tensordot(Pm.T @ zb, cb, axes=([1], [l])), 0, l)
    return float(np.linalg.norm(ca - cb) / np.linalg.norm(cb))


RSC = dict(workload="newton_long_range_sum_n2048_N1000", n=2048, N=1000, R=20000, seed=0, eps=1e-6, r_max=64,
           oversample=32, sketch_seed=2024, precision="mixed", out_fp32=True)


def rs_collective_leg(P, dev, steps, warmup):
    """The range-separated collective potential: long-range Newton Gaussians (20 a charge,
    exponents e^{2kh}, h = 0.4, k = -19..0) of N = 1000 unit charges at centres U[-8, 8]^3, on
    n = 2048 cell centres of [-10, 10]: R = 20000 terms, eps = 1e-6, the mixed form with FP32
    outputs (Z and beta), and the plain form beside it.  Inputs (983 MB of factors) exceed L2,
    so no flush is needed.  Roofline: the whole reduction against two reads of the factors
    (1.97 GB) at the measured HBM rate; the dominant stage against its own peak."""
    import numpy as np
    import torch
    import workloads
    cp = workloads.newton_long_range_sum(n=RSC["n"], N=RSC["N"], seed=RSC["seed"])
    Ud = [P.to_device_factor(u) for u in cp.U]
    xd = torch.from_numpy(cp.xi).to(dev)
    n, R = RSC["n"], cp.xi.shape[0]
    rec = {**RSC, "l2": "inputs (983 MB) larger than L2: no flush"}
    host = None
    for prec, fp32 in (("mixed", True), ("plain", False)):
        opts = dict(eps=RSC["eps"], r_max=RSC["r_max"], oversample=RSC["oversample"], seed=RSC["sketch_seed"],
                    precision=PRECISIONS[prec], out_fp32=fp32)
        ws = torch.empty(P.rhosvd_c2t_workspace_size(P.make_cp(Ud, xd), P.make_opts(**opts)), dtype=torch.uint8,
                         device=dev)
        out = P.alloc_tucker([n, n, n], R, RSC["r_max"], dev, fp32=fp32)
        for _ in range(max(warmup, 3)):
            P.rhosvd_c2t(Ud, xd, out=out, workspace=ws, **opts)
        info = out.info()
        if info.status != 0:
            rec[prec] = {"status": info.status, "error": P.rhosvd_strerror(info.status)}
            continue
        nst = steps if prec == "mixed" else max(2, steps // 2)
        a = [torch.cuda.Event(enable_timing=True) for _ in range(nst)]
        b = [torch.cuda.Event(enable_timing=True) for _ in range(nst)]
        torch.cuda.synchronize()
        for i in range(nst):
            a[i].record()
            P.rhosvd_c2t(Ud, xd, out=out, workspace=ws, **opts)
            b[i].record()
        torch.cuda.synchronize()
        ms = sum(x.elapsed_time(y) for x, y in zip(a, b)) / nst
        r = [info.r[l] for l in range(3)]
        alg = 2 * 3 * n * R * 8
        hbm = peaks().get("hbm_gbs", 6800.0)
        entry = {"ms": ms, "value": 1000.0 / ms, "unit": UNIT, "ranks": r, "k": [info.k[l] for l in range(3)],
                 "tails": [info.tail[l] for l in range(3)], "status": 0,
                 "roofline_whole": {"bound": "hbm", "algorithmic_bytes": alg, "achieved": alg / (ms * 1e-3) / 1e9,
                                    "peak": hbm, "unit": "GB/s", "frac": alg / (ms * 1e-3) / 1e9 / hbm,
                                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}}
        entry["roofline_dominant"] = stage_roofline(
            P, lambda: P.rhosvd_c2t(Ud, xd, out=out, workspace=ws, **opts), lambda res: res.info(), n, R,
            RSC["r_max"] + RSC["oversample"], prec)
        rec[prec] = entry
        if prec == "mixed":
            cnt = r[0] * r[1] * r[2]
            host = (out.beta[:cnt].double().cpu().numpy().reshape(r, order="F"),
                    [out.Z[l][:, : r[l]].double().cpu().numpy() for l in range(3)], r)
        del ws, out
    if "ms" in rec.get("mixed", {}) and "ms" in rec.get("plain", {}):
        rec["speedup_mixed_vs_plain"] = rec["plain"]["ms"] / rec["mixed"]["ms"]
    rec["_host"] = (host, cp)
    return rec


def rs_collective_oracle_error(host_cp):
    """The rs_collective leg's Tucker error against the oracle: the oracle's truncated bases of
    this workload are stored (tests/golden/newton_n2048_N1000_eps1e-6_Z.npz, written by
    tests/golden/make_full_size.py from oracle/ alone); V = Z^T U~ and the core are rebuilt here
    at the GPU's ranks with the oracle's own routines."""
    import numpy as np
    import oracle
    host, cp = host_cp
    if host is None:
        return {"tucker_rel_diff_vs_oracle": None, "note": "mixed run failed"}
    beta, Z, r = host
    path = os.path.join(ROOT, "tests", "golden", "newton_n2048_N1000_eps1e-6_Z.npz")
    zs = np.load(path)
    Zo = [np.asfortranarray(zs[f"Z{l}"][:, : r[l]]) for l in range(3)]
    if any(Zo[l].shape[1] < r[l] for l in range(3)):
        return {"tucker_rel_diff_vs_oracle": None, "note": f"ranks {r} beyond the stored oracle bases"}
    t0 = time.perf_counter()
    Un, xin, _, _ = oracle.normalize(cp.U, cp.xi)
    Vo = [oracle.project(Zo[l], Un[l]) for l in range(3)]
    bo = oracle.core(Vo, xin)
    return {"vs": "oracle (FP64 CPU, exact SVDs; bases stored, V and core rebuilt by the oracle)",
            "tucker_rel_diff_vs_oracle": tucker_rel_diff_np(beta, Z, bo, Zo), "outputs": "fp32 Z and beta",
            "oracle_rebuild_s": time.perf_counter() - t0}


def tucker_rel_diff_torch(beta_a, Z_a, beta_b, Z_b):
    """||T_a - T_b|| / ||T_b|| for orthonormal Tucker factors, via a common basis per mode
    (measurement aid for the bench line; torch linear algebra on the host, not the product
    path)."""
    import torch
    ca, cb = beta_a.cpu(), beta_b.cpu()
    Za = [z.cpu() for z in Z_a]
    Zb = [z.cpu() for z in Z_b]
    for l in range(3):
        Pm, _ = torch.linalg.qr(torch.cat([Za[l], Zb[l]], dim=1))
        ca = torch.movedim(torch.tensordot(Pm.T @ Za[l], ca, dims=([1], [l])), 0, l)
        cb = torch.movedim(torch.tensordot(Pm.T @ Zb[l], cb, dims=([1], [l])), 0, l)
    return (torch.linalg.norm(ca - cb) / torch.linalg.norm(cb)).item()


BATCH = dict(workload="batched_gaussian_sums_512", count=512, n_choices=[128, 256, 512, 1024],
             R_range=[100, 8000], eps=1e-6, r_max=160, oversample=32, seed=7)


def batched_leg(P, dev, steps, warmup, precision):
    """The batched workload: 512 Gaussian sums of uneven n and R at eps = 1e-6 (factor columns
    evaluated on the device from workloads.gaussian_sum_params), reduced by one batched call
    (stream lanes, one cached CUDA graph) and by a per-tensor launch loop for comparison."""
    import torch
    import workloads
    members = workloads.batched_gaussian_sums(BATCH["count"], n_choices=tuple(BATCH["n_choices"]),
                                              R_range=tuple(BATCH["R_range"]))
    tensors = []
    for n, R, seed in members:
        x, ce, a, c = workloads.gaussian_sum_params(n, R, seed)
        xt = torch.from_numpy(x).to(dev)
        at = torch.from_numpy(a).to(dev)
        U = []
        for l in range(3):
            d = xt[:, None] - torch.from_numpy(ce[:, l].copy()).to(dev)[None, :]
            U.append(torch.exp(-at[None, :] * d * d).t().contiguous().t())     # column-major n x R
        tensors.append((U, torch.from_numpy(c).to(dev)))
    opts = dict(eps=BATCH["eps"], r_max=BATCH["r_max"], oversample=BATCH["oversample"], seed=BATCH["seed"],
                precision=PRECISIONS[precision])
    outs = [P.alloc_tucker([U[l].shape[0] for l in range(3)], U[0].shape[1], BATCH["r_max"], dev)
            for U, _ in tensors]
    call = P.BatchedCall(tensors, outs, lanes=0, device=dev, **opts)
    t0 = time.perf_counter()
    call.run()                                  # autotunes the lane count, builds the graph
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    statuses = [o.info().status for o in outs]
    for _ in range(max(warmup, 1)):
        call.run()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        starts[i].record()
        call.run()
        ends[i].record()
    torch.cuda.synchronize()
    ms_batch = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / steps
    prev = P.rhosvd_batch_latency_enable(True)
    call.run()
    torch.cuda.synchronize()
    lat = sorted(P.rhosvd_batch_latency_read(len(tensors)))
    P.rhosvd_batch_latency_enable(bool(prev))
    # per-tensor launch loop on one stream, one workspace
    need = max(P.rhosvd_c2t_workspace_size(P.make_cp(U, xi), P.make_opts(**opts)) for U, xi in tensors)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    for (U, xi), o in zip(tensors[:8], outs[:8]):
        P.rhosvd_c2t(U, xi, out=o, workspace=ws, **opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for (U, xi), o in zip(tensors, outs):
        P.rhosvd_c2t(U, xi, out=o, workspace=ws, **opts)
    e1.record()
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1)
    ok = sum(1 for s_ in statuses if s_ == 0)
    return {**BATCH, "precision": precision, "tensors_per_s": len(tensors) * 1000.0 / ms_batch,
            "ms_per_batch": ms_batch, "p50_ms": lat[len(lat) // 2], "p99_ms": lat[int(0.99 * (len(lat) - 1))],
            "latency": "completion time since the batch started, per tensor",
            "loop_tensors_per_s": len(tensors) * 1000.0 / ms_loop, "loop_ms": ms_loop,
            "speedup_vs_loop": ms_loop / ms_batch, "status_ok": ok, "first_call_s": t_first,
            "input_gb": sum(3 * U[0].shape[0] * U[0].shape[1] * 8 for U, _ in tensors) / 1e9,
            "l2": "inputs (about 10 GB) larger than L2"}


LEARNED = dict(workload="learned_proposal_n1024_R2000_8000", n=1024, R_range=[2000, 8000], eps=1e-6,
               r_max=160, oversample=32, seed=5, nprop=32, train_seed=10**6, eval_seed=10**6 + 20000,
               batch=256, lr=1e-3, epochs=10)


def _quantiles(v):
    import numpy as np
    v = np.asarray(v, dtype=np.float64)
    return {"p10": float(np.quantile(v, 0.1)), "p50": float(np.quantile(v, 0.5)), "p90": float(np.quantile(v, 0.9))}


def learned_leg(P, dev, n_train, n_eval, precision):
    """The learned-proposal workload (n = 1024, R log-uniform in [2000, 8000], eps = 1e-6): the
    network is trained on the GPU, by the library's own kernels, on the leading bases the method
    without it computes for n_train instances, then evaluated on n_eval held-out seeds.  Reports
    the energy its 32-vector subspace misses (no pass over U, and after one subspace iteration)
    against a random start of the same width and against the best 32-vector subspace, the
    fallback rate of the proposal -> iteration -> plain path at eps, and that path's wall time
    per reduction next to the plain call's."""
    import numpy as np
    import torch
    import workloads
    from paper_2201_12663_gb300 import learned
    L = LEARNED
    opts = dict(eps=L["eps"], r_max=L["r_max"], oversample=L["oversample"], seed=L["seed"],
                precision=PRECISIONS[precision])
    prop = learned.LearnedProposal(L["n"], batch_max=L["batch"], seed=0)
    t0 = time.perf_counter()
    X, G, ranks = [], [], []
    for n, R, s in workloads.learned_instances(n_train, L["train_seed"], L["n"], tuple(L["R_range"])):
        U, xi, params = workloads.gaussian_sum_device(n, R, s, dev)
        res = P.rhosvd_c2t(U, xi, **opts)
        info = res.info()
        if info.status != 0:
            continue
        f = prop.features(params)
        for l in range(3):
            X.append(f[l])
            G.append(prop.target(res.Z[l], max(1, info.r[l])))
        ranks.append([info.r[l] for l in range(3)])
    X, G = torch.stack(X), torch.stack(G)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    steps = max(300, L["epochs"] * X.shape[0] // L["batch"])
    t0 = time.perf_counter()
    losses = learned.train(prop, X, G, steps=steps, batch=L["batch"], lr=L["lr"])
    t_train = time.perf_counter() - t0
    del X, G
    g = torch.Generator(device=dev).manual_seed(0)
    missed = {k: [] for k in ("learned_iters0", "learned_iters1", "random_iters0", "random_iters1", "best_32")}
    fallbacks, path_ok, t_plain, t_path = 0, 0, 0.0, 0.0
    fixed = {**opts, "ranks": (L["nprop"],) * 3, "deflate": -1}
    for n, R, s in workloads.learned_instances(n_eval, L["eval_seed"], L["n"], tuple(L["R_range"])):
        U, xi, params = workloads.gaussian_sum_device(n, R, s, dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = P.rhosvd_c2t(U, xi, **opts)
        info = res.info()
        t_plain += time.perf_counter() - t0
        sig = res.sigma.cpu().numpy()
        for l in range(3):
            tail = float(np.sum(sig[l, L["nprop"]:info.k[l]] ** 2))
            missed["best_32"].append((info.resid[l] + tail) / info.total[l])
        t0 = time.perf_counter()
        res2, fell = learned.reduce_learned(prop, U, xi, params, attempts=(0, 1), **opts)
        st2 = res2.info().status
        t_path += time.perf_counter() - t0
        fallbacks += int(fell)
        starts = {"learned": prop.propose(prop.features(params)),
                  "random": [torch.randn(L["nprop"], n, generator=g, device=dev, dtype=torch.float64).t()
                             for _ in range(3)]}
        for k, Q0 in starts.items():
            for it in (0, 1):
                r3 = P.rhosvd_c2t_start(U, xi, Q0, iters=it, **fixed).info()
                for l in range(3):
                    missed[f"{k}_iters{it}"].append(r3.resid[l] / r3.total[l])
        path_ok += int(st2 == 0)
    q = {k: _quantiles(v) for k, v in missed.items()}
    prop.mlp.close()
    return {**L, "precision": precision, "n_train": n_train, "n_eval": n_eval, "train_samples": 3 * len(ranks),
            "train_steps": steps, "loss_first10": float(np.mean(losses[:10])), "loss_last10": float(np.mean(losses[-10:])),
            "data_s": t_data, "train_s": t_train,
            "eps_ranks_p50": [int(np.median([r[l] for r in ranks])) for l in range(3)],
            "missed_energy": q, "missed_energy_is": "residual energy outside the 32-vector subspace / total, per mode",
            "fallback_rate": fallbacks / max(1, n_eval), "path_status_ok": path_ok,
            "eps_at_50pct_accept_iters1": float(np.sqrt(q["learned_iters1"]["p50"])),
            "ms_per_reduction_plain": 1000.0 * t_plain / max(1, n_eval),
            "ms_per_reduction_learned_path": 1000.0 * t_path / max(1, n_eval),
            "speedup_vs_plain": t_plain / max(t_path, 1e-12),
            "timing": "host wall clock with synchronisation per reduction (the path decides on the host)"}


T2C = dict(workload="t2c_of_the_bench_reduction", eps=1e-5, source="Tucker tensor of the timed reduction (mixed form)")


def t2c_leg(P, out, steps, warmup):
    """Tucker-to-canonical transform of the bench reduction's Tucker tensor at eps = 1e-5 (the
    paper's T2C threshold): CUDA-event time per transform, the canonical rank, and the oracle
    (numpy slice SVDs) timed on the host for the same core.  Algorithmic FP64 work per slice:
    the Golub-Kahan count 4 r1 r2^2 + 8 r2^3 for singular values and left vectors, plus
    2 (n1 r1 + r1 r2 + n2 r2) per kept triple for the factors."""
    import numpy as np
    import torch
    from oracle import t2c as ot
    r, beta3, Z = out.tucker()
    flat = out.beta[: r[0] * r[1] * r[2]]
    cap = r[2] * min(r[0], r[1])
    res = P.rhosvd_t2c(Z, flat, T2C["eps"], cap)
    for _ in range(max(warmup, 1)):
        res = P.rhosvd_t2c(Z, flat, T2C["eps"], cap, out=res)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        P.rhosvd_t2c(Z, flat, T2C["eps"], cap, out=res)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    R, st = res.rank()
    p = res.p[: r[2]].cpu().numpy()
    n = [int(z.shape[0]) for z in Z]
    fl = r[2] * (4.0 * r[0] * r[1] ** 2 + 8.0 * r[1] ** 3) + R * 2.0 * (n[0] * r[0] + r[0] * r[1] + n[1] * r[1])
    bh = beta3.cpu().numpy()
    t0 = time.perf_counter()
    ref = ot.t2c_core(bh, T2C["eps"])
    t_or = time.perf_counter() - t0
    return {**T2C, "core": r, "ms_per_t2c": ms, "canonical_rank": R, "status": st,
            "rank_bound": cap, "p_min_median_max": [int(p.min()), int(np.median(p)), int(p.max())],
            "oracle_rank": ref["R"], "oracle_s": t_or, "oracle_cores": 1,
            "roofline": {"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": fp64_peak()[0],
                         "unit": "TFLOP/s", "frac": fl / (ms * 1e-3) / 1e12 / fp64_peak()[0],
                         "work": "Golub-Kahan count per slice + factor GEMVs",
                         "peak_source": fp64_peak()[1]}}


POLY = dict(workload="newton_cube_n257_eps1e-5", n=257, eps_tucker=1e-5, eps_t2c=1e-5,
            kernel="sinc Newton kernel R=19 (t_k = e^{0.7k}, k=-9..9), long-range part R_l=10 (k<=0)",
            paper_soft={"full": {"R_in": 6859, "tucker": 13, "canonical": 122},
                        "long_range": {"R_in": 1000, "tucker": 8, "canonical": 58}})


def poly_leg(P, steps, warmup, precision):
    """The cube P^(3) = P (.) P (.) P of the discretised Newton kernel at n = 257, eps = 1e-5, as the
    paper's Sec. 5 example: directly (two Hadamard products to rank 19^3 = 6859, or 10^3 for the
    long-range part, then one C2C) and by the Horner scheme (coefficients 0, 0, 0, 1: a reduction
    after every product).  Time per cube (CUDA events around the whole call, which synchronises
    for the ranks), the ranks, and the oracle timed on the host for the same inputs."""
    import numpy as np
    import torch
    import workloads
    from oracle import horner as oh
    out = {**POLY}
    for name, lr in (("full", False), ("long_range", True)):
        cp = workloads.newton_kernel(n=POLY["n"], long_range=lr)
        U = [P.to_device_factor(u) for u in cp.U]
        x = torch.from_numpy(cp.xi).cuda()

        def direct():
            U2, x2 = P.rhosvd_cp_hadamard(U, x, U, x)
            U3, x3 = P.rhosvd_cp_hadamard(U2, x2, U, x)
            return P.rhosvd_c2c(U3, x3, POLY["eps_tucker"], POLY["eps_t2c"], R_max=4000, r_max=64,
                                precision=PRECISIONS[precision])

        def horner():
            return P.rhosvd_cp_horner(U, x, [0, 0, 0, 1], POLY["eps_tucker"], POLY["eps_t2c"], R_max=2000,
                                      r_max=64, precision=PRECISIONS[precision])

        rec = {"roofline_direct": stage_roofline(P, direct, lambda r_: r_[1].info(), POLY["n"], cp.R ** 3, 96,
                                                 precision)}
        for tag, fn in (("direct", direct), ("horner", horner)):
            for _ in range(max(warmup, 1)):
                res = fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                res = fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            if tag == "direct":
                can, tk = res
                R, st = can.rank()
                info = tk.info()
                rec[tag] = {"ms": ms, "R_in": cp.R ** 3, "tucker": [info.r[l] for l in range(3)], "canonical": R,
                            "status": st}
            else:
                rec[tag] = {"ms": ms, "canonical": res.R,
                            "steps": [{"R_in": s_["R_in"], "tucker": s_["r"], "R": s_["R"]} for s_ in res.steps]}
        t0 = time.perf_counter()
        od = oh.power_direct(cp.U, cp.xi, 3, POLY["eps_tucker"], POLY["eps_t2c"])
        t_d = time.perf_counter() - t0
        t0 = time.perf_counter()
        ohr = oh.horner(cp.U, cp.xi, [0, 0, 0, 1], POLY["eps_tucker"], POLY["eps_t2c"])
        t_h = time.perf_counter() - t0
        rec["oracle"] = {"direct_s": t_d, "tucker": od["tucker"]["ranks"], "canonical": od["R"], "horner_s": t_h,
                         "horner_canonical": ohr["R"], "cores": 1}
        rec["speedup_vs_oracle"] = {"direct": t_d * 1e3 / rec["direct"]["ms"], "horner": t_h * 1e3 / rec["horner"]["ms"]}
        out[name] = rec
    return out


# the paper's printed long-range Slater ranks (Tables Tab:random_ranks and Tab:func_ranks):
# lattice -> (Tucker ranks, R_ini, R_comp); context only (other discretisation, garbled captions)
PAPER_SLATER = {
    "random": {(4, 4, 4): ([13] * 3, 192, 56), (6, 6, 6): ([15] * 3, 649, 95), (8, 8, 8): ([19] * 3, 1536, 131),
               (16, 16, 8): ([32, 32, 19], 6141, 253), (16, 16, 16): ([32] * 3, 12288, 380)},
    "func": {(4, 4, 4): ([7] * 3, 256, 25), (6, 6, 6): ([7] * 3, 648, 23), (8, 8, 8): ([7] * 3, 1536, 30),
             (16, 16, 8): ([10, 9, 6], 6144, 47), (16, 16, 16): ([10, 9, 8], 12288, 55)},
}


def rs_leg(P, steps, warmup, precision):
    """Range-separated workloads (Sec. 4.2-4.4): the C2C reduction of the long-range multi-Slater
    lattice sums at eps_Tucker = 1e-3, eps_T2C = 1e-5 (the paper's rank tables; ours beside the
    printed ones), and the interaction energy of 16^3 lattice charges from the C2C-reduced
    long-range Newton potential (Lemma lem:InterEnergy) against the unreduced potential and the
    direct O(N^2) Coulomb sum (the oracle, timed on the host)."""
    import numpy as np
    import torch
    import workloads
    from oracle import energy as oe
    out = {"slater": {}}

    def timed(fn):
        for _ in range(max(warmup, 1)):
            res = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            res = fn()
        e1.record()
        torch.cuda.synchronize()
        return res, e0.elapsed_time(e1) / steps

    for name in ("slater_lattice_random_n384", "slater_lattice_func_n232"):
        C = dict(workloads.CONFIGS[name])
        lattices, eps_t, eps_c = C.pop("lattices"), C.pop("eps_tucker"), C.pop("eps_t2c")
        rows = []
        for L in lattices:
            cp = workloads.multi_slater_long_range(L=L, **C)
            U = [P.to_device_factor(u) for u in cp.U]
            x = torch.from_numpy(cp.xi).cuda()
            (can, tk), ms = timed(lambda: P.rhosvd_c2c(U, x, eps_t, eps_c, R_max=64 * 64, r_max=64,
                                                       precision=PRECISIONS[precision]))
            R, st = can.rank()
            info = tk.info()
            pt = PAPER_SLATER[C["amplitudes"]][tuple(L)]
            rows.append({"lattice": list(L), "N": cp.meta["N"], "R_ini": cp.R, "tucker": [info.r[l] for l in range(3)],
                         "R_comp": R, "status": st or info.status, "ms_c2c": ms,
                         "paper": {"tucker": pt[0], "R_ini": pt[1], "R_comp": pt[2]}})
            del U, x, can, tk
        out["slater"][name] = {"n_points": C["n_cells"] + 1, "eps_tucker": eps_t, "eps_t2c": eps_c, "rows": rows}

    C = dict(workloads.CONFIGS["newton_lattice_energy_N4096"])
    eps_t, eps_c = C.pop("eps_tucker"), C.pop("eps_t2c")
    cp = workloads.newton_lattice_long_range(**C)
    M = cp.meta
    U = [P.to_device_factor(u) for u in cp.U]
    x = torch.from_numpy(cp.xi).cuda()
    z = torch.from_numpy(M["z"]).cuda()
    c2c_e = lambda: P.rhosvd_c2c(U, x, eps_t, eps_c, R_max=160 * 160, r_max=160, precision=PRECISIONS[precision])
    roof_e = stage_roofline(P, c2c_e, lambda r_: r_[1].info(), C["n_cells"] + 1, cp.R, 192, precision)
    (can, tk), ms_c2c = timed(c2c_e)
    R, st = can.rank()
    info = tk.info()
    Ur = [can.U[l][:, :R] for l in range(3)]
    xr = can.xi[:R].contiguous()
    (E_red, _), ms_e_red = timed(lambda: P.rhosvd_rs_energy(Ur, xr, M["idx"], z, M["p0"]))
    (E_full, _), ms_e_full = timed(lambda: P.rhosvd_rs_energy(U, x, M["idx"], z, M["p0"]))
    t0 = time.perf_counter()
    Ec = oe.pair_sum(M["coords"], M["z"], oe.coulomb)
    t_c = time.perf_counter() - t0
    Er, Ef = float(E_red.item()), float(E_full.item())
    out["energy"] = {"workload": "newton_lattice_energy_N4096", "N": M["N"], "R_l": M["R_l"], "R_ini": cp.R,
                     "n_points": C["n_cells"] + 1, "eps_tucker": eps_t, "eps_t2c": eps_c,
                     "tucker": [info.r[l] for l in range(3)], "R_comp": R, "status": st or info.status,
                     "ms_c2c": ms_c2c, "ms_energy_reduced": ms_e_red, "ms_energy_unreduced": ms_e_full,
                     "E_reduced": Er, "E_unreduced": Ef, "E_coulomb_direct": Ec,
                     "rel_diff_reduced_vs_unreduced": abs(Er - Ef) / abs(Ef),
                     "rel_diff_unreduced_vs_coulomb": abs(Ef - Ec) / abs(Ec),
                     "oracle_coulomb_s": t_c, "oracle_cores": 1, "roofline_c2c": roof_e}
    return out


def als_leg(P, steps, warmup, precision):
    """RHOSVD followed by one ALS sweep (Sec. 2.2, eq. can_A_Tuck_als) on the small config
    (gauss_n128_R200, plain FP64, direct modes) and on the bench workload (hadamard_n1024_R64x64,
    the chosen precision for the RHOSVD part): time per call against the RHOSVD alone, the gain
    in captured energy ||beta||^2 over the sweep, and for the small config the relative Tucker
    error before and after, measured on the full 128^3 tensor (torch on the device)."""
    import numpy as np
    import torch
    import workloads
    from oracle import als as oa
    out = {}

    def timed(fn):
        for _ in range(max(warmup, 1)):
            res = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            res = fn()
        e1.record()
        torch.cuda.synchronize()
        return res, e0.elapsed_time(e1) / steps

    def full_err(U, x, res):
        info = res.info()
        r = [info.r[l] for l in range(3)]
        A = torch.einsum("k,ik,jk,mk->ijm", x, *U)
        beta = res.beta[: r[0] * r[1] * r[2]].reshape(r[2], r[1], r[0]).permute(2, 1, 0)
        T = torch.einsum("abc,ia,jb,mc->ijm", beta, *[res.Z[l][:, : r[l]] for l in range(3)])
        return float(torch.linalg.norm(A - T) / torch.linalg.norm(A))

    cases = []
    c0 = workloads.CONFIGS["gauss_n128_R200"]
    cp = workloads.gaussian_sum(c0["n"], c0["R"], c0["seed"])
    cases.append(("gauss_n128_R200", [P.to_device_factor(u) for u in cp.U], torch.from_numpy(cp.xi).cuda(),
                  dict(eps=c0["eps"], r_max=128, precision=0), cp))
    A, B = workloads.hartree_like_factors(WORKLOAD["n"], WORKLOAD["Ra"], WORKLOAD["Rb"], WORKLOAD["seeds"])
    Ua = [P.to_device_factor(u) for u in A.U]
    Ub = [P.to_device_factor(u) for u in B.U]
    Uc, xc = P.rhosvd_cp_hadamard(Ua, torch.from_numpy(A.xi).cuda(), Ub, torch.from_numpy(B.xi).cuda())
    cases.append(("hadamard_n1024_R64x64", Uc, xc, dict(eps=WORKLOAD["eps"], r_max=WORKLOAD["r_max"],
                                                          oversample=WORKLOAD["oversample"], seed=12345,
                                                          precision=PRECISIONS[precision]), None))
    for name, U, x, kw, cp in cases:
        (res, hist), ms_als = timed(lambda: P.rhosvd_c2t_als(U, x, sweeps=1, **kw))
        P.rhosvd_profile_filter("als_contract")
        roof = stage_roofline(P, lambda: P.rhosvd_c2t_als(U, x, sweeps=1, energies=False, **kw)[0],
                              lambda r_: r_.info(), U[0].shape[0], x.shape[0], kw["r_max"] + kw.get("oversample", 32),
                              "plain")
        P.rhosvd_profile_filter(None)
        rh, ms_rh = timed(lambda: P.rhosvd_c2t(U, x, **kw))
        e0, e1 = hist[0][0], hist[-1][1]
        info = res.info()
        rec = {"ms_rhosvd_plus_1_sweep": ms_als, "ms_rhosvd": ms_rh, "ms_sweep": ms_als - ms_rh,
               "ranks": [info.r[l] for l in range(3)], "status": info.status,
               "energy_gain_rel": (e1 - e0) / e0, "energy_steps": [[b, a] for b, a in hist],
               "roofline_contract": roof}
        if cp is not None:
            rec["rel_err_rhosvd"] = full_err(U, x, rh)
            rec["rel_err_als"] = full_err(U, x, res)
            t0 = time.perf_counter()
            oa.c2t_als(cp.U, cp.xi, kw["eps"], sweeps=1)
            rec["oracle_s"] = time.perf_counter() - t0
            rec["oracle_cores"] = 1
        out[name] = rec
    return out


def stage_roofline(P, fn, info_of, n, R, kin, precision):
    """Run fn() once with the library's stage tracing and give the roofline of its dominant
    stage (the one with the most time): algorithmic FP64-class flops of a launch (from the ranks
    the call returned, info_of(result)) over the launch's average duration; tensor-core stages
    against the measured BF16 rate over the digit pairs, FP64 stages against the FP64 rate
    measured in this run (fp64_peak).  None when the stage has no flop model."""
    import torch
    torch.cuda.synchronize()
    P.rhosvd_profile_read()
    P.rhosvd_profile_enable(True)
    res = fn()
    torch.cuda.synchronize()
    P.rhosvd_profile_enable(False)
    prof = P.rhosvd_profile_read()
    if not prof:
        return None
    name, (cnt, ms_tot) = max(prof.items(), key=lambda kv: kv[1][1])
    avg = ms_tot / cnt
    fl = algorithmic_flops(name, info_of(res), n, R, kin)
    out = {"kernel": name, "avg_launch_ms": avg, "launches": cnt, "stage_ms_total": ms_tot,
           "call_ms_traced": sum(v[1] for v in prof.values()),
           "stage_ms": {k: round(v[1], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}}
    if fl is None:
        out.update({"bound": None, "achieved": None, "note": "no flop model for this stage"})
        return out
    ach = fl / (avg * 1e-3) / 1e12
    if precision == "mixed" and name in MIXED_PAIRS:
        peak = peaks().get("bf16_tflops", 1912.0) / MIXED_PAIRS[name]
        out.update({"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "peak_source": f"MEASURED_PEAKS.json bf16_tflops (of measured) / {MIXED_PAIRS[name]} digit pairs"})
    else:
        out.update({"bound": "alu", "achieved": ach, "peak": fp64_peak()[0], "unit": "TFLOP/s",
                    "frac": ach / fp64_peak()[0], "peak_source": fp64_peak()[1]})
    out["algorithmic_flops_per_launch"] = fl
    return out


def max_over_ranks(x, dev, world):
    """The largest of every rank's value (the slowest replica sets the job's step time); the
    value itself when there is one rank.  Works with any torch.distributed backend."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_rate(ms_step, world):
    """Whole-job reductions per second: every replica reduces one tensor a step."""
    return world * 1000.0 / ms_step


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2201_12663_gb300 as P
    import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.load()

    A, B = workloads.hartree_like_factors(WORKLOAD["n"], WORKLOAD["Ra"], WORKLOAD["Rb"], WORKLOAD["seeds"])
    n, Ra, Rb = WORKLOAD["n"], WORKLOAD["Ra"], WORKLOAD["Rb"]
    R = Ra * Rb
    # pinned host inputs (column-major factor storage = (R, n) row-major)
    hA = [torch.from_numpy(np.ascontiguousarray(u.T)).pin_memory() for u in A.U]
    hB = [torch.from_numpy(np.ascontiguousarray(u.T)).pin_memory() for u in B.U]
    hxa = torch.from_numpy(A.xi.copy()).pin_memory()
    hxb = torch.from_numpy(B.xi.copy()).pin_memory()
    dA = [h.to(dev) for h in hA]
    dB = [h.to(dev) for h in hB]
    xa, xb = hxa.to(dev), hxb.to(dev)
    Ua = [t.t() for t in dA]
    Ub = [t.t() for t in dB]
    Uc = [torch.empty(R, n, dtype=torch.float64, device=dev).t() for _ in range(3)]
    xc = torch.empty(R, dtype=torch.float64, device=dev)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)   # 256 MB > L2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def make_form(prec, fused=args.fused):
        opts = dict(eps=WORKLOAD["eps"], r_max=WORKLOAD["r_max"], oversample=WORKLOAD["oversample"], seed=12345,
                    precision=PRECISIONS[prec])
        cp = P.make_cp(Uc, xc)
        ws = torch.empty(P.rhosvd_c2t_workspace_size(cp, P.make_opts(**opts)), dtype=torch.uint8, device=dev)
        out = P.alloc_tucker([n, n, n], R, WORKLOAD["r_max"], dev)

        if fused:       # the product's columns formed inside the reduction, never stored
            def step():
                P.rhosvd_c2t_hadamard(Ua, xa, Ub, xb, out=out, workspace=ws, **opts)
        else:           # the product stored by rhosvd_cp_hadamard, then reduced
            def step():
                P.rhosvd_cp_hadamard(Ua, xa, Ub, xb, U_out=Uc, xi_out=xc)
                P.rhosvd_c2t(Uc, xc, out=out, workspace=ws, **opts)
        return step, out, ws

    def time_form(step, out, steps, profile):
        for _ in range(max(args.warmup, 3)):
            step()
        info = out.info()
        if info.status != 0:
            raise RuntimeError(P.rhosvd_strerror(info.status))
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier()
        P.rhosvd_profile_read()
        P.rhosvd_profile_enable(profile)
        l0 = P.rhosvd_launch_count()
        for i in range(steps):
            flush.zero_()
            starts[i].record()
            step()
            ends[i].record()
        barrier()
        launches = P.rhosvd_launch_count() - l0
        P.rhosvd_profile_enable(False)
        prof = P.rhosvd_profile_read()
        tot = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), dev, world)
        return tot / steps, prof, launches, out.info()

    main_prec = args.precision
    other = "plain" if main_prec == "mixed" else "mixed"
    step, out, ws = make_form(main_prec)
    # per-stage event tracing of every stage in a separate pass (about 120 event records a step,
    # not part of the workload); the timed region then records events around the dominant
    # stage only, for its roofline
    prof_steps = max(3, args.steps // 2)
    _, prof, _, _ = time_form(step, out, prof_steps, True)
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    # the same step as direct calls, the dominant stage's launches timed in the region
    P.rhosvd_profile_filter(dom)
    ms_direct, prof_dom_direct, _, _ = time_form(step, out, args.steps, dom is not None)
    P.rhosvd_profile_filter(None)
    # headline: the step captured once into a CUDA graph through the C ABI (rhosvd_graph_*) and
    # replayed, the dominant stage's two events per launch captured with it (record nodes that
    # every replay executes, read after each step)
    gstream = torch.cuda.Stream()
    with torch.cuda.stream(gstream):
        for _ in range(3):
            step()
        barrier()
        P.rhosvd_profile_read()
        P.rhosvd_profile_filter(dom)
        P.rhosvd_profile_keep(True)
        P.rhosvd_profile_enable(dom is not None)
        graph = P.rhosvd_capture(step, gstream)
        P.rhosvd_profile_enable(False)
        for _ in range(max(args.warmup, 3)):
            graph.replay(gstream)
        barrier()
        P.rhosvd_profile_read()
        e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        sampler = ClockSampler(local)
        barrier()
        sampler.start()
        t_wall = time.perf_counter()
        l0 = P.rhosvd_launch_count()
        dom_cnt, dom_ms = 0, 0.0
        for i in range(args.steps):
            flush.zero_()
            e_s[i].record()
            graph.replay(gstream)
            e_e[i].record()
            torch.cuda.synchronize()
            pr = P.rhosvd_profile_read()
            if dom in pr:
                dom_cnt += pr[dom][0]
                dom_ms += pr[dom][1]
        barrier()
        launches = P.rhosvd_launch_count() - l0
        t_wall = time.perf_counter() - t_wall
        clocks = sampler.stop()
        P.rhosvd_profile_keep(False)
        P.rhosvd_profile_filter(None)
    info = out.info()
    if info.status != 0:
        raise RuntimeError(P.rhosvd_strerror(info.status))
    prof_dom = {dom: (dom_cnt, dom_ms)} if dom_cnt else {}
    ms_per_step = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(e_s, e_e)), dev, world) / args.steps
    value = job_rate(ms_per_step, world)

    # the other form, same run, same inputs (comparison; not the headline)
    step2, out2, ws2 = make_form(other)
    ms2, prof2, _, info2 = time_form(step2, out2, max(3, args.steps // 2), False)
    # the same precision with the product formed inside the reduction (or stored, under --fused)
    step3, out3, ws3 = make_form(main_prec, fused=not args.fused)
    ms3, _, _, _ = time_form(step3, out3, max(3, args.steps // 2), False)
    del ws3

    # agreement of the two forms (Tucker tensors), computed on the device with torch
    def tucker_of(res):
        inf = res.info()
        r = [inf.r[l] for l in range(3)]
        beta = res.beta[: r[0] * r[1] * r[2]].reshape(r[2], r[1], r[0]).permute(2, 1, 0)
        return beta, [res.Z[l][:, : r[l]] for l in range(3)], r
    bm, Zm, rm = tucker_of(out)
    bp, Zp, rp = tucker_of(out2)
    agree = tucker_rel_diff_torch(bm, Zm, bp, Zp)     # common basis per mode: ranks may differ
    host_main = (bm.cpu().numpy(), [z.cpu().numpy() for z in Zm], rm)
    host_other = (bp.cpu().numpy(), [z.cpu().numpy() for z in Zp], rp)
    fp64 = fp64_rate(P, dev)

    # ---- end to end through the C ABI: H2D inputs into the captured buffers, the graph replay,
    #      D2H result, per step, all on the graph's stream
    gctx = torch.cuda.stream(gstream)
    gctx.__enter__()
    e_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    h2d = sum(h.numel() * 8 for h in hA + hB) + (hxa.numel() + hxb.numel()) * 8
    hinfo = torch.empty(out.info_buf.numel(), dtype=torch.uint8).pin_memory()
    hZ = [torch.empty(WORKLOAD["r_max"], n, dtype=torch.float64).pin_memory() for _ in range(3)]
    hsig = torch.empty(3, P.RHOSVD_K_MAX, dtype=torch.float64).pin_memory()
    hbeta = torch.empty(WORKLOAD["r_max"] ** 3, dtype=torch.float64).pin_memory()
    d2h = 0
    barrier()
    for i in range(args.steps):
        flush.zero_()
        e_s[i].record()
        for l in range(3):
            dA[l].copy_(hA[l], non_blocking=True)
            dB[l].copy_(hB[l], non_blocking=True)
        xa.copy_(hxa, non_blocking=True)
        xb.copy_(hxb, non_blocking=True)
        graph.replay(gstream)
        hinfo.copy_(out.info_buf, non_blocking=True)
        for l in range(3):
            hZ[l].copy_(out.Z[l].t(), non_blocking=True)
        hsig.copy_(out.sigma, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        inf = P.rhosvd_info.from_buffer_copy(bytes(hinfo.numpy().tobytes()))
        cnt = inf.r[0] * inf.r[1] * inf.r[2]
        hbeta[:cnt].copy_(out.beta[:cnt], non_blocking=True)
        e_e[i].record()
        d2h = hinfo.numel() + sum(z.numel() * 8 for z in hZ) + hsig.numel() * 8 + cnt * 8
    barrier()
    gctx.__exit__(None, None, None)
    graph.close()
    e2e_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(e_s, e_e)) / args.steps
    e2e_value = job_rate(max_over_ranks(e2e_ms, dev, world), world)

    # ---- roofline of the dominant stage (largest share in the traced pass), its launches timed
    #      by CUDA events on the launching stream inside the timed region
    total_ms = sum(v[1] for v in prof.values()) if prof else 0.0
    shares = {k: round(v[1] / total_ms, 4) for k, v in prof.items()} if prof else {}
    roof = None
    if prof and dom in prof_dom:
        name = dom
        cnt, ms_tot = prof_dom[dom]
        avg_ms = ms_tot / cnt
        fl = algorithmic_flops(name, info, n, R)
        pk = peaks()
        if fl is not None and main_prec == "mixed" and name in MIXED_PAIRS:
            # the digit-plane scheme executes MIXED_PAIRS BF16 products per FP64-class product,
            # so its FP64-class peak is the measured BF16 rate divided by that count
            ach = fl / (avg_ms * 1e-3) / 1e12
            bf16 = pk.get("bf16_tflops", 1912.0)
            peak = bf16 / MIXED_PAIRS[name]
            roof = {"bound": "tensor", "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": NCU_TRAFFIC.get(name),
                    "peak_source": f"MEASURED_PEAKS.json bf16_tflops {bf16} (burst, of measured) / "
                                   f"{MIXED_PAIRS[name]} digit-plane products",
                    "avg_launch_ms": avg_ms, "algorithmic_flops_per_launch": fl}
        elif fl is not None:
            ach = fl / (avg_ms * 1e-3) / 1e12
            pk64 = fp64["probe_tflops"]
            roof = {"bound": "alu", "kernel": name, "achieved": ach, "peak": pk64, "unit": "TFLOP/s",
                    "frac": ach / pk64, "traffic": NCU_TRAFFIC.get(name),
                    "peak_source": "FP64 fma rate measured on this GPU by the library's probe in this run "
                                   "(of measured; MEASURED_PEAKS.json has no FP64 entry)",
                    "note": "sequential pivot steps on a 16-block cluster per mode: bound by the per-step exchange and cluster barrier, not by FP64 issue or memory",
                    "avg_launch_ms": avg_ms, "algorithmic_flops_per_launch": fl}
        else:
            roof = {"bound": "alu", "kernel": name, "achieved": None, "peak": fp64["probe_tflops"], "unit": "TFLOP/s",
                    "frac": None, "traffic": None, "note": "no flop model for this stage",
                    "avg_launch_ms": avg_ms}
    if roof is not None:
        # the whole step against the HBM roofline of the reduction: two reads of the three FP64
        # side matrices (n R 8 bytes each) per reduction
        hbm = peaks().get("hbm_gbs", 6800.0)
        alg = 2 * 3 * n * R * 8
        roof["whole_step"] = {"bound": "hbm", "algorithmic_bytes": alg, "ms_per_step": ms_per_step,
                              "achieved": alg / (ms_per_step * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                              "frac": alg / (ms_per_step * 1e-3) / 1e9 / hbm,
                              "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (mixed: bf16 digit planes, fp32 accumulate)" if main_prec == "mixed"
            else "f64", "data": "synthetic",
            "config": {**WORKLOAD, "precision": main_prec,
                       "product": "formed inside the reduction (rhosvd_c2t_hadamard)" if args.fused
                       else "stored by rhosvd_cp_hadamard, then reduced",
                       "launch": "the step's library calls captured once into a CUDA graph (rhosvd_graph_*) "
                                 "and replayed each step",
                       "l2": "flushed (256 MB write) before every timed step",
                       "ranks": [info.r[l] for l in range(3)], "k": [info.k[l] for l in range(3)],
                       "tails": [info.tail[l] for l in range(3)]},
            "error": {"vs": f"{other} GPU form, same sketch", "tucker_rel_diff": agree,
                      "ranks_other": [info2.r[l] for l in range(3)]},
            "fp64_peak": fp64,
            f"{other}_form": {"value": world * 1000.0 / ms2, "ms_per_step": ms2,
                              "stage_ms_per_step": {k: v[1] / max(3, args.steps // 2) for k, v in prof2.items()}},
            "speedup_vs_other_form": ms2 / ms_per_step,
            "direct_calls": {"ms_per_step": ms_direct, "value": world * 1000.0 / ms_direct,
                             "note": "the same step as ~120 separate launches through the C ABI, no graph"},
            ("fused_product" if not args.fused else "stored_product"): {
                "ms_per_step": ms3, "value": world * 1000.0 / ms3,
                "note": "same precision; rhosvd_c2t_hadamard (no stored product)" if not args.fused
                else "same precision; rhosvd_cp_hadamard into a buffer, then rhosvd_c2t"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "stage_shares": shares,
            "stage_ms_per_step": {k: v[1] / prof_steps for k, v in prof.items()},
            "clocks": clocks, "wall_s_timed": t_wall, "parallelism": f"replicas{world}"}
    if not args.no_batched:
        line["batched"] = batched_leg(P, dev, args.steps, args.warmup, main_prec)
    if args.learned_train > 0:
        line["learned"] = learned_leg(P, dev, args.learned_train, args.learned_eval, main_prec)
    if not args.no_t2c:
        line["t2c"] = t2c_leg(P, out, max(3, args.steps // 2), args.warmup)
    if not args.no_poly:
        line["poly"] = poly_leg(P, max(3, args.steps // 2), args.warmup, main_prec)
    if not args.no_rs:
        line["rs"] = rs_leg(P, 3, 1, main_prec)
    if not args.no_als:
        line["als"] = als_leg(P, 3, 1, main_prec)
    if not args.no_rs_collective:
        rsc = rs_collective_leg(P, dev, max(3, args.steps // 2), args.warmup)
        line["rs_collective"] = rsc
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's whole reduction of the same workload on all host cores (threads over the
        # modes and over slices of the core's terms): the CPU baseline, and the reference the
        # headline's error is stated against
        nth = nproc() or 1
        orc = oracle_full_threads(nth)
        line["cpu_baseline"] = {
            "value": 1.0 / orc["wall"], "unit": UNIT, "cores": nth, "kind": "oracle",
            "sample": (f"one whole reduction of the bench workload (no extrapolation): Hadamard product and "
                       f"normalisation on one thread, the three side-matrix SVDs and projections one mode a "
                       f"thread, the core over {nth} term slices one a thread; {orc['wall']:.1f} s wall, "
                       f"{orc['busy']:.1f} s of busy thread time (1-core equivalent "
                       f"{1.0 / orc['busy']:.4f} reductions/s)"),
            "value_1core_equivalent": 1.0 / orc["busy"], "ranks": orc["ranks"]}
        err = line["error"]
        for key, (b_, Z_, r_) in (("tucker_rel_diff_vs_oracle", host_main), (f"{other}_tucker_rel_diff_vs_oracle", host_other)):
            if r_ == orc["ranks"]:
                err[key] = tucker_rel_diff_np(b_, Z_, orc["beta"], orc["Z"])
            else:
                err[key] = None
                err[key + "_note"] = f"ranks {r_} differ from the oracle's {orc['ranks']}"
        err["vs"] = "oracle (FP64 CPU, exact SVDs, same input)"
        err["vs_other_form"] = f"{other} GPU form, same sketch"
        if "rs_collective" in line:
            line["rs_collective"]["error"] = rs_collective_oracle_error(line["rs_collective"].pop("_host"))
    elif "rs_collective" in line:
        line["rs_collective"].pop("_host", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-workload leg")
    ap.add_argument("--no-t2c", action="store_true", help="skip the Tucker-to-canonical leg")
    ap.add_argument("--no-poly", action="store_true", help="skip the Newton-cube / Horner leg")
    ap.add_argument("--no-rs", action="store_true", help="skip the range-separated Slater / energy leg")
    ap.add_argument("--no-als", action="store_true", help="skip the RHOSVD + ALS leg")
    ap.add_argument("--no-rs-collective", action="store_true",
                    help="skip the range-separated collective potential leg (n=2048, R=20000)")
    ap.add_argument("--fused", action="store_true",
                    help="headline step forms the Hadamard product inside the reduction (rhosvd_c2t_hadamard)")
    ap.add_argument("--precision", choices=["mixed", "plain"], default="mixed")
    ap.add_argument("--learned-train", type=int, default=600,
                    help="training instances of the learned-proposal leg (0 skips it; the full workload is 20000)")
    ap.add_argument("--learned-eval", type=int, default=60, help="held-out instances (the full workload is 2000)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Host-side argument checks of the entry points beyond rhosvd_c2t (T2C, Horner, C2T-ALS, the
fused Hadamard reduction, node sampling and the interaction energy, replayable call sequences):
every case here is rejected, or finishes with nothing to do, before any device memory is touched
or any kernel is launched, so it runs without a GPU.  The pointers are placeholders that the
library must not dereference on these paths."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAKE = 0x1000          # a non-null placeholder address; never dereferenced on these paths


def _define(name):
    txt = open(os.path.join(ROOT, "include", "rhosvd.h")).read()
    return int(re.search(r"#define\s+" + name + r"\s+(\d+)", txt).group(1))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_12663_gb300 import build_lib
    build_lib.build()
    import paper_2201_12663_gb300 as P
    return P, P.load()


def _cp(P, n=(32, 32, 32), R=10):
    cp = P.rhosvd_cp()
    for l in range(3):
        cp.n[l] = n[l]
        cp.ld[l] = n[l]
        cp.U[l] = FAKE
    cp.R = R
    cp.xi = FAKE
    return cp


def _ptr3():
    return (ctypes.c_void_p * 3)(FAKE, FAKE, FAKE)


def _int3(*v):
    return (ctypes.c_int * 3)(*v)


def test_horner_checks(lib):
    P, L = lib
    cp = _cp(P)
    o = P.make_opts(eps=1e-6, r_max=16, oversample=8)
    size = L.rhosvd_cp_horner_workspace_size
    assert size(ctypes.byref(cp), 3, ctypes.byref(o), 200) % 256 == 0
    assert size(ctypes.byref(cp), 3, ctypes.byref(o), 200) > 0
    assert size(ctypes.byref(cp), 0, ctypes.byref(o), 200) == 0          # no coefficients
    assert size(ctypes.byref(cp), 3, ctypes.byref(o), 0) == 0            # R_max < 1
    o_bad = P.make_opts(eps=1e-6, r_max=P.RHOSVD_K_MAX + 1, oversample=8)
    assert size(ctypes.byref(cp), 3, ctypes.byref(o_bad), 200) == 0
    R_out = ctypes.c_int(-1)
    steps = (P.rhosvd_horner_step * 4)()

    def call(coeffs, ws_bytes=1 << 40, eps_t2c=1e-8, ldu=(32, 32, 32)):
        c = (ctypes.c_double * len(coeffs))(*coeffs)
        return L.rhosvd_cp_horner(ctypes.byref(cp), c, len(coeffs), ctypes.byref(o), eps_t2c, 200, _ptr3(),
                                  _int3(*ldu), FAKE, ctypes.byref(R_out), steps, ctypes.c_void_p(0x100000),
                                  ws_bytes, None)

    assert call([1.0, math.nan, 2.0]) == P.RHOSVD_ERR_INVALID_ARG       # non-finite coefficient
    assert call([1.0, 2.0], eps_t2c=-1.0) == P.RHOSVD_ERR_INVALID_ARG
    assert call([1.0, 2.0], ldu=(32, 31, 32)) == P.RHOSVD_ERR_INVALID_ARG
    assert call([1.0, 2.0], ws_bytes=16) == P.RHOSVD_ERR_WORKSPACE
    assert R_out.value == -1                                              # nothing written


def test_als_sweep_bounds(lib):
    P, L = lib
    cp = _cp(P)
    o = P.make_opts(eps=1e-6, r_max=16, oversample=8)
    smax = _define("RHOSVD_ALS_MAX_SWEEPS")
    size = L.rhosvd_c2t_als_workspace_size
    base = L.rhosvd_c2t_workspace_size(ctypes.byref(cp), ctypes.byref(o))
    assert size(ctypes.byref(cp), ctypes.byref(o), 0) == base
    assert size(ctypes.byref(cp), ctypes.byref(o), smax) >= base
    assert size(ctypes.byref(cp), ctypes.byref(o), -1) == 0
    assert size(ctypes.byref(cp), ctypes.byref(o), smax + 1) == 0
    t = P.rhosvd_tucker()
    e = (ctypes.c_double * (6 * (smax + 1)))()
    for sw in (-1, smax + 1):
        rc = L.rhosvd_c2t_als(ctypes.byref(cp), ctypes.byref(o), sw, ctypes.byref(t), e, None, 0, None)
        assert rc == P.RHOSVD_ERR_INVALID_ARG


def test_t2c_checks(lib):
    P, L = lib
    t = P.rhosvd_tucker_in()
    for l in range(3):
        t.n[l] = 32
        t.r[l] = 6
        t.Z[l] = FAKE
        t.ldz[l] = 32
    t.beta = FAKE
    ws = L.rhosvd_t2c_workspace_size(ctypes.byref(t))
    assert ws > 0 and ws % 256 == 0
    R_out, p_out, st = ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_int(-1)

    def call(tt, eps=1e-6, R_max=100, ws_bytes=ws):
        return L.rhosvd_t2c(ctypes.byref(tt), eps, R_max, _ptr3(), _int3(32, 32, 32), FAKE, ctypes.byref(R_out),
                            ctypes.byref(p_out), ctypes.byref(st), ctypes.c_void_p(0x100000), ws_bytes, None)

    assert call(t, eps=-1.0) == P.RHOSVD_ERR_INVALID_ARG
    assert call(t, R_max=-1) == P.RHOSVD_ERR_INVALID_ARG
    assert call(t, ws_bytes=ws - 256) == P.RHOSVD_ERR_WORKSPACE
    bad = P.rhosvd_tucker_in.from_buffer_copy(t)
    bad.ldz[2] = 31
    assert call(bad) == P.RHOSVD_ERR_INVALID_ARG
    big = P.rhosvd_tucker_in.from_buffer_copy(t)
    big.r[0] = big.r[1] = 200                                             # r1 r2 above the slice limit
    assert _define("RHOSVD_T2C_SLICE_MAX") < 200 * 200
    assert L.rhosvd_t2c_workspace_size(ctypes.byref(big)) == 0
    assert call(big) == P.RHOSVD_ERR_INVALID_ARG
    assert (R_out.value, st.value) == (-1, -1)


def test_fused_hadamard_checks(lib):
    P, L = lib
    o = P.make_opts(eps=1e-7, r_max=32, oversample=8)
    a, b = _cp(P, R=8), _cp(P, R=5)
    ws = L.rhosvd_c2t_hadamard_workspace_size(ctypes.byref(a), ctypes.byref(b), ctypes.byref(o))
    prod = _cp(P, R=40)
    assert ws == L.rhosvd_c2t_workspace_size(ctypes.byref(prod), ctypes.byref(o)) and ws > 0
    b2 = _cp(P, n=(32, 33, 32), R=5)                                     # the grids must agree
    assert L.rhosvd_c2t_hadamard_workspace_size(ctypes.byref(a), ctypes.byref(b2), ctypes.byref(o)) == 0
    t = P.rhosvd_tucker()
    rc = L.rhosvd_c2t_hadamard(ctypes.byref(a), ctypes.byref(b2), ctypes.byref(o), ctypes.byref(t), None, 0, None)
    assert rc == P.RHOSVD_ERR_INVALID_ARG


def test_sample_and_energy_checks(lib):
    P, L = lib
    cp = _cp(P)
    assert L.rhosvd_cp_sample(ctypes.byref(cp), -1, FAKE, FAKE, None) == P.RHOSVD_ERR_INVALID_ARG
    assert L.rhosvd_cp_sample(ctypes.byref(cp), 4, None, FAKE, None) == P.RHOSVD_ERR_INVALID_ARG
    assert L.rhosvd_cp_sample(ctypes.byref(cp), 4, FAKE, None, None) == P.RHOSVD_ERR_INVALID_ARG
    assert L.rhosvd_cp_sample(ctypes.byref(cp), 0, None, None, None) == P.RHOSVD_OK   # nothing to do
    nx = _cp(P)
    nx.xi = None
    assert L.rhosvd_cp_sample(ctypes.byref(nx), 4, FAKE, FAKE, None) == P.RHOSVD_ERR_INVALID_ARG
    e = L.rhosvd_rs_energy
    assert e(ctypes.byref(cp), 4, FAKE, FAKE, 0.5, FAKE, None, None) == P.RHOSVD_ERR_INVALID_ARG   # no energy
    assert e(ctypes.byref(cp), 4, FAKE, None, 0.5, FAKE, FAKE, None) == P.RHOSVD_ERR_INVALID_ARG   # no charges
    assert e(ctypes.byref(cp), 4, FAKE, FAKE, math.inf, FAKE, FAKE, None) == P.RHOSVD_ERR_INVALID_ARG


def test_graph_null_handles(lib):
    P, L = lib
    h = ctypes.c_void_p()
    assert L.rhosvd_graph_begin(None) == P.RHOSVD_ERR_INVALID_ARG
    assert L.rhosvd_graph_end(None, ctypes.byref(h)) == P.RHOSVD_ERR_INVALID_ARG
    assert L.rhosvd_graph_launch(None, None) == P.RHOSVD_ERR_INVALID_ARG
    assert L.rhosvd_graph_destroy(None) == P.RHOSVD_OK


def test_mlp_checkpoint_file_checks(lib, tmp_path):
    """rhosvd_mlp_load validates the whole file before it touches the handle: a missing file, a
    wrong tag, other layer widths, a short body and trailing bytes are all INVALID_ARG (the
    placeholder handle is never dereferenced on these paths)."""
    import numpy as np
    P, L = lib
    bad = P.RHOSVD_ERR_INVALID_ARG
    h = ctypes.c_void_p(FAKE)
    assert L.rhosvd_mlp_load(h, os.fsencode(str(tmp_path / "none.bin"))) == bad
    assert L.rhosvd_mlp_load(None, os.fsencode(str(tmp_path / "none.bin"))) == bad
    dims = [128, 512, 512, 512, 2048]
    nbody = sum(3 * dims[i] * dims[i + 1] + 3 * dims[i + 1] for i in range(4))   # W, b and their moments

    def write(name, tag=b"RHMLPv01", d=dims, step=7, n=nbody, extra=b""):
        p = tmp_path / name
        with open(p, "wb") as f:
            f.write(tag)
            f.write(np.array([4] + list(d), dtype="<i4").tobytes())
            f.write(np.array([step], dtype="<i8").tobytes())
            f.write(np.zeros(n, dtype="<f4").tobytes())
            f.write(extra)
        return os.fsencode(str(p))
    assert L.rhosvd_mlp_load(h, write("tag.bin", tag=b"RHMLPv99")) == bad
    assert L.rhosvd_mlp_load(h, write("dims.bin", d=[128, 256, 512, 512, 2048])) == bad
    assert L.rhosvd_mlp_load(h, write("short.bin", n=nbody - 1)) == bad
    assert L.rhosvd_mlp_load(h, write("extra.bin", extra=b"\0")) == bad
    assert L.rhosvd_mlp_load(h, write("step.bin", step=-1)) == bad

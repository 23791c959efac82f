"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/rhosvd.h declares.  Host-only entry points (workspace planning, argument
checking) are exercised without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rhosvd_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2201_12663_gb300 import build_lib
    path = build_lib.build()
    import paper_2201_12663_gb300 as P
    return P, P.load()


def test_every_declared_symbol_is_exported(lib):
    P, L = lib
    decl = _declared_functions()
    assert len(decl) >= 7
    out = subprocess.run(["nm", "-D", "--defined-only", P.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rhosvd_[a-z0-9_]+)", out))
    missing = [d for d in decl if d not in exported]
    assert not missing, missing
    for d in decl:
        assert hasattr(L, d)


def test_library_is_built_for_sm103a(lib):
    P, _ = lib
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", P.lib_path()],
                         capture_output=True, text=True).stdout
    assert "sm_103a" in out


def _cp(P, n=(64, 64, 64), R=100):
    cp = P.rhosvd_cp()
    for l in range(3):
        cp.n[l] = n[l]
        cp.ld[l] = n[l]
        cp.U[l] = 0x1000
    cp.R = R
    cp.xi = 0x1000
    return cp


def test_workspace_planning_host_only(lib):
    P, _ = lib
    cp = _cp(P, (1024, 1024, 1024), 4096)
    o = P.make_opts(eps=1e-7, r_max=160, oversample=32)
    ws = P.rhosvd_c2t_workspace_size(cp, o)
    assert ws > 0 and ws % 256 == 0
    assert [P.rhosvd_subspace_width(cp, o, l) for l in range(3)] == [192, 192, 192]
    # n <= k: the direct (exact Gram) mode searches the whole space
    cp2 = _cp(P, (128, 128, 300), 200)
    assert [P.rhosvd_subspace_width(cp2, o, l) for l in range(3)] == [128, 128, 192]
    # R < k: the sketch never exceeds the canonical rank
    cp3 = _cp(P, (512, 512, 512), 50)
    assert P.rhosvd_subspace_width(cp3, o, 0) == 50


@pytest.mark.parametrize("bad", ["rmax0", "rmax_big", "neg_eps", "prec", "ld", "n0"])
def test_invalid_arguments_are_rejected_before_any_launch(lib, bad):
    P, L = lib
    cp = _cp(P)
    o = P.make_opts(eps=1e-6, r_max=32, oversample=8)
    if bad == "rmax0":
        o.r_max = 0
    elif bad == "rmax_big":
        o.r_max = P.RHOSVD_K_MAX + 1
    elif bad == "neg_eps":
        o.eps = -1.0
    elif bad == "prec":
        o.precision = 7
    elif bad == "ld":
        cp.ld[1] = 3
    elif bad == "n0":
        cp.n[2] = 0
    assert P.rhosvd_c2t_workspace_size(cp, o) == 0
    t = P.rhosvd_tucker()
    rc = L.rhosvd_c2t(ctypes.byref(cp), ctypes.byref(o), ctypes.byref(t), None, 0, None)
    assert rc == P.RHOSVD_ERR_INVALID_ARG


def test_workspace_too_small_is_reported(lib):
    P, L = lib
    cp = _cp(P)
    o = P.make_opts(eps=1e-6, r_max=32, oversample=8)
    t = P.rhosvd_tucker()
    for l in range(3):
        t.Z[l] = 0x1000
        t.sigma[l] = 0x1000
    t.beta = 0x1000
    t.info = 0x1000
    rc = L.rhosvd_c2t(ctypes.byref(cp), ctypes.byref(o), ctypes.byref(t), ctypes.c_void_p(0x100000), 16, None)
    assert rc == P.RHOSVD_ERR_WORKSPACE


def test_strerror_and_version(lib):
    P, _ = lib
    assert P.rhosvd_version() >= 100
    assert "rank" in P.rhosvd_strerror(P.RHOSVD_ERR_RANK_OVERFLOW)
    assert P.rhosvd_strerror(12345) == "unknown status"

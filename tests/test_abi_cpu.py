"""CPU-side checks of the C ABI (no device work): the library builds and loads,
exports every function include/opendust.h declares, the ctypes structures match the
header's layout, and invalid parameters are rejected before any CUDA call."""
import ctypes
import os
import re

import pytest

import paper_2205_06557_gb300 as od
from paper_2205_06557_gb300 import build
from paper_2205_06557_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "opendust.h")


@pytest.fixture(scope="module")
def L():
    build.build()
    return od.lib()


def test_exports_every_declared_function(L):
    names = set(re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(od_[a-z_]+)\s*\(", open(HEADER).read(), re.M))
    assert {"od_create", "od_step", "od_dust_state", "od_destroy"} <= names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing


def test_struct_layout_matches_header():
    # 13 doubles, int64, 2 x int32, pointer, uint64, int64, pointer, 2 x int32, pointer
    assert ctypes.sizeof(od.od_params) == 13 * 8 + 8 + 8 + 8 + 8 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(od.od_dust) == 40
    assert od.od_params.cuda_stream.offset == ctypes.sizeof(od.od_params) - 8


def _rc(L, p):
    s, keep = od.make_params(p)
    h = ctypes.c_void_p()
    return L.od_create(ctypes.byref(s), ctypes.byref(h)), od.od_last_error()


@pytest.mark.parametrize("change", [
    dict(R=-1.0), dict(dt=0.0), dict(T_e=float("nan")), dict(mach=1.0, E_ext=100.0), dict(mach=0.0, E_ext=100.0, nu=0.0),
    dict(dust=[dict(x=1.95e-4, y=0.0, z=0.0, a=1e-5, q0=0.0)]),
    dict(dust=[dict(x=0.0, y=0.0, z=0.0, a=2e-5, q0=0.0)] * 9),
    dict(n_ions=-3), dict(weight=0.0),
])
def test_invalid_parameters_rejected_on_host(L, change):
    p = W.tiny()
    p.update(change)
    rc, msg = _rc(L, p)
    assert rc == -1 and msg


@pytest.mark.parametrize("mach,nu,a", [(1.0, 1e6, 2e-5), (0.3, 0.0, 8e-6), (2.0, 5e6, 1.5e-5), (1e-9, 0.0, 1e-5)])
def test_library_oml_charge_matches_oracle(L, mach, nu, a):
    """host-side OML charge of the library (Gauss-Legendre) vs the oracle's (scipy quad)"""
    from oracle import oml

    p = dict(W.tiny(), mach=mach, nu=nu)
    q_lib = od.od_oml_charge(p, a)
    q_ref = oml.oml_charge(a, p["n_inf"], p["m_i"], p["T_i"], p["T_e"], mach)
    assert abs(q_lib / q_ref - 1) < 1e-9


def test_null_arguments(L):
    assert L.od_create(None, None) == -1
    assert L.od_step(None, 1) == -1
    L.od_destroy(None)


def test_checkpoint_loader_rejects_foreign_files_on_host(L, tmp_path):
    """od_load checks the file before any device work"""
    h = ctypes.c_void_p()
    bad = tmp_path / "not_a_checkpoint.bin"
    bad.write_bytes(b"hello, this is not a checkpoint" * 10)
    assert L.od_load(os.fsencode(str(bad)), None, ctypes.byref(h)) == -1
    assert "checkpoint" in od.od_last_error()
    trunc = tmp_path / "truncated.bin"
    trunc.write_bytes(b"ODCKPT01" + b"\x01\x00\x00\x00")
    assert L.od_load(os.fsencode(str(trunc)), None, ctypes.byref(h)) == -1
    assert L.od_load(os.fsencode(str(tmp_path / "missing.bin")), None, ctypes.byref(h)) == -1
    assert not h.value


def test_observability_calls_reject_null_handles(L, tmp_path):
    path = os.fsencode(str(tmp_path / "x.xyz"))
    assert L.od_save(None, path) == -1
    assert L.od_write_ions(None, path, 0) == -1
    assert L.od_density_enable(None, 8, 8) == -1
    assert L.od_density_read(None, None, None, None) == -1
    assert L.od_num_dust(None) == -1

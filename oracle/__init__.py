"""Oracle for the ion-flow-around-dust time step (OpenDust, arXiv 2205.06557).

TEST INFRASTRUCTURE ONLY.  A plain FP64 CPU restatement of the method (``oracle.c``)
used to check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA
library and never calls it.

Parameters are passed as a plain dict of SI values (the same dict the workload
generators produce for both sides); see ``_to_struct`` for the keys.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MAX_DUST = 8
REC = 13  # q, F_orbit[3], F_dd[3], F_collect[3], F_ext[3]
EV = 13  # absorbed[8], outflow, injected bottom/top/side, collided

F_NO_IONION = 1
F_NO_EOUT = 2
F_NO_BOUNDARY = 4
F_NO_ABSORB = 8
F_PAPER_SIDE = 16
F_FLUX_INJECT = 32

Q_MODELS = {"given": 0, "consistent": 1}


class _Dust(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("x", "y", "z", "a", "q0")]


class _Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "m_i", "Z", "T_i", "T_n", "T_e", "n_inf", "mach", "E_ext", "nu", "R", "H", "dt", "weight")] + [
        ("n_ions", ctypes.c_int64),
        ("n_dust", ctypes.c_int32),
        ("charge_model", ctypes.c_int32),
        ("dust", _Dust * MAX_DUST),
        ("seed", ctypes.c_uint64),
        ("avg_start", ctypes.c_int64),
        ("has_alpha", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("alpha", ctypes.c_double * 15),
        ("grid_nx", ctypes.c_int32),
        ("grid_nz", ctypes.c_int32),
        ("quad_n", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("r_cut", ctypes.c_double),
        ("r_switch", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i32, i64, u64, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [P(_Params), ctypes.c_char_p, ctypes.c_int]
        L.orc_destroy.argtypes = [vp]
        L.orc_step.argtypes = [vp, i64]
        L.orc_num_ions.restype = i64
        L.orc_num_ions.argtypes = [vp]
        L.orc_step_index.restype = i64
        L.orc_step_index.argtypes = [vp]
        L.orc_get_ions.argtypes = [vp, vp, vp, vp, vp]
        L.orc_set_ions.argtypes = [vp, i64, vp, vp, vp, i64]
        L.orc_forces.argtypes = [vp, i64, i64, vp, vp]
        L.orc_load_ions.argtypes = [vp, i64, vp, vp, vp, i64]
        L.orc_derived.argtypes = [vp, vp]
        L.orc_alpha.argtypes = [vp, vp]
        L.orc_eout.argtypes = [vp, d, d, d, vp]
        L.orc_cyl_integral.restype = d
        L.orc_cyl_integral.argtypes = [P(_Params), d, d]
        L.orc_inject_sample.argtypes = [vp, u64, ctypes.c_uint32, vp, vp, vp]
        L.orc_injections.restype = i64
        L.orc_injections.argtypes = [vp, ctypes.c_uint32]
        L.orc_records.argtypes = [vp, i64, i64, vp, vp]
        L.orc_dust_q.argtypes = [vp, vp]
        L.orc_dust_terms.argtypes = [vp, vp, vp]
        L.orc_philox.argtypes = [vp, vp, vp]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _to_struct(p):
    s = _Params()
    for k in ("m_i", "T_i", "T_e", "n_inf", "R", "H", "dt"):
        setattr(s, k, float(p[k]))
    s.Z = float(p.get("Z", 1.0))
    s.T_n = float(p.get("T_n", 0.0))
    s.mach = float(p.get("mach", 0.0))
    s.E_ext = float(p.get("E_ext", 0.0))
    s.nu = float(p.get("nu", 0.0))
    s.weight = float(p.get("weight", 1.0))
    s.n_ions = int(p.get("n_ions", 0))
    dust = p.get("dust", [])
    s.n_dust = len(dust)
    for k, g in enumerate(dust):
        s.dust[k] = _Dust(g["x"], g["y"], g["z"], g["a"], g.get("q0", 0.0))
    s.charge_model = Q_MODELS[p.get("charge_model", "given")]
    s.seed = int(p.get("seed", 0))
    s.avg_start = int(p.get("avg_start", 1))
    if p.get("alpha") is not None:
        s.has_alpha = 1
        for t in range(15):
            s.alpha[t] = float(p["alpha"][t])
    s.flags = int(p.get("oracle_flags", 0))
    s.grid_nx = int(p.get("grid_nx", 0))
    s.grid_nz = int(p.get("grid_nz", 0))
    s.quad_n = int(p.get("quad_n", 0))
    s.r_cut = float(p.get("r_cut", 0.0))
    s.r_switch = float(p.get("r_switch", 0.0))
    return s


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(key, ctr):
    """Philox4x32-10 block for key (2 words) and counter (4 words)."""
    k = np.asarray(key, dtype=np.uint32)
    c = np.asarray(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(k), _ptr(c), _ptr(out))
    return out


def cyl_integral(params, r0, z0):
    """int over the cylinder of exp(-|r-r'|/lambda_De)/|r-r'| d^3r' at (r0, 0, z0), m^2."""
    s = _to_struct(params)
    return lib().orc_cyl_integral(ctypes.byref(s), float(r0), float(z0))


def num_threads():
    return lib().orc_num_threads()


class Oracle:
    """One oracle run; mirrors the library's create/step/state calls."""

    DERIVED = ("lam", "cs", "sig", "sig_n", "u", "E", "q", "m", "pb", "pt", "ps", "Tb", "Tbt",
               "Tcoll", "N", "Ie0", "pcoll", "next_id")

    def __init__(self, params):
        self.params = dict(params)
        self.D = len(params.get("dust", []))
        s = _to_struct(params)
        err = ctypes.create_string_buffer(256)
        h = lib().orc_create(ctypes.byref(s), err, 256)
        if not h:
            raise ValueError("oracle: " + err.value.decode())
        self.h = h

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_ions(self):
        return lib().orc_num_ions(self.h)

    @property
    def step_index(self):
        return lib().orc_step_index(self.h)

    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    def get_ions(self):
        N = self.n_ions
        x = np.zeros((N, 3))
        v = np.zeros((N, 3))
        a = np.zeros((N, 3))
        ids = np.zeros(N, dtype=np.uint64)
        lib().orc_get_ions(self.h, _ptr(x), _ptr(v), _ptr(a), _ptr(ids))
        return x, v, a, ids

    def set_ions(self, x, v, ids, next_id=None):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        n = x.shape[0]
        if next_id is None:
            next_id = int(ids.max()) + 1 if n else 0
        lib().orc_set_ions(self.h, n, _ptr(x), _ptr(v), _ptr(ids), int(next_id))

    def load_ions(self, x, v, ids, next_id=None):
        """replace the ion state without a force pass (accelerations zero)"""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        n = x.shape[0]
        if next_id is None:
            next_id = int(ids.max()) + 1 if n else 0
        lib().orc_load_ions(self.h, n, _ptr(x), _ptr(v), _ptr(ids), int(next_id))

    def forces(self, i0=0, i1=None, dust=True):
        """accelerations of target ions [i0, i1) and the Eq. 1 force on every grain"""
        if i1 is None:
            i1 = self.n_ions
        acc = np.zeros((max(i1 - i0, 0), 3))
        fo = np.zeros((MAX_DUST, 3))
        lib().orc_forces(self.h, int(i0), int(i1), _ptr(acc), _ptr(fo) if dust else None)
        return acc, fo[: self.D]

    def injections(self, step):
        """superions injected in step `step` (1-based) under the flux rule"""
        return lib().orc_injections(self.h, int(step))

    def derived(self):
        o = np.zeros(24)
        lib().orc_derived(self.h, _ptr(o))
        return dict(zip(self.DERIVED, o))

    def alpha(self):
        a = np.zeros(15)
        lib().orc_alpha(self.h, _ptr(a))
        return a

    def eout(self, x, y, z):
        E = np.zeros(3)
        lib().orc_eout(self.h, float(x), float(y), float(z), _ptr(E))
        return E

    def inject_sample(self, ion_id, step):
        pos = np.zeros(3)
        vel = np.zeros(3)
        face = ctypes.c_int(0)
        lib().orc_inject_sample(self.h, int(ion_id), int(step), _ptr(pos), _ptr(vel), ctypes.byref(face))
        return pos, vel, face.value

    def records(self, first=1, count=None):
        """per-step dust records [count, D, 13] and event counts [count, 13]"""
        if count is None:
            count = self.step_index - first + 1
        rec = np.zeros((count, MAX_DUST, REC))
        ev = np.zeros((count, EV), dtype=np.int32)
        lib().orc_records(self.h, int(first), int(count), _ptr(rec), _ptr(ev))
        return rec[:, : self.D], ev

    def dust_q(self):
        q = np.zeros(MAX_DUST)
        lib().orc_dust_q(self.h, _ptr(q))
        return q[: self.D]

    def dust_terms(self):
        """window means and batch-means standard errors, each [D, 13]"""
        mean = np.zeros((MAX_DUST, REC))
        se = np.zeros((MAX_DUST, REC))
        lib().orc_dust_terms(self.h, _ptr(mean), _ptr(se))
        return mean[: self.D], se[: self.D]

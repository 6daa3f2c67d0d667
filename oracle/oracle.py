"""ctypes front of the FP64 CPU oracle (``lbfe_oracle.c``).

TEST INFRASTRUCTURE: only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA product
path never imports it.

Fields use the interface layout documented in ``lbfe_oracle.c``:
``f`` is ``[2][19][Lz][Ly][Lx]`` float64, ``C`` is ``[6][Lz][Ly][Lx]``
(xx, yy, zz, xy, xz, yz), densities ``[2][Lz][Ly][Lx]``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liblbfe_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP on the outer loops)."""
    src = os.path.join(_HERE, "lbfe_oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-D_DEFAULT_SOURCE", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(ct.Structure):
    _fields_ = [("Lx", ct.c_int), ("Ly", ct.c_int), ("Lz", ct.c_int), ("visco_phase", ct.c_int),
                ("Uw", ct.c_double), ("G", ct.c_double), ("eta_M", ct.c_double),
                ("lambda_", ct.c_double), ("eta_P", ct.c_double), ("tau_P", ct.c_double),
                ("L2", ct.c_double), ("rho_in", ct.c_double), ("rho_out", ct.c_double),
                ("gx", ct.c_double), ("gy", ct.c_double), ("gz", ct.c_double), ("advection", ct.c_int)]


class Obs(ct.Structure):
    _fields_ = [("mass", ct.c_double * 2), ("volume", ct.c_double), ("centroid", ct.c_double * 3),
                ("D", ct.c_double), ("theta_deg", ct.c_double), ("Lp", ct.c_double),
                ("M", ct.c_double * 6), ("necks", ct.c_int), ("fragments", ct.c_int),
                ("broken", ct.c_int), ("nan_seen", ct.c_int)]


class Derived(ct.Structure):
    _fields_ = [("nu_A", ct.c_double), ("nu_B", ct.c_double), ("pi_coef", ct.c_double),
                ("visc_comp", ct.c_int)]


_D = ct.POINTER(ct.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ct.CDLL(_SO)
        P = ct.POINTER(Params)
        L.orc_params_size.restype = ct.c_size_t
        L.orc_obs_size.restype = ct.c_size_t
        assert L.orc_params_size() == ct.sizeof(Params), "oracle params struct mismatch"
        assert L.orc_obs_size() == ct.sizeof(Obs), "oracle obs struct mismatch"
        L.orc_derive.argtypes = [P, ct.POINTER(Derived)]
        L.orc_init.argtypes = [P, _D, _D, _D]
        L.orc_step.argtypes = [P, _D, _D, ct.c_longlong]
        L.orc_step_detail.argtypes = [P, _D, _D, _D, _D, _D, _D, _D]
        L.orc_moments.argtypes = [P, _D, _D, _D]
        L.orc_sc_force.argtypes = [P, _D, _D]
        L.orc_polymer_stress.argtypes = [P, ct.POINTER(Derived), _D, _D, _D]
        L.orc_polymer_force.argtypes = [P, _D, _D]
        L.orc_fene_update.argtypes = [P, _D, _D, _D]
        L.orc_stream.argtypes = [P, _D, _D, _D]
        L.orc_observables.argtypes = [P, _D, ct.c_int, ct.POINTER(Obs)]
        L.orc_count_components.argtypes = [P, _D]
        L.orc_eig3.argtypes = [_D, _D, _D]
        L.orc_profile.argtypes = [ct.POINTER(ct.c_longlong), ct.c_int] + [ct.POINTER(ct.c_int)] * 4
        _lib = L
    return _lib


def make_params(d: dict) -> Params:
    p = Params()
    p.Lx, p.Ly, p.Lz = int(d["Lx"]), int(d["Ly"]), int(d["Lz"])
    p.visco_phase = int(d.get("visco_phase", 0))
    p.Uw = float(d.get("Uw", 0.0))
    p.G = float(d.get("G", 0.0))
    p.eta_M = float(d["eta_M"])
    p.lambda_ = float(d.get("lambda", 1.0))
    p.eta_P = float(d.get("eta_P", 0.0))
    p.tau_P = float(d.get("tau_P", 1.0))
    p.L2 = float(d.get("L2", 100.0))
    p.rho_in = float(d.get("rho_in", 1.0))
    p.rho_out = float(d.get("rho_out", 0.0))
    g = d.get("g", (0.0, 0.0, 0.0))
    p.gx, p.gy, p.gz = float(g[0]), float(g[1]), float(g[2])
    p.advection = int(d.get("advection", 0))
    return p


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class Oracle:
    """One oracle simulation: state (f, C) in float64 and the parameters."""

    def __init__(self, params: dict, rho_init: np.ndarray | None = None):
        self.d = dict(params)
        self.p = make_params(params)
        Lx, Ly, Lz = self.p.Lx, self.p.Ly, self.p.Lz
        self.shape = (Lz, Ly, Lx)
        self.N = Lx * Ly * Lz
        self.f = np.zeros((2, 19) + self.shape)
        self.C = np.zeros((6,) + self.shape)
        if rho_init is not None:
            self.init(rho_init)

    def derived(self) -> Derived:
        d = Derived()
        rc = lib().orc_derive(ct.byref(self.p), ct.byref(d))
        if rc:
            raise ValueError("invalid parameters for the oracle")
        return d

    def init(self, rho_init: np.ndarray):
        rho = np.ascontiguousarray(rho_init, dtype=np.float64).reshape((2,) + self.shape)
        self.derived()
        lib().orc_init(ct.byref(self.p), _ptr(rho), _ptr(self.f), _ptr(self.C))

    def step(self, n: int = 1):
        rc = lib().orc_step(ct.byref(self.p), _ptr(self.f), _ptr(self.C), int(n))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")

    def detail(self):
        """Intermediate fields of one step (f and C unchanged)."""
        fpost = np.zeros_like(self.f)
        rho = np.zeros((2,) + self.shape)
        u = np.zeros((3,) + self.shape)
        Ftot = np.zeros((2, 3) + self.shape)
        Cn = np.zeros_like(self.C)
        rc = lib().orc_step_detail(ct.byref(self.p), _ptr(self.f), _ptr(self.C), _ptr(fpost),
                                   _ptr(rho), _ptr(u), _ptr(Ftot), _ptr(Cn))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")
        return dict(fpost=fpost, rho=rho, u=u, Ftot=Ftot, Cnew=Cn)

    def observables(self, indicator_fp32: bool = False) -> dict:
        o = Obs()
        lib().orc_observables(ct.byref(self.p), _ptr(self.f), int(indicator_fp32), ct.byref(o))
        return obs_to_dict(o)

    def components(self) -> int:
        return lib().orc_count_components(ct.byref(self.p), _ptr(self.f))


def obs_to_dict(o: Obs) -> dict:
    return dict(mass=(o.mass[0], o.mass[1]), volume=o.volume, centroid=tuple(o.centroid),
                D=o.D, theta_deg=o.theta_deg, Lp=o.Lp, M=tuple(o.M), necks=o.necks,
                fragments=o.fragments, broken=o.broken, nan_seen=o.nan_seen)


# --- direct access to the sub-steps (used by the pins) ----------------------

def sc_force(params: dict, rho: np.ndarray) -> np.ndarray:
    p = make_params(params)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.zeros((2, 3) + rho.shape[1:])
    lib().orc_sc_force(ct.byref(p), _ptr(rho), _ptr(out))
    return out


def polymer_force(params: dict, rho: np.ndarray, C: np.ndarray) -> np.ndarray:
    p = make_params(params)
    d = Derived()
    if lib().orc_derive(ct.byref(p), ct.byref(d)):
        raise ValueError("invalid parameters")
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    Pi = np.zeros((6,) + rho.shape[1:])
    FP = np.zeros((3,) + rho.shape[1:])
    lib().orc_polymer_stress(ct.byref(p), ct.byref(d), _ptr(rho), _ptr(C), _ptr(Pi))
    lib().orc_polymer_force(ct.byref(p), _ptr(Pi), _ptr(FP))
    return FP


def fene_update(params: dict, C: np.ndarray, u: np.ndarray) -> np.ndarray:
    p = make_params(params)
    C = np.ascontiguousarray(C, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(C)
    lib().orc_fene_update(ct.byref(p), _ptr(C), _ptr(u), _ptr(out))
    return out


def eig3(Msym) -> tuple[np.ndarray, np.ndarray]:
    M = np.ascontiguousarray(np.asarray(Msym, dtype=np.float64))
    ev = np.zeros(3)
    V = np.zeros(9)
    lib().orc_eig3(_ptr(M), _ptr(ev), _ptr(V))
    return ev, V.reshape(3, 3)


def profile(A) -> dict:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.int64))
    outs = [ct.c_int() for _ in range(4)]
    lib().orc_profile(A.ctypes.data_as(ct.POINTER(ct.c_longlong)), int(A.size), *[ct.byref(o) for o in outs])
    return dict(Lp=outs[0].value, start=outs[1].value, necks=outs[2].value, fragments=outs[3].value)

"""Python binding of the C ABI in ``include/lbfe.h`` (argument marshalling only).

PyTorch supplies the device block and the CUDA stream; every step of the
method runs in the CUDA kernels of ``liblbfe.so``.  Importing this module
loads that library and raises if it has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import asdict

import numpy as np

from .params import (Params, FP32, FP16_OFFSET, BF16_OFFSET, NEWTONIAN, DROPLET_VISCOELASTIC, MATRIX_VISCOELASTIC,
                     ADVECTION_UPWIND1, ADVECTION_UPWIND2_MINMOD)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbfe.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"liblbfe.so is not built ({LIB_PATH}); run paper_1411_2181_gb300/build.py")

_lib = ct.CDLL(LIB_PATH)

FIELD_F, FIELD_C, FIELD_RHO, FIELD_U = 0, 1, 2, 3
STEP_CELL, STEP_PAIR = 0, 1   # lbfe_step_kernel
INJECT_SHORT_COPIES = 1       # lbfe_test_inject

OK, ERR_BAD_PARAM, ERR_NO_MEMORY, ERR_CUDA, ERR_DIVERGED, ERR_TIMEOUT, ERR_STATE, ERR_IO = range(8)


class CParams(ct.Structure):
    _fields_ = [("Lx", ct.c_int), ("Ly", ct.c_int), ("Lz", ct.c_int), ("visco_phase", ct.c_int),
                ("precision", ct.c_int), ("advection", ct.c_int),
                ("R", ct.c_double), ("Uw", ct.c_double), ("G", ct.c_double), ("eta_M", ct.c_double),
                ("lambda_", ct.c_double), ("eta_P", ct.c_double), ("tau_P", ct.c_double),
                ("L2", ct.c_double), ("rho_in", ct.c_double), ("rho_out", ct.c_double),
                ("sigma", ct.c_double), ("g", ct.c_double * 3), ("rho0", ct.c_double * 2)]


class CDerived(ct.Structure):
    _fields_ = [(n, ct.c_double) for n in
                ("nu_A", "nu_B", "tau_A", "tau_B", "pi_coef", "gamma_dot", "Ca", "tau_em", "De", "De_N1")]


class CObs(ct.Structure):
    _fields_ = [("step", ct.c_longlong), ("mass", ct.c_double * 2), ("volume", ct.c_double),
                ("centroid", ct.c_double * 3), ("M", ct.c_double * 6), ("D", ct.c_double),
                ("theta_deg", ct.c_double), ("Lp", ct.c_double), ("Lp_over_2R", ct.c_double),
                ("t_over_tem", ct.c_double), ("necks", ct.c_int), ("fragments", ct.c_int),
                ("broken", ct.c_int), ("flags", ct.c_int)]


_H = ct.c_void_p
_P = ct.POINTER(CParams)
_lib.lbfe_status_str.restype = ct.c_char_p
_lib.lbfe_status_str.argtypes = [ct.c_int]
_lib.lbfe_last_cuda_error.restype = ct.c_char_p
_lib.lbfe_params_size.restype = ct.c_size_t
_lib.lbfe_obs_size.restype = ct.c_size_t
_lib.lbfe_derive.argtypes = [_P, ct.POINTER(CDerived)]
_lib.lbfe_required_bytes.argtypes = [_P, ct.c_int, ct.POINTER(ct.c_size_t)]
_lib.lbfe_create.argtypes = [ct.POINTER(_H), _P, ct.c_int, ct.c_void_p, ct.c_size_t, ct.c_void_p]
_lib.lbfe_init.argtypes = [_H, ct.c_int, ct.POINTER(ct.c_double)]
_lib.lbfe_step.argtypes = [_H, ct.c_longlong]
_lib.lbfe_observables.argtypes = [_H, ct.c_int, ct.POINTER(CObs)]
_lib.lbfe_check.argtypes = [_H]
_lib.lbfe_get_field.argtypes = [_H, ct.c_int, ct.c_int, ct.c_void_p, ct.c_size_t]
_lib.lbfe_set_field.argtypes = [_H, ct.c_int, ct.c_int, ct.c_void_p, ct.c_size_t]
_lib.lbfe_destroy.argtypes = [_H]
_lib.lbfe_launches_per_step.argtypes = [_H]
_lib.lbfe_launches_per_step.restype = ct.c_int
_lib.lbfe_tune.argtypes = [_H, ct.c_int, ct.c_int, ct.c_int]
_lib.lbfe_tune.restype = ct.c_int
_lib.lbfe_launch_config.argtypes = [_H] + [ct.POINTER(ct.c_int)] * 5
_lib.lbfe_launch_config.restype = ct.c_int
_lib.lbfe_test_inject.argtypes = [_H, ct.c_uint]
_lib.lbfe_test_inject.restype = ct.c_int
_lib.lbfe_save.argtypes = [_H, ct.c_int, ct.c_char_p]
_lib.lbfe_save.restype = ct.c_int
_lib.lbfe_load.argtypes = [_H, ct.c_int, ct.c_char_p]
_lib.lbfe_load.restype = ct.c_int
_lib.lbfe_crc32.argtypes = [ct.c_void_p, ct.c_size_t, ct.c_uint]
_lib.lbfe_crc32.restype = ct.c_uint
_lib.lbfe_columns_bytes.argtypes = [_H, ct.c_int, ct.c_int, ct.POINTER(ct.c_size_t)]
_lib.lbfe_columns_bytes.restype = ct.c_int
_lib.lbfe_get_columns.argtypes = [_H, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p]
_lib.lbfe_get_columns.restype = ct.c_int
_lib.lbfe_set_columns.argtypes = [_H, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p]
_lib.lbfe_set_columns.restype = ct.c_int
_lib.lbfe_observables_noalloc.argtypes = [_P, ct.c_void_p, ct.c_longlong, ct.POINTER(CObs), ct.c_void_p]
_lib.lbfe_observables_noalloc.restype = ct.c_int
for _fn in ("lbfe_derive", "lbfe_required_bytes", "lbfe_create", "lbfe_init", "lbfe_step",
            "lbfe_observables", "lbfe_check", "lbfe_get_field", "lbfe_set_field", "lbfe_destroy"):
    getattr(_lib, _fn).restype = ct.c_int

assert _lib.lbfe_params_size() == ct.sizeof(CParams), "lbfe_params layout mismatch"
assert _lib.lbfe_obs_size() == ct.sizeof(CObs), "lbfe_obs layout mismatch"


def _to_c(p: Params) -> CParams:
    c = CParams()
    for k, v in asdict(p).items():
        if k in ("g", "rho0"):
            arr = getattr(c, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        else:
            setattr(c, k, v)
    return c


class LbfeError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.lbfe_status_str(status).decode()
        if status == ERR_CUDA:
            msg += ": " + _lib.lbfe_last_cuda_error().decode()
        super().__init__(f"{where}: {msg}")
        self.status = status


def _check(status: int, where: str):
    if status != OK:
        raise LbfeError(status, where)


def derive(p: Params) -> dict:
    d = CDerived()
    _check(_lib.lbfe_derive(ct.byref(_to_c(p)), ct.byref(d)), "lbfe_derive")
    return {n: getattr(d, n) for n, _ in CDerived._fields_}


def required_bytes(params: list[Params]) -> int:
    arr = (CParams * len(params))(*[_to_c(p) for p in params])
    nb = ct.c_size_t()
    _check(_lib.lbfe_required_bytes(arr, len(params), ct.byref(nb)), "lbfe_required_bytes")
    return nb.value


def obs_to_dict(o: CObs) -> dict:
    return dict(step=o.step, mass=(o.mass[0], o.mass[1]), volume=o.volume, centroid=tuple(o.centroid),
                M=tuple(o.M), D=o.D, theta_deg=o.theta_deg, Lp=o.Lp, Lp_over_2R=o.Lp_over_2R,
                t_over_tem=o.t_over_tem, necks=o.necks, fragments=o.fragments, broken=o.broken,
                flags=o.flags)


def observables_noalloc(p: Params, f_dev_ptr: int, stride: int, stream_ptr: int = 0) -> dict:
    """Observables of a device population field the caller holds (see
    ``lbfe_observables_noalloc``): no allocation inside the call."""
    o = CObs()
    c = _to_c(p)
    _check(_lib.lbfe_observables_noalloc(ct.byref(c), ct.c_void_p(f_dev_ptr), int(stride), ct.byref(o),
                                         ct.c_void_p(stream_ptr)), "lbfe_observables_noalloc")
    return obs_to_dict(o)


class Solver:
    """A batch of droplet instances advanced together on one GPU.

    ``device`` and ``stream`` default to torch's current ones; the device
    block is one torch tensor held by the solver."""

    def __init__(self, params: Params | list[Params], device=None, stream=None):
        import torch
        self.params = [params] if isinstance(params, Params) else list(params)
        self.n = len(self.params)
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        nbytes = required_bytes(self.params)
        self.block = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        arr = (CParams * self.n)(*[_to_c(p) for p in self.params])
        h = _H()
        _check(_lib.lbfe_create(ct.byref(h), arr, self.n, ct.c_void_p(self.block.data_ptr()), nbytes,
                                ct.c_void_p(self.stream.cuda_stream)), "lbfe_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.lbfe_destroy(h)
            self._h = None

    def close(self):
        self.__del__()

    def init(self, k: int, rho_init: np.ndarray):
        p = self.params[k]
        rho = np.ascontiguousarray(rho_init, dtype=np.float64)
        assert rho.size == 2 * p.N, "rho_init must be [2][Lz][Ly][Lx]"
        _check(_lib.lbfe_init(self._h, k, rho.ctypes.data_as(ct.POINTER(ct.c_double))), "lbfe_init")

    def init_from_host_ptr(self, k: int, ptr: int):
        """Initialise from a raw host pointer (e.g. pinned memory) to float64 [2][N]."""
        _check(_lib.lbfe_init(self._h, k, ct.cast(ct.c_void_p(ptr), ct.POINTER(ct.c_double))), "lbfe_init")

    def step(self, n: int = 1):
        _check(_lib.lbfe_step(self._h, int(n)), "lbfe_step")

    def observables(self, k: int = 0, raise_on_diverged: bool = True) -> dict:
        o = CObs()
        st = _lib.lbfe_observables(self._h, k, ct.byref(o))
        if st != OK and not (st == ERR_DIVERGED and not raise_on_diverged):
            _check(st, "lbfe_observables")
        return obs_to_dict(o)

    def launches_per_step(self) -> int:
        return _lib.lbfe_launches_per_step(self._h)

    def tune(self, tile_y: int = 8, z_chunk: int = 0, kernel: int = 0):
        """Launch shape of the step: kernel STEP_CELL (tile_y in 8, 12, 16) or
        STEP_PAIR (tile_y 16, even Lx), and the z-chunk depth (0 = auto)."""
        _check(_lib.lbfe_tune(self._h, int(kernel), int(tile_y), int(z_chunk)), "lbfe_tune")

    def launch_config(self) -> dict:
        v = [ct.c_int() for _ in range(5)]
        _check(_lib.lbfe_launch_config(self._h, *[ct.byref(x) for x in v]), "lbfe_launch_config")
        return dict(kernel=v[0].value, tile_y=v[1].value, z_chunk=v[2].value, grid=v[3].value, items=v[4].value)

    def check(self) -> int:
        return _lib.lbfe_check(self._h)

    def save(self, k: int, path: str):
        """Checkpoint instance k to a file (lbfe_save)."""
        _check(_lib.lbfe_save(self._h, int(k), os.fsencode(path)), "lbfe_save")

    def load(self, k: int, path: str):
        """Resume instance k from a checkpoint written by save (lbfe_load)."""
        _check(_lib.lbfe_load(self._h, int(k), os.fsencode(path)), "lbfe_load")

    def test_inject(self, what: int):
        """Test hook of the step kernel's failure path (lbfe_test_inject)."""
        _check(_lib.lbfe_test_inject(self._h, int(what)), "lbfe_test_inject")

    def columns_bytes(self, k: int, nx: int) -> int:
        nb = ct.c_size_t()
        _check(_lib.lbfe_columns_bytes(self._h, int(k), int(nx), ct.byref(nb)), "lbfe_columns_bytes")
        return nb.value

    def get_columns(self, k: int, x0: int, nx: int, dev_ptr: int):
        """Stored state of x-columns [x0, x0 + nx) into a device buffer (lbfe_get_columns)."""
        _check(_lib.lbfe_get_columns(self._h, int(k), int(x0), int(nx), ct.c_void_p(dev_ptr)), "lbfe_get_columns")

    def set_columns(self, k: int, x0: int, nx: int, dev_ptr: int):
        """A column block from a device buffer into x-columns [x0, x0 + nx) (lbfe_set_columns)."""
        _check(_lib.lbfe_set_columns(self._h, int(k), int(x0), int(nx), ct.c_void_p(dev_ptr)), "lbfe_set_columns")

    def _shape(self, k, which):
        p = self.params[k]
        lead = {FIELD_F: (2, 19), FIELD_C: (6,), FIELD_RHO: (2,), FIELD_U: (3,)}[which]
        return lead + (p.Lz, p.Ly, p.Lx)

    def get_field(self, k: int, which: int) -> np.ndarray:
        out = np.empty(self._shape(k, which), dtype=np.float32)
        _check(_lib.lbfe_get_field(self._h, k, which, out.ctypes.data, out.nbytes), "lbfe_get_field")
        return out

    def set_field(self, k: int, which: int, data: np.ndarray):
        arr = np.ascontiguousarray(data, dtype=np.float32).reshape(self._shape(k, which))
        _check(_lib.lbfe_set_field(self._h, k, which, arr.ctypes.data, arr.nbytes), "lbfe_set_field")

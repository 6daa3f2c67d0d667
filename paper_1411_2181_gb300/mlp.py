"""Python binding of ``include/lbfe_mlp.h`` (argument marshalling only) and
the training loop of the Ca_cr proposal network.

Every forward, backward and AdamW computation runs in the CUDA kernels of
``liblbfe.so``; PyTorch supplies the device block, the device copies of
the batch and the stream.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from .lbfe import _lib, _check

_M = ct.c_void_p
_F = ct.POINTER(ct.c_float)
_lib.lbfe_mlp_param_count.restype = ct.c_size_t
_lib.lbfe_mlp_required_bytes.argtypes = [ct.c_int, ct.POINTER(ct.c_size_t)]
_lib.lbfe_mlp_create.argtypes = [ct.POINTER(_M), ct.c_int, ct.c_int, ct.c_void_p, ct.c_size_t, ct.c_void_p]
_lib.lbfe_mlp_set_params.argtypes = [_M, _F]
_lib.lbfe_mlp_get_params.argtypes = [_M, _F]
_lib.lbfe_mlp_forward.argtypes = [_M, ct.c_void_p, ct.c_int, ct.c_void_p]
_lib.lbfe_mlp_loss_grad.argtypes = [_M, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int, _F]
_lib.lbfe_mlp_get_grads.argtypes = [_M, _F]
_lib.lbfe_mlp_adamw.argtypes = [_M, ct.c_float, ct.c_float, ct.c_float, ct.c_float, ct.c_float]
_lib.lbfe_mlp_destroy.argtypes = [_M]
for _fn in ("lbfe_mlp_required_bytes", "lbfe_mlp_create", "lbfe_mlp_set_params", "lbfe_mlp_get_params",
            "lbfe_mlp_forward", "lbfe_mlp_loss_grad", "lbfe_mlp_get_grads", "lbfe_mlp_adamw", "lbfe_mlp_destroy"):
    getattr(_lib, _fn).restype = ct.c_int

DIMS = (6, 128, 128, 128, 128, 4)
N_PARAMS = int(_lib.lbfe_mlp_param_count())


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, in the flat [Wt, b] per-layer layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(DIMS) - 1):
        i, j = DIMS[l], DIMS[l + 1]
        parts.append(rng.normal(0.0, np.sqrt(2.0 / i), size=(i, j)).ravel())
        parts.append(np.zeros(j))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == N_PARAMS
    return p


class MLP:
    """The proposal network on one GPU (device block held as a torch tensor)."""

    def __init__(self, max_batch: int = 4096, bf16: bool = True, device=None, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        nb = ct.c_size_t()
        _check(_lib.lbfe_mlp_required_bytes(int(max_batch), ct.byref(nb)), "lbfe_mlp_required_bytes")
        self.block = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        h = _M()
        _check(_lib.lbfe_mlp_create(ct.byref(h), int(max_batch), int(bool(bf16)),
                                    ct.c_void_p(self.block.data_ptr()), nb.value,
                                    ct.c_void_p(self.stream.cuda_stream)), "lbfe_mlp_create")
        self._h = h
        self.max_batch = max_batch

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.lbfe_mlp_destroy(h)
            self._h = None

    def _dev(self, a, cols):
        t = self.torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32).reshape(-1, cols) if cols else
                                 np.ascontiguousarray(a, dtype=np.float32))
        return t.to(self.device, non_blocking=False).contiguous()

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == N_PARAMS
        _check(_lib.lbfe_mlp_set_params(self._h, p.ctypes.data_as(_F)), "lbfe_mlp_set_params")

    def get_params(self) -> np.ndarray:
        p = np.empty(N_PARAMS, dtype=np.float32)
        _check(_lib.lbfe_mlp_get_params(self._h, p.ctypes.data_as(_F)), "lbfe_mlp_get_params")
        return p

    def forward(self, x) -> np.ndarray:
        xd = self._dev(x, 6)
        B = xd.shape[0]
        yd = self.torch.empty((B, 4), dtype=self.torch.float32, device=self.device)
        self.torch.cuda.synchronize(self.device)
        _check(_lib.lbfe_mlp_forward(self._h, ct.c_void_p(xd.data_ptr()), B, ct.c_void_p(yd.data_ptr())),
               "lbfe_mlp_forward")
        self.stream.synchronize()
        return yd.cpu().numpy()

    def loss_grad(self, x, t, mask=None) -> float:
        xd, td = self._dev(x, 6), self._dev(t, 4)
        md = self._dev(mask, 0) if mask is not None else None
        self.torch.cuda.synchronize(self.device)
        loss = ct.c_float()
        _check(_lib.lbfe_mlp_loss_grad(self._h, ct.c_void_p(xd.data_ptr()), ct.c_void_p(td.data_ptr()),
                                       ct.c_void_p(md.data_ptr() if md is not None else 0), xd.shape[0],
                                       ct.byref(loss)), "lbfe_mlp_loss_grad")
        return loss.value

    def grads(self) -> np.ndarray:
        g = np.empty(N_PARAMS, dtype=np.float32)
        _check(_lib.lbfe_mlp_get_grads(self._h, g.ctypes.data_as(_F)), "lbfe_mlp_get_grads")
        return g

    def adamw(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
        _check(_lib.lbfe_mlp_adamw(self._h, lr, beta1, beta2, eps, weight_decay), "lbfe_mlp_adamw")

    def fit(self, X, T, M=None, epochs=2000, lr=2e-3, weight_decay=1e-4, batch=None, seed=0,
            lr_final=1e-4, verbose=False):
        """Mini-batch AdamW with a cosine learning-rate decay; returns the
        loss history (one value per epoch)."""
        torch = self.torch
        X = np.asarray(X, np.float32)
        T = np.asarray(T, np.float32)
        M = np.ones(len(X), np.float32) if M is None else np.asarray(M, np.float32)
        n = len(X)
        bs = min(batch or n, self.max_batch)
        rng = np.random.default_rng(seed)
        Xd, Td, Md = self._dev(X, 6), self._dev(T, 4), self._dev(M, 0)
        hist = []
        for ep in range(epochs):
            perm = torch.as_tensor(rng.permutation(n), device=self.device)
            lr_e = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * ep / max(1, epochs - 1)))
            tot = 0.0
            for s in range(0, n, bs):
                idx = perm[s:s + bs]
                xb, tb, mb = Xd[idx].contiguous(), Td[idx].contiguous(), Md[idx].contiguous()
                torch.cuda.synchronize(self.device)
                loss = ct.c_float()
                _check(_lib.lbfe_mlp_loss_grad(self._h, ct.c_void_p(xb.data_ptr()), ct.c_void_p(tb.data_ptr()),
                                               ct.c_void_p(mb.data_ptr()), xb.shape[0], ct.byref(loss)),
                       "lbfe_mlp_loss_grad")
                _check(_lib.lbfe_mlp_adamw(self._h, float(lr_e), 0.9, 0.999, 1e-8, float(weight_decay)),
                       "lbfe_mlp_adamw")
                tot += loss.value * xb.shape[0]
            hist.append(tot / n)
            if verbose and ep % max(1, epochs // 10) == 0:
                print(f"epoch {ep} loss {hist[-1]:.5f}")
        return hist

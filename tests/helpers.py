"""Shared helpers of the test-suite (no method arithmetic)."""
import numpy as np


def norm_err(gpu: np.ndarray, ref: np.ndarray, lead: int) -> float:
    """max over arrays of max |gpu - ref| / max |ref| (one array per index of
    the first ``lead`` axes): the per-population (per-component) normalised
    error; pointwise relative error is ill-posed for the dissolved
    component's populations."""
    g = gpu.reshape(int(np.prod(gpu.shape[:lead])), -1).astype(np.float64)
    r = ref.reshape(g.shape[0], -1)
    scale = np.abs(r).max(axis=1)
    scale[scale == 0] = 1.0
    return float((np.abs(g - r).max(axis=1) / scale).max())


def random_populations(shape, seed, amp=0.03):
    """Non-equilibrium populations around w_i rho for a random state."""
    from paper_1411_2181_gb300 import synth
    Lx, Ly, Lz = shape
    rho, vel, C = synth.random_state(Lx, Ly, Lz, seed, amp=amp)
    cx = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0])
    cy = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1])
    cz = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1])
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    rng = np.random.default_rng(seed + 1)
    f = np.empty((2, 19, Lz, Ly, Lx))
    for s in range(2):
        cu = (cx[:, None, None, None] * vel[0] + cy[:, None, None, None] * vel[1]
              + cz[:, None, None, None] * vel[2])
        uu = (vel ** 2).sum(0)
        f[s] = w[:, None, None, None] * rho[s] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu)
        f[s] *= 1 + rng.uniform(-0.01, 0.01, f[s].shape)
    return f.astype(np.float32).astype(np.float64), C.astype(np.float32).astype(np.float64)


def tensor_err(gpu: np.ndarray, ref: np.ndarray) -> float:
    """max |C_gpu - C_ref| over cells and components, divided by the largest
    |C_ref| component: a tensor-wide scale (the components mix under
    rotation, and components that vanish by symmetry have no scale of their
    own)."""
    return float(np.abs(gpu.astype(np.float64) - ref).max() / np.abs(ref).max())


def component_report(gpu: np.ndarray, ref: np.ndarray) -> str:
    g = gpu.reshape(gpu.shape[0], -1).astype(np.float64)
    r = ref.reshape(ref.shape[0], -1)
    return "; ".join(f"k{k}: |d|max={np.abs(g[k]-r[k]).max():.2e} |ref|max={np.abs(r[k]).max():.2e}"
                     for k in range(g.shape[0]))


C_NAMES = ("xx", "yy", "zz", "xy", "xz", "yz")


def component_errors(gpu: np.ndarray, ref: np.ndarray) -> dict:
    """Per conformation component k: (max |C_gpu,k - C_ref,k| / max |C_ref,k|,
    max |C_ref,k|), each component normalised by its own scale."""
    g = gpu.reshape(6, -1).astype(np.float64)
    r = ref.reshape(6, -1)
    out = {}
    for k, name in enumerate(C_NAMES):
        scale = float(np.abs(r[k]).max())
        out[name] = (float(np.abs(g[k] - r[k]).max() / scale) if scale > 0 else 0.0, scale)
    return out

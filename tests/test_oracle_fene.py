"""Pins of the oracle's finite-difference FENE-P update (Eq. 2 / Eq. 4)
against the paper's steady homogeneous-shear solution (Eqs. 6 and 7), the
Oldroyd-B start-up limit and exact properties of the stencils (no GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1411_2181_gb300 import synth


def couette_u(Lx, Ly, Lz, Uw):
    """u_x = Uw (2 (z+1/2)/W - 1): linear with shear rate 2 Uw/W, and
    consistent with the wall ghosts u_ghost = 2 U_wall - u."""
    z = np.arange(Lz)
    u = np.zeros((3, Lz, Ly, Lx))
    u[0] = (Uw * (2 * (z + 0.5) / Lz - 1))[:, None, None]
    return u


def iterate(p, C, u, n):
    for _ in range(n):
        C = O.fene_update(p, C, u)
    return C


def identity_C(Lx, Ly, Lz):
    C = np.zeros((6, Lz, Ly, Lx))
    C[:3] = 1.0
    return C


def test_oldroyd_b_startup_discrete_closed_form():
    """L^2 -> infinity (f = 1): the explicit update of the homogeneous
    start-up gives C_xz^n = tau gdot (1 - (1 - 1/tau)^n) exactly, C_zz = 1."""
    Lx, Ly, Lz, Uw = 2, 2, 4, 0.02
    gdot = 2 * Uw / Lz
    tau = 50.0
    p = dict(Lx=Lx, Ly=Ly, Lz=Lz, Uw=Uw, eta_M=1, tau_P=tau, L2=1e14)
    u = couette_u(Lx, Ly, Lz, Uw)
    C = identity_C(Lx, Ly, Lz)
    for n in range(1, 301):
        C = O.fene_update(p, C, u)
        exact = tau * gdot * (1 - (1 - 1 / tau) ** n)
        assert np.abs(C[4] - exact).max() < 1e-11 * tau * gdot
        assert np.abs(C[2] - 1).max() < 1e-12
        assert np.abs(C[1] - 1).max() < 1e-12
        if n == 300:
            # continuous start-up C_xz = tau gdot (1 - exp(-t/tau)), to O(1/tau)
            cont = tau * gdot * (1 - np.exp(-n / tau))
            assert abs(C[4].mean() - cont) < 2.0 / tau * tau * gdot


def test_oldroyd_b_steady_state():
    """Oldroyd-B steady shear: C_xz = Wi, C_xx = 1 + 2 Wi^2, C_yy = C_zz = 1."""
    Lx, Ly, Lz = 1, 1, 2
    tau, Wi = 20.0, 0.7
    gdot = Wi / tau
    Uw = gdot * Lz / 2
    p = dict(Lx=Lx, Ly=Ly, Lz=Lz, Uw=Uw, eta_M=1, tau_P=tau, L2=1e14)
    C = iterate(p, identity_C(Lx, Ly, Lz), couette_u(Lx, Ly, Lz, Uw), 2500)
    assert np.allclose(C[4], Wi, rtol=1e-10)
    assert np.allclose(C[0], 1 + 2 * Wi ** 2, rtol=1e-10)
    assert np.allclose(C[1], 1, rtol=1e-10) and np.allclose(C[2], 1, rtol=1e-10)
    assert np.abs(C[3]).max() < 1e-14 and np.abs(C[5]).max() < 1e-14


def eq_S(Wi, L2):
    """Eq. 6 divided by eta_P/tau_P: f C_xz in steady homogeneous shear."""
    return 2 * np.sqrt(L2 / 6) * np.sinh(np.arcsinh(Wi * L2 / 4 * (L2 / 6) ** -1.5) / 3)


def eq_N1(Wi, L2):
    """Eq. 7 divided by eta_P/tau_P: f (C_xx - C_yy)."""
    return 8 * (L2 / 6) * np.sinh(np.arcsinh(Wi * L2 / 4 * (L2 / 6) ** -1.5) / 3) ** 2


@pytest.mark.parametrize("L2", [100.0, 400.0])
@pytest.mark.parametrize("Wi", [0.1, 1.0, 10.0])
def test_fene_p_steady_shear_paper_closed_form(L2, Wi):
    """Eqs. 6 and 7: the FD update driven by u_x = gdot z converges to the
    paper's steady FENE-P shear stress and first normal-stress difference.
    This also fixes the index convention (grad u)_ij = d_i u_j: the
    transposed convention would stretch C_zz instead of C_xx."""
    Lx, Ly, Lz = 1, 1, 2
    tau = 20.0
    gdot = Wi / tau
    Uw = gdot * Lz / 2
    p = dict(Lx=Lx, Ly=Ly, Lz=Lz, Uw=Uw, eta_M=1, tau_P=tau, L2=L2)
    C = iterate(p, identity_C(Lx, Ly, Lz), couette_u(Lx, Ly, Lz, Uw), 3000)
    f = (L2 - 3) / (L2 - C[:3].sum(0))
    assert np.allclose(f * C[4], eq_S(Wi, L2), rtol=1e-9)
    assert np.allclose(f * (C[0] - C[1]), eq_N1(Wi, L2), rtol=1e-9)
    # the normal stresses in y and z relax to f C = 1
    assert np.allclose(f * C[1], 1, rtol=1e-9) and np.allclose(f * C[2], 1, rtol=1e-9)


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)])
def test_upwind_advection_is_exact_shift_at_unit_courant(axis, sign):
    """First-order upwind with |u| = 1, dt = 1 moves C by one cell per step
    (no polymer relaxation: tau_P -> infinity).  Wall-adjacent layers see the
    wall ghost velocity and are excluded."""
    Lx, Ly, Lz = 6, 5, 7
    _, _, C = synth.random_state(Lx, Ly, Lz, seed=5)
    u = np.zeros((3, Lz, Ly, Lx))
    u[axis] = sign
    p = dict(Lx=Lx, Ly=Ly, Lz=Lz, Uw=0.0, eta_M=1, tau_P=1e300, L2=1e14)
    Cn = O.fene_update(p, C, u)
    shifted = np.roll(C, sign, axis=3 - axis)
    assert np.abs(Cn - shifted)[:, 1:-1].max() < 1e-14


def test_velocity_gradient_central_difference():
    """With C = I and no relaxation, one update adds grad u + (grad u)^T;
    for u_x = A sin(k y), u_y = B sin(k' x) the central difference is
    C_xy = A sin(k) cos(k y) + B sin(k') cos(k' x), other components 0."""
    Lx, Ly, Lz = 8, 10, 3
    A, B = 0.03, -0.02
    k, kp = 2 * np.pi / Ly, 2 * np.pi / Lx
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    u = np.zeros((3, Lz, Ly, Lx))
    u[0] = A * np.sin(k * y)
    u[1] = B * np.sin(kp * x)
    p = dict(Lx=Lx, Ly=Ly, Lz=Lz, Uw=0.0, eta_M=1, tau_P=1e300, L2=1e14)
    C0 = identity_C(Lx, Ly, Lz)
    Cn = O.fene_update(p, C0, u)
    expect = A * np.sin(k) * np.cos(k * y) + B * np.sin(kp) * np.cos(kp * x)
    assert np.abs(Cn[3] - expect).max() < 1e-15
    assert np.abs(Cn[[0, 1, 2]] - 1).max() < 1e-15
    assert np.abs(Cn[[4, 5], 1:-1]).max() < 1e-15
    # wall layers: u_ghost = 2 U_wall - u (still walls) gives d_z u_x = +u_x
    # at the bottom layer and -u_x at the top layer
    assert np.abs(Cn[4, 0] - u[0, 0]).max() < 1e-15
    assert np.abs(Cn[4, -1] + u[0, -1]).max() < 1e-15
    assert np.abs(Cn[5, 0] - u[1, 0]).max() < 1e-15


def test_peterlin_relaxation_at_rest():
    """No flow: each step C -> C - (f C - I)/tau_P with f = (L^2-3)/(L^2-tr C)
    (Eq. 2); C = I is a fixed point and a stretched state relaxes towards it."""
    Lx, Ly, Lz = 2, 2, 2
    p = dict(Lx=Lx, Ly=Ly, Lz=Lz, Uw=0.0, eta_M=1, tau_P=10.0, L2=50.0)
    u = np.zeros((3, Lz, Ly, Lx))
    C0 = identity_C(Lx, Ly, Lz)
    assert np.abs(O.fene_update(p, C0, u) - C0).max() < 1e-15
    C = C0.copy()
    C[0] = 20.0
    tr = 22.0
    f = (50 - 3) / (50 - tr)
    Cn = O.fene_update(p, C, u)
    assert abs(Cn[0, 0, 0, 0] - (20 - (f * 20 - 1) / 10)) < 1e-13
    assert abs(Cn[1, 0, 0, 0] - (1 - (f - 1) / 10)) < 1e-13


# --- second-order minmod-limited upwind advection (advection = 1) -----------

def pure_advection_params(Lx, Ly, Lz, advection):
    """No relaxation (tau_P huge), no Peterlin factor (L^2 huge): with a
    uniform velocity the update is C - u . grad C alone."""
    return dict(Lx=Lx, Ly=Ly, Lz=Lz, Uw=0.0, eta_M=1, tau_P=1e30, L2=1e30, advection=advection)


def uniform_u(Lx, Ly, Lz, v, axis=0):
    u = np.zeros((3, Lz, Ly, Lx))
    u[axis] = v
    return u


@pytest.mark.parametrize("v", [0.3, -0.3])
def test_second_order_upwind_exact_on_monotone_quadratic(v):
    """On a convex monotone profile the minmod slopes pick the one-sided
    differences: the scheme becomes the three-point second-order upwind
    (v > 0) or the central difference (v < 0), both exact for a quadratic:
    u . grad C = v * 2 (x - x0)."""
    Lx, Ly, Lz, x0 = 40, 2, 2, 5.0
    p = pure_advection_params(Lx, Ly, Lz, 1)
    x = np.arange(Lx, dtype=float)
    C = identity_C(Lx, Ly, Lz)
    C[0] = ((x - x0) ** 2)[None, None, :]
    Cn = O.fene_update(p, C, uniform_u(Lx, Ly, Lz, v))
    D = (C[0] - Cn[0])[0, 0] / v
    cells = np.arange(int(x0) + 2, Lx - 2)
    assert np.allclose(D[cells], 2 * (x[cells] - x0), rtol=0, atol=1e-9)
    # the first-order scheme is off by the second difference there
    Cn1 = O.fene_update(pure_advection_params(Lx, Ly, Lz, 0), C, uniform_u(Lx, Ly, Lz, v))
    D1 = (C[0] - Cn1[0])[0, 0] / v
    assert np.allclose(np.abs(D1[cells] - 2 * (x[cells] - x0)), 1.0, atol=1e-9)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_second_order_upwind_is_bounded_and_sharper(axis):
    """Pure advection of a step at Courant number 0.25 along x, y (periodic)
    and z (walls): the limited scheme creates no new extremum, and it keeps
    the front sharper than the first-order scheme (smaller L1 distance to
    the exactly shifted profile).  Read on an interior plane and away from
    the walls: the wall ghosts u_ghost = -u of a uniform flow stretch C in
    the wall planes, which is not advection."""
    n = 48
    shape = [4, 4, 4]
    shape[axis] = n
    Lx, Ly, Lz = shape
    x = np.arange(n)
    prof = np.where((x >= 12) & (x < 24), 2.0, 1.0)
    def field():
        C = identity_C(Lx, Ly, Lz)
        sl = [None, None, None]
        sl[2 - axis] = slice(None)
        C[0] = np.broadcast_to(prof[tuple(sl)], (Lz, Ly, Lx)).copy()
        return C
    v, steps = 0.25, 40                       # shift of 10 cells
    err = {}
    for adv in (0, 1):
        p = pure_advection_params(Lx, Ly, Lz, adv)
        C = field()
        u = uniform_u(Lx, Ly, Lz, v, axis)
        for _ in range(steps):
            C = O.fene_update(p, C, u)
        line = np.moveaxis(C[0], 2 - axis, 0)[:, 1, 1]     # interior z (or y) = 1
        win = slice(11, 44)
        assert line[win].min() >= 1.0 - 1e-12 and line[win].max() <= 2.0 + 1e-12
        exact = np.where((x >= 22) & (x < 34), 2.0, 1.0)
        err[adv] = np.abs(line[win] - exact[win]).sum()
    assert err[1] < 0.75 * err[0]

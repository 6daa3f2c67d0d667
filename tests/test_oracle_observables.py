"""Pins of the oracle's droplet observables: deformation D and orientation
theta of known ellipsoids, projected length, necks and break-up of built
shapes, and brute-force checks (no GPU)."""
import numpy as np
import pytest

from oracle import oracle as O

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def fields_from_indicator(ind, rho_in=1.0, rho_out=0.04):
    """Populations at rest (f_i = w_i rho) for a droplet given by a mask."""
    rA = np.where(ind, rho_in, rho_out)
    rB = np.where(ind, rho_out, rho_in)
    return np.stack([W[:, None, None, None] * rA, W[:, None, None, None] * rB])


def oracle_with(ind):
    Lz, Ly, Lx = ind.shape
    o = O.Oracle(dict(Lx=Lx, Ly=Ly, Lz=Lz, eta_M=1.0))
    o.f[:] = fields_from_indicator(ind)
    return o


def ellipsoid(shape, center, axes, theta_deg):
    Lz, Ly, Lx = shape
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    th = np.deg2rad(theta_deg)
    dx, dy, dz = x - center[0], y - center[1], z - center[2]
    xr = np.cos(th) * dx + np.sin(th) * dz
    zr = -np.sin(th) * dx + np.cos(th) * dz
    return (xr / axes[0]) ** 2 + (dy / axes[1]) ** 2 + (zr / axes[2]) ** 2 <= 1


@pytest.mark.parametrize("theta", [0.0, 25.0, -40.0, 60.0])
def test_ellipsoid_deformation_and_orientation(theta):
    """Uniform ellipsoid with semi-axes (a, b, b): second moments V a^2/5,
    so D = (a-b)/(a+b) and theta is the tilt of the a-axis in x-z."""
    a, b = 14.0, 7.0
    ind = ellipsoid((48, 32, 64), (31.3, 15.6, 23.8), (a, b, b), theta)
    obs = oracle_with(ind).observables()
    assert abs(obs["D"] - (a - b) / (a + b)) < 0.01
    assert abs(obs["theta_deg"] - theta) < 0.5
    assert obs["volume"] == ind.sum()
    assert obs["necks"] == 0 and obs["fragments"] == 1 and obs["broken"] == 0


def test_moments_brute_force_and_periodic_wrap():
    """Brute force over the cells (numpy eigh) and invariance when the droplet
    straddles the periodic x boundary."""
    ind = ellipsoid((40, 24, 56), (27.2, 11.4, 19.1), (15.0, 6.0, 8.0), 33.0)
    o1 = oracle_with(ind).observables()
    z, y, x = np.nonzero(ind)
    X = np.stack([x, y, z]).astype(float)
    c = X.mean(1)
    M = (X - c[:, None]) @ (X - c[:, None]).T
    ev, V = np.linalg.eigh(M)
    a, b = np.sqrt(5 * ev[-1] / ind.sum()), np.sqrt(5 * ev[0] / ind.sum())
    th = np.degrees(np.arctan2(V[2, -1], V[0, -1]))
    th = th + 180 if th <= -90 else (th - 180 if th > 90 else th)
    assert abs(o1["D"] - (a - b) / (a + b)) < 1e-12
    assert abs(o1["theta_deg"] - th) < 1e-9
    assert np.allclose(o1["centroid"], c, atol=1e-9)
    assert o1["Lp"] == len(np.unique(x))
    rolled = np.roll(ind, 40, axis=2)
    o2 = oracle_with(rolled).observables()
    for k in ("D", "theta_deg", "Lp", "volume"):
        assert abs(o1[k] - o2[k]) < 1e-9
    assert abs(o2["centroid"][0] - (c[0] + 40) % 56) < 1e-9


def beads(shape, xs, R, neck_r):
    """Spheres of radius R centred on the axis at x in xs, joined by
    cylinders of radius neck_r (neck_r = 0: no joints)."""
    Lz, Ly, Lx = shape
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    cy, cz = (Ly - 1) / 2, (Lz - 1) / 2
    ind = np.zeros(shape, bool)
    for xc in xs:
        ind |= (x - xc) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= R * R
    if neck_r > 0:
        r2 = (y - cy) ** 2 + (z - cz) ** 2
        ind |= (r2 <= neck_r ** 2) & (x >= min(xs)) & (x <= max(xs))
    return ind


def test_single_neck_dumbbell():
    ind = beads((24, 24, 64), [18, 44], 7.0, 1.5)
    o = oracle_with(ind)
    obs = o.observables()
    assert obs["necks"] == 1 and obs["fragments"] == 1 and obs["broken"] == 0
    assert o.components() == 1


def test_two_necks_before_ternary_break_up():
    ind = beads((24, 24, 96), [20, 47, 74], 7.0, 1.5)
    obs = oracle_with(ind).observables()
    assert obs["necks"] == 2 and obs["broken"] == 0


def test_break_up_into_daughters():
    ind = beads((24, 24, 96), [20, 47, 74], 7.0, 0.0)
    o = oracle_with(ind)
    obs = o.observables()
    assert obs["fragments"] == 3 and obs["broken"] == 1 and obs["necks"] == 0
    assert o.components() == 3
    # a satellite below 1% of the volume does not count as a fragment
    ind2 = beads((24, 24, 96), [30], 9.0, 0.0)
    ind2[12, 12, 80] = True
    obs2 = oracle_with(ind2).observables()
    assert obs2["fragments"] == 1 and obs2["broken"] == 0


def test_profile_hand_cases():
    # plateau on a maximum, a shallow dip (not a neck), a deep dip (neck)
    r = O.profile([0, 0, 3, 8, 8, 7, 8, 2, 6, 1, 0, 0])
    assert r == dict(Lp=8, start=2, necks=1, fragments=1)
    # occupied across the periodic boundary
    r = O.profile([5, 6, 0, 0, 0, 0, 2, 4])
    assert r["Lp"] == 4 and r["start"] == 6 and r["necks"] == 0
    # all planes occupied: L_p = Lx
    r = O.profile([3, 3, 1, 3, 3, 3])
    assert r["Lp"] == 6 and r["necks"] == 1
    # two runs, second tiny (< 1%): one fragment
    r = O.profile([0, 200, 300, 0, 1, 0])
    assert r["fragments"] == 1
    assert O.profile([0, 0, 0])["Lp"] == 0


def test_eig3_matches_lapack():
    rng = np.random.default_rng(0)
    for _ in range(20):
        A = rng.normal(size=(3, 3))
        S = A + A.T
        ev, V = O.eig3([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]])
        assert np.allclose(np.sort(ev), np.linalg.eigvalsh(S), atol=1e-12)
        for k in range(3):
            assert np.allclose(S @ V[:, k], ev[k] * V[:, k], atol=1e-11)

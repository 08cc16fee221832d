"""Pins of the oracle's hexahedral hydro update (no GPU): hexahedron volume
against boxes, parallelepipeds and an independent 3-point Gauss quadrature of
numpy determinants; the volume gradient against finite differences and the
translation / scaling identities; the time step against the causal cone of a
nearest-neighbour stencil, axis-permutation symmetry, energy convergence under
time-step refinement, and determinism."""
import itertools

import numpy as np
import pytest

from paper_2308_16877_gb300 import workloads as W

CORNERS = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], dtype=np.float64)


def test_box_and_parallelepiped_volumes(orc):
    X, Y, Z = (CORNERS[:, k] for k in range(3))
    assert orc.hex_volume(X, Y, Z) == pytest.approx(1.0, rel=1e-15)
    assert orc.hex_volume(2 * X, 3 * Y, 0.5 * Z) == pytest.approx(3.0, rel=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(5):
        A = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
        b = rng.normal(size=3)
        P = CORNERS @ A.T + b
        assert orc.hex_volume(P[:, 0], P[:, 1], P[:, 2]) == pytest.approx(abs(np.linalg.det(A)), rel=1e-13)


def _volume_numpy(P):
    """Independent: 3-point Gauss-Legendre per axis on [0,1] of numpy det J."""
    gx, gw = np.polynomial.legendre.leggauss(3)
    gx, gw = 0.5 * (gx + 1.0), 0.5 * gw
    vol = 0.0
    for (a, wa), (b, wb), (c, wc) in itertools.product(zip(gx, gw), repeat=3):
        J = np.zeros((3, 3))
        for k, (i, j, l) in enumerate(CORNERS.astype(int)):
            fa, fb, fc = (a if i else 1 - a), (b if j else 1 - b), (c if l else 1 - c)
            da, db, dc = (1 if i else -1), (1 if j else -1), (1 if l else -1)
            J[:, 0] += P[k] * da * fb * fc
            J[:, 1] += P[k] * fa * db * fc
            J[:, 2] += P[k] * fa * fb * dc
        vol += wa * wb * wc * np.linalg.det(J)
    return vol


def test_distorted_hex_volume_matches_independent_quadrature(orc):
    rng = np.random.default_rng(1)
    for _ in range(10):
        P = CORNERS + 0.2 * rng.uniform(-1, 1, size=(8, 3))
        assert orc.hex_volume(P[:, 0], P[:, 1], P[:, 2]) == pytest.approx(_volume_numpy(P), rel=1e-13)


def test_volume_gradient(orc):
    rng = np.random.default_rng(2)
    P = CORNERS + 0.2 * rng.uniform(-1, 1, size=(8, 3))
    G = orc.hex_volume_grad(P[:, 0], P[:, 1], P[:, 2])
    h = 1e-6
    for c in range(8):
        for k in range(3):
            Pp, Pm = P.copy(), P.copy()
            Pp[c, k] += h
            Pm[c, k] -= h
            fd = (orc.hex_volume(*Pp.T) - orc.hex_volume(*Pm.T)) / (2 * h)
            assert G[k, c] == pytest.approx(fd, rel=1e-7, abs=1e-9)
    # translation invariance: the gradient sums to zero on every axis
    assert np.allclose(G.sum(axis=1), 0.0, atol=1e-14)
    # V is homogeneous of degree 3 in the positions: sum_c x_c . dV/dx_c = 3 V
    V = orc.hex_volume(*P.T)
    assert np.sum(P.T * G) == pytest.approx(3 * V, rel=1e-13)


def _run(orc, n, steps, jitter=W.HYDRO_JITTER, dt_scale=1.0):
    x, y, z, e = W.hydro_initial(n, jitter=jitter)
    S = orc.HydroState(n, x, y, z, e)
    dt = W.hydro_dt(n) * dt_scale
    for _ in range(steps):
        S.step(dt)
    return S


def test_initial_masses(orc):
    x, y, z, e = W.hydro_initial(8)
    S = orc.HydroState(8, x, y, z, e)
    assert S.V0.sum() == pytest.approx(1.0, rel=1e-13)      # jitter keeps the unit cube
    assert S.mnode.sum() == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("steps", [1, 3, 6])
def test_causal_cone(orc, steps):
    """Each step couples nearest neighbours only: elements more than `steps`
    elements away (Chebyshev) from the corner are untouched, bit for bit."""
    n = 12
    S = _run(orc, n, steps)
    E = n ** 3
    idx = np.arange(E)
    i, j, k = idx % n, (idx // n) % n, idx // (n * n)
    far = np.maximum(np.maximum(i, j), k) > steps
    assert np.all(S.e[far] == 0) and np.all(S.p[far] == 0) and np.all(S.q[far] == 0)
    assert np.all(S.vrel[far] == 1.0)
    near = np.maximum(np.maximum(i, j), k) <= steps
    assert np.any(S.e[near & (idx > 0)] > 0)
    n1 = n + 1
    nd = np.arange(n1 ** 3)
    ni, nj, nk = nd % n1, (nd // n1) % n1, nd // (n1 * n1)
    nfar = np.maximum(np.maximum(ni, nj), nk) > steps
    assert np.all(S.u[nfar] == 0) and np.all(S.v[nfar] == 0) and np.all(S.w[nfar] == 0)


def test_axis_permutation_symmetry(orc):
    """Without jitter the problem is symmetric under swapping axes."""
    n = 10
    S = _run(orc, n, 20, jitter=0.0)
    e = S.e.reshape(n, n, n)          # [k, j, i]
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        assert np.allclose(e, e.transpose(perm), rtol=1e-10, atol=1e-6 * e.max())


def test_energy_conservation_in_the_limit_of_small_time_steps(orc):
    """Total energy (internal + kinetic) is not conserved step by step: the
    nodal forces use p + q of the step's start and the old and new velocities'
    mean, while the energy update charges the trapezoid pressure and the new
    viscosity against the volume change, which differ by O(dt) per unit of
    work. So the drift at equal physical time is first order in dt, and its
    Richardson extrapolation to dt -> 0 (2 D(dt/2) - D(dt)) vanishes at second
    order: what an exactly consistent force and work pair gives. A force or
    work term scaled by 1 + eps adds eps times the work done (here ~40% of the
    energy becomes kinetic) at every dt, which the extrapolation exposes."""
    n = 10
    drift = []
    for scale, steps in ((1.0, 40), (0.5, 80), (0.25, 160)):
        x, y, z, e = W.hydro_initial(n)
        S = orc.HydroState(n, x, y, z, e)
        e0 = sum(S.energies())
        dt = W.hydro_dt(n) * scale
        for _ in range(steps):
            S.step(dt)
        ie, ke = S.energies()
        assert ke > 0.3 * e0                      # the blast did work
        drift.append((ie + ke - e0) / e0)
    d = np.array(drift)
    assert abs(d[0]) < 1e-2
    assert 0.45 < d[1] / d[0] < 0.55 and 0.45 < d[2] / d[1] < 0.55   # first order
    r = 2 * d[1:] - d[:-1]                        # extrapolated to dt -> 0
    assert abs(r[0]) < 0.1 * abs(d[1]) and abs(r[1]) < 0.35 * abs(r[0])  # second order
    assert abs(r[1]) < 5e-5


def test_step_is_deterministic_and_resumable(orc):
    n = 8
    a = _run(orc, n, 10)
    x, y, z, e = W.hydro_initial(n)
    b = orc.HydroState(n, x, y, z, e)
    dt = W.hydro_dt(n)
    for _ in range(5):
        b.step(dt)
    c = b.copy()                       # checkpoint, then resume from the copy
    for _ in range(5):
        c.step(dt)
    for f in orc.HydroState.FIELDS:
        assert np.array_equal(getattr(a, f), getattr(c, f)), f


def test_eos_inputs_are_what_the_region_receives(orc):
    """Under an exact EOS the new pressure equals the EOS region applied to the
    step's recorded inputs."""
    n = 8
    S = _run(orc, n, 4)
    eos_in, mask, cnt = S.step(W.hydro_dt(n))
    p = orc.run_exact(orc.EOS, eos_in, orc.GAMMA)
    assert np.array_equal(p, S.p)
    assert np.all(mask == 0)


def test_taf_on_eos_with_zero_threshold_is_exact(orc):
    n = 8
    A = _run(orc, n, 3)
    B = A.copy()
    dt = W.hydro_dt(n)
    A.step(dt)
    B.step(dt, orc.eos_knobs(orc.EOS_TAF, hsize=2, psize=4, thresh=0.0, threads=64, block=64))
    for f in orc.HydroState.FIELDS:
        assert np.array_equal(getattr(A, f), getattr(B, f)), f

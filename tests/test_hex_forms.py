"""The element kernel evaluates the trilinear hexahedron's volume in Grandy's
three-triple-product form (J. Grandy, "Efficient computation of volume of
hexahedral cells", LLNL UCRL-ID-128886, 1997) and its gradient by the product
rule on that form. This pins the identity on the CPU: the form, written here
in numpy with corners in lexicographic order, equals the oracle's volume (the
integral of det J over the reference cube) and its gradient on random
hexahedra, including strongly distorted ones, and is translation invariant."""
import numpy as np
import pytest

import oracle

CUBE = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=np.float64)


def grandy(P):
    """12 V and the gradient 12 dV/dP_c (8 x 3) of corners P (8 x 3)."""
    s1 = (P[2] - P[1]) + (P[6] - P[3])
    s2 = (P[4] - P[2]) + (P[5] - P[6])
    s3 = (P[1] - P[4]) + (P[3] - P[5])
    c = [P[7] - P[2], P[7] - P[4], P[7] - P[1]]
    d = [P[3] - P[0], P[6] - P[0], P[5] - P[0]]
    s = [s1, s2, s3]
    v12 = sum(np.dot(s[i], np.cross(c[i], d[i])) for i in range(3))
    A = [np.cross(c[i], d[i]) for i in range(3)]
    B = [np.cross(d[i], s[i]) for i in range(3)]
    C = [np.cross(s[i], c[i]) for i in range(3)]
    g = np.zeros((8, 3))
    # s1 = P2 - P1 + P6 - P3, s2 = P4 - P2 + P5 - P6, s3 = P1 - P4 + P3 - P5
    for (i, plus, minus) in ((0, (2, 6), (1, 3)), (1, (4, 5), (2, 6)), (2, (1, 3), (4, 5))):
        for k in plus:
            g[k] += A[i]
        for k in minus:
            g[k] -= A[i]
    for i, q in enumerate((2, 4, 1)):      # c_i = P7 - P_q
        g[7] += B[i]
        g[q] -= B[i]
    for i, q in enumerate((3, 6, 5)):      # d_i = P_q - P0
        g[q] += C[i]
        g[0] -= C[i]
    return v12, g


@pytest.mark.parametrize("distortion", [0.0, 0.1, 0.3])
def test_grandy_form_equals_the_trilinear_volume_and_gradient(distortion):
    rng = np.random.default_rng(int(distortion * 100) + 1)
    for _ in range(50):
        P = CUBE * rng.uniform(0.5, 2.0, 3) + rng.normal(scale=distortion, size=(8, 3)) + rng.normal(size=3)
        X, Y, Z = (np.ascontiguousarray(P[:, k]) for k in range(3))
        v = oracle.hex_volume(X, Y, Z)
        g_ref = np.array(oracle.hex_volume_grad(X, Y, Z)).T  # (8, 3)
        v12, g = grandy(P)
        scale = np.abs(g_ref).max()
        assert v12 / 12.0 == pytest.approx(v, rel=1e-13)
        assert np.abs(g / 12.0 - g_ref).max() <= 1e-13 * scale


def test_grandy_form_is_translation_invariant_and_sums_to_zero():
    rng = np.random.default_rng(5)
    P = CUBE + rng.normal(scale=0.2, size=(8, 3))
    v12, g = grandy(P)
    v12t, gt = grandy(P + np.array([3.0, -7.0, 11.0]))
    assert v12t == pytest.approx(v12, rel=1e-12)
    assert np.abs(gt - g).max() <= 1e-12 * np.abs(g).max()
    assert np.abs(g.sum(axis=0)).max() <= 1e-14 * np.abs(g).max()


def test_unit_cube():
    v12, g = grandy(CUBE.copy())
    assert v12 == 12.0
    # d V / d P_c of the unit cube: +-1/4 of the outward face normals at corner c
    for c in range(8):
        expect = np.array([(1 if (c >> a) & 1 else -1) * 0.25 for a in range(3)])
        assert np.allclose(g[c] / 12.0, expect)

"""Pins for the oracle of the two-phase IMPES scheme (Section 6): the fluid
model's end points and a hand-evaluated middle point, the well index's
symmetry, scaling and its square-cell reduction, upstream weighting on a
three-cell problem worked by hand (both flow directions), and the discrete
conservation of water by the saturation sub-steps."""
import numpy as np

from oracle import impes


def test_fluid_model_end_points_and_middle():
    fl = impes.Fluid()
    lam, fw = impes.mobilities(np.array([0.2, 0.8, 0.5, 0.0, 1.0]), fl)
    # S = s_wc: only oil moves (k_ro = 1); S = 1 - s_or: only water; S* = 1/2 by hand
    np.testing.assert_allclose(lam[:2], [1 / 3.0, 1 / 0.3], rtol=1e-15)
    np.testing.assert_allclose(fw[:2], [0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(lam[2], 0.25 / 0.3 + 0.25 / 3.0, rtol=1e-15)
    np.testing.assert_allclose(fw[2], (0.25 / 0.3) / (0.25 / 0.3 + 0.25 / 3.0), rtol=1e-15)
    np.testing.assert_allclose(lam[3:], lam[:2], rtol=0)         # S* clipped to [0, 1]


def test_well_index_symmetry_scaling_and_square_cells():
    wi = impes.well_index
    assert abs(wi(20.0, 10.0, 1.0) - wi(10.0, 20.0, 1.0)) < 1e-16
    np.testing.assert_allclose(wi(40.0, 20.0, 2.0), wi(20.0, 10.0, 1.0) / 4.0, rtol=1e-14)
    # hx = hy = h: h^2 WI = (pi/2) / ln(r_eq / r_w), r_eq = (sqrt(10)/2) exp(-pi/4) h (worked by hand
    # from the printed formula: r1 = r2 = sqrt(10) h / 2)
    h, rw = 12.0, 0.5
    req = np.sqrt(10.0) / 2.0 * np.exp(-np.pi / 4.0) * h
    np.testing.assert_allclose(h * h * wi(h, h, rw), (np.pi / 2.0) / np.log(req / rw), rtol=1e-13)


def test_upstream_weighting_by_hand():
    fl = impes.Fluid()
    S = np.array([0.8, 0.2, 0.2]).reshape(1, 1, 3)          # f_w = 1, 0, 0
    z = np.zeros((1, 1, 3))
    h = (1.0, 1.0, 1.0)
    v = np.zeros((3, 1, 1, 3))
    v[0, 0, 0, :2] = 1.0                                     # flow to +x through both interior faces
    r = impes.saturation_rate(S, v, z, z, 0.0, z, np.ones((1, 1, 3)), h, fl)
    # fluxes f_w(upstream) v: 1 (water leaves cell 0 into 1), 0 (cell 1 still dry)
    np.testing.assert_allclose(r.ravel(), [-1.0, 1.0, 0.0], atol=1e-15)
    v[0] = -v[0]                                             # flow to -x: upstream is the +x cell
    r = impes.saturation_rate(S, v, z, z, 0.0, z, np.ones((1, 1, 3)), h, fl)
    np.testing.assert_allclose(r.ravel(), [0.0, 0.0, 0.0], atol=1e-15)
    S2 = np.array([0.2, 0.2, 0.8]).reshape(1, 1, 3)
    r = impes.saturation_rate(S2, v, z, z, 0.0, z, np.ones((1, 1, 3)), h, fl)
    np.testing.assert_allclose(r.ravel(), [0.0, 1.0, -1.0], atol=1e-15)


def test_substeps_conserve_water_and_bound_the_change():
    rng = np.random.default_rng(3)
    shape = (4, 5, 6)
    h = (1 / 6, 1 / 5, 1 / 4)
    fl = impes.Fluid()
    S = rng.uniform(0.2, 0.8, size=shape)
    v = rng.normal(size=(3,) + shape)
    p = rng.normal(size=shape)
    W = np.zeros(shape)
    W[:, 0, 0] = 2.0
    q = np.zeros(shape)
    q[:, 2, 3] = 5.0
    phi = rng.uniform(0.05, 0.3, size=shape)
    r = impes.saturation_rate(S, v, p, W, 1.0, q, phi, h, fl)
    _, fw = impes.mobilities(S, fl)
    qw = q + fw * W * (1.0 - p)
    # sum of phi dS/dt = sum of the water sources: the face fluxes cancel (no-flow boundary)
    np.testing.assert_allclose((phi * r).sum(), qw.sum(), rtol=1e-12, atol=1e-12 * np.abs(qw).sum())
    S1, t = impes.transport(S, v, p, W, 1.0, q, phi, h, 1, 0.001, fl)
    assert abs(np.abs(S1 - S).max() - 0.001) < 1e-15 and t > 0

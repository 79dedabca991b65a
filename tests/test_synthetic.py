"""The seeded synthetic workloads match the recipe the measurements are quoted on: sizes, media,
frequency, order, radius ranges, packing fraction, boundary conditions, incidences, receivers,
the separation rule and the contour rule (the node count the bench line reports)."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import sommerfeld
from oracle.media import Layered


def _check_admissible(wl):
    """Burial and the separation rule |x_l - x_m| >= 1.1 (R_l + R_m) for every pair (k-d tree over
    the candidate pairs closer than 1.1 * 2 max R)."""
    from scipy.spatial import cKDTree
    c, r = wl.centres, wl.radius
    assert np.all(c[:, 1] + syn.SEP * r <= 0.0)
    pairs = cKDTree(c).query_pairs(syn.SEP * 2 * r.max(), output_type="ndarray")
    if len(pairs):
        d = np.linalg.norm(c[pairs[:, 0]] - c[pairs[:, 1]], axis=1)
        assert np.all(d >= syn.SEP * (r[pairs[:, 0]] + r[pairs[:, 1]]))


def _nodes(wl):
    L = Layered(wl.media, wl.omega)
    xi, _ = sommerfeld.contour(wl.n_panels, wl.nodes_per_panel, wl.t_max, wl.depth, wl.grade,
                               (L.kp_u, L.ks_u, L.kp_l, L.ks_l))
    return xi.size


def test_config1_recipe():
    wl = syn.config1()
    assert (wl.M, wl.p, wl.omega, wl.nrhs) == (16, 10, 2.0, 1)
    assert np.all(wl.radius == 0.5) and np.all(wl.bc == 0)
    assert np.all((wl.centres[:, 0] >= -10) & (wl.centres[:, 0] <= 10))
    assert np.all((wl.centres[:, 1] >= -8) & (wl.centres[:, 1] <= -1))
    assert wl.inc_kind[0] == 0 and wl.inc_angle[0] == pytest.approx(math.radians(30.0))
    assert wl.receivers.shape == (256, 2) and np.all(wl.receivers[:, 1] == -0.5)
    assert _nodes(wl) == 512 and wl.depth == 0.5          # the paper's depth, 32 x 16 nodes
    _check_admissible(wl)


def test_config3_recipe_is_the_benchmarked_workload():
    wl = syn.config3()
    assert (wl.M, wl.p, wl.omega, wl.nrhs) == (10000, 20, 6.0, 64)
    assert wl.name == "discs_stars10000_p20_rhs64"
    assert wl.radius.min() >= 0.2 and wl.radius.max() <= 0.5
    side = np.ptp(wl.centres[:, 0])
    packing = wl.M * np.mean(np.pi * wl.radius ** 2) / (143.0 * 143.0)
    assert 0.18 < packing < 0.21 and 140 < side < 144
    # half discs (even index), half stars (odd): 16 quantised sizes x 2 boundary conditions
    star = wl.proto >= 0
    assert np.array_equal(star, np.arange(wl.M) % 2 == 1) and wl.n_proto == 32
    assert np.array_equal(wl.bc, (np.arange(wl.M) // 2) % 2)
    levels = syn.star_levels(0.2, 0.5, 16)
    q = wl.proto[star]
    assert np.allclose(wl.radius[star], levels[q % 16]) and np.array_equal(wl.bc[star], q // 16)
    sh = wl.proto_shape[q]
    assert np.allclose(sh[:, 0] + sh[:, 1], wl.radius[star]) and np.allclose(sh[:, 1], 0.2 * sh[:, 0])
    assert np.all(np.bincount(q, minlength=32) > 100)
    assert np.sum(wl.inc_kind == 0) == 32 and np.sum(wl.inc_kind == 1) == 32
    assert np.all((wl.inc_angle >= math.radians(10)) & (wl.inc_angle <= math.radians(170)))
    npan, depth, grade = syn.contour_for_width(side)
    assert (wl.n_panels, wl.depth, wl.grade) == (npan, depth, grade)
    assert depth == pytest.approx(3.0 / side) and _nodes(wl) == 4800
    _check_admissible(wl)


def test_config4_recipe():
    wl = syn.config4()
    assert (wl.M, wl.p, wl.omega, wl.nrhs) == (2000, 16, 4.0, 32)
    assert np.all(wl.bc == 0) and np.all(wl.inc_kind == 0)
    assert wl.radius.min() >= 0.2 and wl.radius.max() <= 0.5
    assert wl.receivers.shape == (128, 2)
    _check_admissible(wl)


def test_workloads_are_reproducible():
    a, b = syn.config3(M=500), syn.config3(M=500)
    assert np.array_equal(a.centres, b.centres) and np.array_equal(a.inc_angle, b.inc_angle)
    x1, x2 = syn.random_coeffs(1000, 50, 20, 4), syn.random_coeffs(1000, 50, 20, 4)
    assert np.array_equal(x1, x2) and x1.shape == (50, 2, 41, 4) and x1.dtype == np.complex128


def test_config2_is_all_stars_with_quantised_sizes():
    wl = syn.config2()
    assert (wl.M, wl.p, wl.omega) == (1000, 16, 4.0)
    assert np.all(wl.proto >= 0) and wl.n_proto == 32
    a = wl.proto_shape[wl.proto, 0]
    assert a.min() >= 0.3 and a.max() <= 0.6 and np.allclose(wl.radius, 1.2 * a)
    assert np.array_equal(wl.bc, np.arange(wl.M) % 2) and np.array_equal(wl.proto_bc[wl.proto], wl.bc)
    _check_admissible(wl)


def test_surrogate_tables_follow_the_order_profile():
    ratio = np.array([[0.5, 1.5], [0.3, 0.9]])
    t = syn.surrogate_tables(7, ratio, 6)
    assert t.shape == (2, 26, 26)
    n = np.abs(np.arange(-6, 7))
    prof = 1.5 ** n / np.array([math.factorial(int(k)) for k in n])
    # shear-shear block of prototype 0 divided by its profile is O(1)
    blk = t[0, 13:, 13:] / np.outer(prof, prof)
    assert 0.01 < np.abs(blk).mean() < 10

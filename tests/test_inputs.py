"""Pins of the synthetic-input generators against values the paper prints."""
import math
import os

import numpy as np
import pytest

from paper_2209_02815_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_pole_dipole_counts_match_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "pole_dipole_counts.txt"), dtype=np.int64)
    for n_e, M in rows:
        prot = inputs.paper_pole_dipole(int(n_e))
        assert len(prot) == M == 6 * n_e - 56
        assert prot.min() >= 0 and prot.max() < n_e


def test_geometric_factor_gives_apparent_resistivity_of_half_space():
    """Footnote to Eq. 4.5: on a homogeneous half space with surface electrodes,
    g = k (u_A(x_M) - u_A(x_N)) = 1 / sigma0 for unit current."""
    sigma0 = 0.01
    el = inputs.line_electrodes(128, 32, 1 / 128)
    prot = inputs.pair_protocol(32)
    k = inputs.geometric_factor_pole_dipole(el[prot[:, 0]], el[prot[:, 1]], el[prot[:, 2]])
    u = lambda a, x: 1.0 / (2 * math.pi * sigma0 * np.linalg.norm(a - x, axis=-1))
    g = k * (u(el[prot[:, 0]], el[prot[:, 1]]) - u(el[prot[:, 0]], el[prot[:, 2]]))
    np.testing.assert_allclose(g, 1.0 / sigma0, rtol=1e-12)
    dd = inputs.dipole_dipole_grid(8, 8, 1024)
    assert len(dd) == 1024
    eg = inputs.grid_electrodes(192, 8, 8, 1 / 192)
    k2 = inputs.geometric_factor_dipole_dipole(*(eg[dd[:, c]] for c in range(4)))
    v = lambda a, b, x: u(a, x) - u(b, x)
    g2 = k2 * (v(eg[dd[:, 0]], eg[dd[:, 1]], eg[dd[:, 2]]) - v(eg[dd[:, 0]], eg[dd[:, 1]], eg[dd[:, 3]]))
    np.testing.assert_allclose(g2, 1.0 / sigma0, rtol=1e-10)


def test_pair_protocol_size():
    assert len(inputs.pair_protocol(32)) == 496


def test_random_field_statistics():
    f, clamped = inputs.gaussian_random_field((32, 32, 32), (1 / 32,) * 3, 0.1, math.log(0.01), 1.0)
    assert abs(f.mean() - math.log(0.01)) < 0.3
    assert 0.6 < f.std() < 1.3
    assert clamped < 0.05


def test_ert_problem_small():
    pr = inputs.ert_problem(16, n_e_line=8)
    assert pr.J.shape == (28, 16 ** 3)
    assert np.isfinite(pr.J).all()
    # J . 1 approximates -g (scaling sigma uniformly by e^t scales g by e^-t);
    # on the truncated unit cube the magnitude is below 1/sigma_bg.
    s = pr.J.sum(axis=1)
    assert (s < 0).mean() > 0.9


@pytest.mark.parametrize("n", [32, 128, 192])
def test_ert_surveys_have_finite_geometric_factors(n):
    """The line pair protocol gives C(32, 2) = 496 rows. The 8 x 8 dipole-dipole grid is
    truncated to 1024 rows. The 6 x 8 grid pair protocol of the inversion workload skips
    the rows whose M and N are equidistant from A (1/|AM| - 1/|AN| = 0) and keeps the first
    1000 of the others. Every factor is finite, every electrode cell lies in the top layer,
    and no row repeats an electrode."""
    for cells, abmn, k, _ in (inputs.ert_survey(n), inputs.ert_survey(n, grid=(8, 8), m_rows=1024),
                              inputs.gn_survey(n)):
        assert np.all(np.isfinite(k)) and np.all(k != 0)
        assert np.all((cells >= 0) & (cells < n * n))
        for row in abmn:
            used = [e for e in row if e >= 0]
            assert len(used) == len(set(used))
    assert len(inputs.ert_survey(n)[1]) == 496
    assert len(inputs.ert_survey(n, grid=(8, 8), m_rows=1024)[1]) == 1024
    assert len(inputs.gn_survey(n)[1]) == 1000


def test_gn_truth_anomalies():
    """Two Gaussian anomalies of peak factors 10 and 0.1 on a 0.01 S/m background."""
    ls = inputs.gn_truth(64)
    s = np.exp(ls)
    assert abs(s.max() / 0.01 - 10.0) < 0.5 and abs(s.min() / 0.01 - 0.1) < 0.02
    assert np.median(s) == pytest.approx(0.01, rel=1e-3)

"""The seeded input recipe (workloads.py): the shapes and value distributions
the benchmarks and the parity tests draw from, and their reproducibility.
Statistical checks use sample sizes at which the stated bounds hold with
overwhelming probability (several standard errors of margin)."""
import math

import numpy as np

from paper_2411_12690_gb300 import workloads as W


def test_block_geometries():
    # unit block of the precision configuration: 12x12x10 mesh, degree 2
    b = W.BLOCK_SMALL
    assert (b.lx, b.ly, b.lz, b.ex, b.ey, b.ez, b.r_cu, b.t_liner, b.order) == \
        (10.0, 10.0, 50.0, 12, 12, 10, 2.5, 0.5, 2)
    assert b.ex * b.ey * b.ez == 1440
    for b, pitch in ((W.BLOCK_P15, 15.0), (W.BLOCK_P20, 20.0)):
        assert (b.lx, b.ly, b.ex * b.ey * b.ez, b.order) == (pitch, pitch, 11520, 4)
    d = W.BLOCK_SMALL.dummy()
    assert d.r_cu == 0.0 and d.t_liner == 0.0 and d.ex == W.BLOCK_SMALL.ex


def test_materials_table():
    (e_si, nu_si, a_si), (e_cu, nu_cu, a_cu), (e_ox, nu_ox, a_ox) = W.MATERIALS
    assert (e_si, nu_si, a_si) == (130e3, 0.28, 2.8e-6)
    assert (e_cu, nu_cu, a_cu) == (110e3, 0.35, 17e-6)
    assert (e_ox, nu_ox, a_ox) == (71e3, 0.16, 0.5e-6)


def test_site_types_shape_values_and_seed():
    full = W.site_types(7, 5, 1.0)
    assert full.shape == (5, 7) and full.dtype == np.uint8 and not full.any()
    a = W.site_types(300, 200, 0.8, seed=3)
    b = W.site_types(300, 200, 0.8, seed=3)
    c = W.site_types(300, 200, 0.8, seed=4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert set(np.unique(a)) <= {0, 1}
    occ = float((a == 0).mean())                 # Bernoulli(0.8) over 60 000 sites
    assert abs(occ - 0.8) < 6 * math.sqrt(0.8 * 0.2 / a.size)


def test_batch_arrays_recipe():
    jobs = W.batch_arrays(2000, seed=11)
    assert jobs[0].site_type.shape == (jobs[0].ny, jobs[0].nx)
    sides = np.array([j.nx for j in jobs])
    assert all(j.nx == j.ny for j in jobs)
    assert sides.min() >= 4 and sides.max() <= 64
    # log-uniform on [4, 64]: the log of the side is uniform, mean at log(16)
    ls = np.log(sides)
    assert abs(ls.mean() - math.log(16.0)) < 0.05
    assert abs(np.mean(sides <= 16) - 0.5) < 0.05
    dts = np.array([j.dT for j in jobs])
    assert dts.min() >= -300.0 and dts.max() <= -150.0 and abs(dts.mean() + 225.0) < 3.0
    pitches = np.array([j.pitch for j in jobs])
    assert set(np.unique(pitches)) == {0, 1} and abs(pitches.mean() - 0.5) < 0.05
    occ = np.array([float((j.site_type == 0).mean()) for j in jobs if j.nx >= 32])
    assert occ.min() > 0.4 and occ.max() <= 1.0 and abs(occ.mean() - 0.75) < 0.03   # rho ~ U[0.5, 1]
    again = W.batch_arrays(5, seed=11)
    assert all(np.array_equal(x.site_type, y.site_type) and x.dT == y.dT for x, y in zip(again, jobs[:5]))


def test_request_stream_is_poisson():
    rate = 40.0
    reqs = W.request_stream(rate, 4000, seed=2)
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0) and t[0] > 0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * rate - 1.0) < 0.05               # exponential gaps, mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08         # coefficient of variation 1
    sides = np.array([r.job.nx for r in reqs])
    assert sides.min() >= 2 and sides.max() <= 128
    assert abs(np.log(sides).mean() - math.log(16.0)) < 0.06  # log-uniform on [2, 128]


def test_submodel_recipe():
    """Scenario 2 (section 5.1): a 15x15 TSV array in two rings of dummy
    blocks; the synthetic coarse field is prescribed on exactly the lattice
    points of the six outer faces, is a polynomial of degree <= 2 in the
    coordinates (so it is smooth across the sub-model) and is seeded."""
    st = W.submodel_sites(15, 2)
    assert st.shape == (19, 19) and int((st == 0).sum()) == 225
    assert np.all(st[:2] == 1) and np.all(st[-2:] == 1) and np.all(st[:, :2] == 1) and np.all(st[:, -2:] == 1)
    spec = W.BLOCK_SMALL
    dof, val = W.submodel_boundary(19, 19, spec, seed=5)
    X = Y = 19 * 2 + 1
    Z = 3
    node, comp = dof // 3, dof % 3
    gx, gy, gz = node % X, (node // X) % Y, node // (X * Y)
    assert np.all((gx == 0) | (gx == X - 1) | (gy == 0) | (gy == Y - 1) | (gz == 0) | (gz == Z - 1))
    n_face_points = X * Y * Z - (X - 2) * (Y - 2) * (Z - 2)
    assert dof.size == 3 * n_face_points and np.unique(dof).size == dof.size
    # degree <= 2: exact fit by the ten quadratic monomials, per component
    x, y, z = gx * 5.0, gy * 5.0, gz * 25.0
    Mq = np.stack([np.ones_like(x), x, y, z, x * x, y * y, z * z, x * y, y * z, z * x], 1).astype(float)
    for c in range(3):
        sel = comp == c
        coef, *_ = np.linalg.lstsq(Mq[sel], val[sel], rcond=None)
        assert np.abs(Mq[sel] @ coef - val[sel]).max() <= 1e-12 * np.abs(val).max()
    # magnitude of a thermal mismatch field: alpha_Si |dT| times the half-size
    assert 1e-3 < np.abs(val).max() < 1.0
    d2, v2 = W.submodel_boundary(19, 19, spec, seed=5)
    assert np.array_equal(dof, d2) and np.array_equal(val, v2)
    assert not np.array_equal(val, W.submodel_boundary(19, 19, spec, seed=6)[1])

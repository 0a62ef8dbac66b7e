"""Pins of the oracle's Darcy flow (two-way coupling: the fluid of Eq. 6 in
the slow-flow limit, with the drag reaction of Eq. 7).

* A column of layers of piecewise-constant permeability between a fixed
  pressure and the outlet: the flux is the pressure difference over the
  series resistance of the layers (the exact solution of d/dz(K dp/dz) = 0),
  and the pressure at every cell centre is the flux times the resistance
  below it.
* A box of uniform permeability between two fixed pressures: the pressure
  is linear and the velocity uniform, -K/mu times the gradient.
* The flow of a packed cylinder: every cell's net volume flux is zero, what
  enters from the wall leaves through the outlet, and the flow runs from
  the wall to the outlet.
* The drag reaction per cell equals the brute-force sum of the particles'
  drag forces (in the same integer quanta) over each cell.
The Kozeny-Carman permeability and the pressure-gradient force -V grad p on
a grain are readings (no value of the paper fixes them): parity unpinned
beyond their definitions (the CUDA path is checked against them).
"""
import numpy as np
import pytest

import oracle as O
from tests.helpers import default_dt, oracle_params, small_cylinder


def test_layered_column_matches_series_resistance():
    N, h, mu, dP = 12, (1e-3, 1e-3, 5e-4), 1e-3, 250.0
    K = np.array([3, 1, 4, 1, 5, 9, 2, 6, 5, 3, 5, 8], float) * 1e-11
    t = np.zeros(N, np.int8)
    t[-1] = 1  # the top cell holds the pressure
    o = np.zeros(N, np.uint8)
    o[0] = 1  # the bottom cell drains to the outlet, p = 0
    p0 = np.zeros(N)
    p0[-1] = dP
    p, it = O.darcy_solve((1, 1, N), h, mu, K, t, o, 0.0, p0)
    assert it >= 0
    A, hz = h[0] * h[1], h[2]
    # resistance from the outlet face (z = 0) up to each cell centre
    Rc = np.zeros(N)
    Rc[0] = mu / A * hz / (2 * K[0])
    for i in range(1, N):
        Rc[i] = Rc[i - 1] + mu / A * (hz / (2 * K[i - 1]) + hz / (2 * K[i]))
    Q = dP / Rc[-1]
    np.testing.assert_allclose(p[:-1], Q * Rc[:-1], rtol=1e-11)
    U = O.darcy_velocity((1, 1, N), h, mu, K, t, o, 0.0, p)
    np.testing.assert_allclose(U[:-1, 2] * A, -Q, rtol=1e-11)  # downwards, the same in every layer
    assert np.all(U[:, :2] == 0.0)


def test_uniform_box_gives_a_linear_pressure():
    nf, h, mu, K0 = (9, 4, 3), (2e-4, 3e-4, 5e-4), 1e-3, 2e-11
    nx, ny, nz = nf
    n = nx * ny * nz
    K = np.full(n, K0)
    i = np.arange(n) % nx
    t = np.where((i == 0) | (i == nx - 1), 1, 0).astype(np.int8)
    p0 = np.where(i == 0, 80.0, 0.0)
    p0[i == nx - 1] = 10.0
    p, it = O.darcy_solve(nf, h, mu, K, t, np.zeros(n, np.uint8), 0.0, p0)
    x = i * h[0]
    G = (10.0 - 80.0) / ((nx - 1) * h[0])
    np.testing.assert_allclose(p, 80.0 + G * x, rtol=1e-12, atol=1e-10)
    U = O.darcy_velocity(nf, h, mu, K, t, np.zeros(n, np.uint8), 0.0, p)
    inner = t == 0
    np.testing.assert_allclose(U[inner, 0], -K0 / mu * G, rtol=1e-11)
    assert np.abs(U[inner, 1:]).max() <= 1e-12 * abs(K0 / mu * G)


def darcy_cylinder(p_in=200.0):
    s = small_cylinder()
    dt = default_dt(s)
    p = oracle_params(s, dt)
    p.fluid_mode, p.p_inlet, p.perm_d = 1, p_in, float(np.mean((2 * s.R) ** 3)) ** (1 / 3)
    sim = O.Sim(p, s.x, s.v, s.w, s.R, s.Us)
    sim.bond_touching()
    sim.couple_fluid()
    sim.compute_forces()
    return s, p, sim


def test_cylinder_flow_runs_from_the_wall_to_the_outlet():
    """The injection pressure holds outside the wall; the cells over the
    outlet drain downwards, the cells along the wall flow inwards, and
    Darcy's law gives each cell a positive permeability (grad p against U)."""
    s, p, sim = darcy_cylinder()
    pres, U, gradp, it = sim.fluid()
    assert it > 0
    nx, ny, nz = s.grid.nf
    h = np.array(s.grid.h)
    c = np.arange(nx * ny * nz)
    ii, jj, ll = c % nx, (c // nx) % ny, c // (nx * ny)
    xc = s.grid.lo[0] + (ii + 0.5) * h[0]
    yc = s.grid.lo[1] + (jj + 0.5) * h[1]
    rc = np.hypot(xc, yc)
    unknown = rc < s.domain["Rc"]
    outlet = unknown & (ll == 0) & (rc < s.domain["r_out"])
    assert np.all(pres[~unknown] == p.p_inlet)
    assert np.all((pres[unknown] > 0) & (pres[unknown] < p.p_inlet))
    assert np.all(U[outlet, 2] < 0)
    wall_ring = unknown & (rc > s.domain["Rc"] - 1.5 * h[0])
    radial = (U[wall_ring, 0] * xc[wall_ring] + U[wall_ring, 1] * yc[wall_ring]) / rc[wall_ring]
    assert np.all(radial < 0)
    ok = unknown & (np.abs(U).sum(1) > 0)
    dot = (U[ok] * gradp[ok]).sum(1)
    assert np.all(dot < 0)


def test_cylinder_flow_balance_through_the_faces():
    """Recompute every face flux from the solved pressures and the
    Kozeny-Carman permeability of the oracle's porosity (written out here)
    and check the balance of each cell and of the whole sample."""
    s, p, sim = darcy_cylinder()
    pres, U, gradp, it = sim.fluid()
    nx, ny, nz = s.grid.nf
    h = np.array(s.grid.h)
    mu = s.fluid["mu_f"]
    S = sim.voidfrac().astype(np.float64)
    n = np.clip(1.0 - S * 2.0 ** -40, p.n_min, 1.0)
    n = np.minimum(n, p.n_cap)
    K = (p.perm_d ** 2 / 180.0) * n ** 3 / (1 - n) ** 2
    c = np.arange(nx * ny * nz)
    ii, jj, ll = c % nx, (c // nx) % ny, c // (nx * ny)
    xc = s.grid.lo[0] + (ii + 0.5) * h[0]
    yc = s.grid.lo[1] + (jj + 0.5) * h[1]
    rc = np.hypot(xc, yc)
    unknown = rc < s.domain["Rc"]
    outlet = unknown & (ll == 0) & (rc < s.domain["r_out"])
    net = np.zeros(len(c))
    inflow = 0.0
    strides = (1, nx, nx * ny)
    dims = (nx, ny, nz)
    idx = (ii, jj, ll)
    for k in range(3):
        A = h[(k + 1) % 3] * h[(k + 2) % 3]
        for sg in (-1, 1):
            q = idx[k] + sg
            ok = unknown & (q >= 0) & (q < dims[k])
            nb = c[ok] + sg * strides[k]
            T = A / (mu * h[k]) * 2 * K[c[ok]] * K[nb] / (K[c[ok]] + K[nb])
            Q = T * (pres[c[ok]] - pres[nb])  # out of the cell
            net[c[ok]] += Q
            inflow += -Q[~unknown[nb]].sum()
    To = h[0] * h[1] / (mu * 0.5 * h[2]) * K[outlet]
    out = To * pres[outlet]
    net[outlet] += out
    scale = np.abs(inflow)
    assert np.abs(net[unknown]).max() <= 1e-10 * scale
    assert out.sum() == pytest.approx(inflow, rel=1e-10)


def test_drag_reaction_is_the_brute_force_cell_sum():
    s, p, sim = darcy_cylinder()
    sim.step(3)
    data = sim.closure_data()  # drag force (columns 5-7) and cell (column 9) of the last evaluation
    expect = np.zeros((sim.ncell, 3), np.int64)
    active = sim.removed_step() < 0
    for row in data[active]:
        cell = int(row[9])
        for k in range(3):
            expect[cell, k] += int(np.rint(row[5 + k] * 2.0 ** 60))
    got = sim.reaction()
    assert np.array_equal(got, expect)
    assert np.abs(got).sum() > 0

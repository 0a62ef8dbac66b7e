"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Bars: contact pair lists and porosity cell sums bit-exact; per-step forces
normwise within 1e-10 (FP64) and 1e-4 (mixed) of the oracle, the norm being
the sum of the magnitudes of every force term on the particle.
"""
import numpy as np
import pytest

from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import (default_dt, default_skin, normwise_error, run_oracle, small_cylinder,
                           with_velocities)

pytestmark = pytest.mark.gpu

TOL = {cgdem.FP64: 1e-10, cgdem.MIXED: 1e-4}
PREC = [cgdem.FP64, cgdem.MIXED]


def gpu_context(samples, prec, dt=None, skin=None, max_neighbors=64, bond=True, **kw):
    params, counts = [], []
    for s in samples:
        params.append(cgdem.sample_params(s, dt if dt is not None else default_dt(s),
                                          skin if skin is not None else default_skin(s), **kw))
        counts.append(len(s.R))
    ctx = cgdem.Context(params, counts, precision=prec, max_neighbors=max_neighbors)
    ctx.set_fluid_velocity(np.concatenate([s.Us for s in samples]))
    x = np.concatenate([s.x for s in samples])
    v = np.concatenate([s.v for s in samples])
    w = np.concatenate([s.w for s in samples])
    R = np.concatenate([s.R for s in samples])
    ctx.init_particles(x, v, w, R, bond_touching=bond)
    return ctx


@pytest.fixture(scope="module")
def periodic():
    s = I.cached(I.small_periodic, 2000, 0)
    return with_velocities(s, 2e-3)


@pytest.fixture(scope="module")
def cylinder():
    return with_velocities(small_cylinder(), 1e-3)


def equilibrium_overlap(s):
    """delta_B = (81^(1/3) - 24^(1/3)) (pi^2 gamma^2 R* / E*^2)^(1/3) at the mean R* (Table 1 B)."""
    m = s.material
    Es = m["E"] / (2 * (1 - m["nu"] ** 2))
    Rs = 0.5 * float(np.mean(s.R))
    return (81 ** (1 / 3) - 24 ** (1 / 3)) * (np.pi ** 2 * m["gamma"] ** 2 * Rs / Es ** 2) ** (1 / 3)


def check_contacts(ctx, sim):
    gi, gj, gb = ctx.get_contacts()
    oi, oj, ob, _ = sim.contacts()
    assert len(gi) == len(oi), (len(gi), len(oi))
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    assert np.array_equal(gb, ob)
    return len(gi)


@pytest.mark.parametrize("prec", PREC)
def test_initial_forces_contacts_voidfrac(periodic, prec):
    s = periodic
    dt = default_dt(s)
    ctx = gpu_context([s], prec, dt=dt)
    ctx.compute_forces()
    sim = run_oracle(s, dt)
    n = check_contacts(ctx, sim)
    assert n > len(s.R)  # a connected bonded packing
    assert np.array_equal(ctx.get_voidfrac(s.grid.ncell), sim.voidfrac())
    g, o = ctx.get_state(), sim.state()
    scale = sim.force_scale()
    assert normwise_error(g["F"], o["F"], scale) <= TOL[prec]
    tscale = scale * s.R  # torque terms are force x radius
    assert normwise_error(g["T"], o["T"], tscale) <= TOL[prec]


@pytest.mark.parametrize("prec", PREC)
def test_steps_periodic(periodic, prec):
    s = periodic
    dt = default_dt(s)
    ctx = gpu_context([s], prec, dt=dt)
    ctx.compute_forces()
    sim = run_oracle(s, dt)
    for chunk in [1, 9, 40]:
        ctx.step(chunk)
        sim.step(chunk)
        check_contacts(ctx, sim)
        assert np.array_equal(ctx.get_voidfrac(s.grid.ncell), sim.voidfrac())
        g, o = ctx.get_state(), sim.state()
        scale = sim.force_scale()
        tol = 1e-8 if prec == cgdem.FP64 else 1e-3
        assert normwise_error(g["F"], o["F"], scale) <= tol
        L = s.domain["L"][0]
        dx = g["x"] - o["x"]
        dx -= L * np.round(dx / L)
        # FP64: rounding-order differences only.  Mixed: within 1e-4 of the
        # contact length scale, the JKR equilibrium overlap delta_B (Table 1).
        if prec == cgdem.FP64:
            assert np.abs(dx).max() <= 1e-12 * L
        else:
            assert np.abs(dx).max() <= 1e-4 * equilibrium_overlap(s)


@pytest.mark.parametrize("prec", PREC)
def test_cylinder_walls_outlet_drag(cylinder, prec):
    s = cylinder
    dt = default_dt(s)
    ctx = gpu_context([s], prec, dt=dt)
    ctx.compute_forces()
    sim = run_oracle(s, dt)
    check_contacts(ctx, sim)
    assert np.array_equal(ctx.get_voidfrac(s.grid.ncell), sim.voidfrac())
    g, o = ctx.get_state(), sim.state()
    assert normwise_error(g["F"], o["F"], sim.force_scale()) <= TOL[prec]
    ctx.step(20)
    sim.step(20)
    check_contacts(ctx, sim)
    g, o = ctx.get_state(), sim.state()
    tol = 1e-8 if prec == cgdem.FP64 else 1e-3
    assert normwise_error(g["F"], o["F"], sim.force_scale()) <= tol


def test_fp64_fused_step_equals_verbs(periodic):
    """step(n) and the verbs (integrate 0, couple, forces, integrate 1) give
    the same FP64 state, up to FMA-contraction rounding, when no rebuild
    happens in between."""
    s = periodic
    dt = default_dt(s)
    a = gpu_context([s], cgdem.FP64, dt=dt)
    b = gpu_context([s], cgdem.FP64, dt=dt)
    a.compute_forces()
    b.compute_forces()
    a.step(3)
    for _ in range(3):
        b.integrate(0)
        b.couple_fluid()
        b.compute_forces()
        b.integrate(1)
    assert a.counters()["rebuilds"] == b.counters()["rebuilds"] == 1
    ga, gb = a.get_state(), b.get_state()
    for k in ["x", "v", "w", "F", "T"]:
        scale = np.abs(ga[k]).max()
        np.testing.assert_allclose(ga[k], gb[k], rtol=0, atol=1e-12 * scale)


def test_capacity_error_is_reported(periodic):
    s = periodic
    with pytest.raises(cgdem.CgdemError) as e:
        gpu_context([s], cgdem.MIXED, max_neighbors=2)
    assert e.value.code == cgdem.CGDEM_E_CAPACITY

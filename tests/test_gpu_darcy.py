"""Two-way coupling by Darcy flow against the oracle (both in FP64 for the
flow; the forces in both precisions).

The small sand-production cylinder with fluid_mode 1 (injection pressure
outside the wall, zero at the outlet, Kozeny-Carman permeability of the
porosity): the pressure, superficial velocity and pressure gradient of the
library's solve equal the oracle's to the solvers' tolerance; the forces
(drag of the solved flow, -V grad p) are within the per-step tolerance plus
what the two fields' difference moves the drag (its slope times the
velocity difference of the grain's cell); the drag reaction sums of Eq. 7
agree to the same accuracy; contacts stay bit-exact in FP64 over 20 steps
with the flow re-solved every 5 steps.
"""
import copy

import numpy as np
import pytest

import oracle as O
from paper_2211_06142_gb300 import cgdem
from tests.helpers import (check_mixed_forces, default_dt, default_skin, oracle_params, small_cylinder,
                           with_velocities)

pytestmark = pytest.mark.gpu

P_IN = 150.0
TOL = {cgdem.FP64: 1e-10, cgdem.MIXED: 1e-4}


def gpu_context(s, prec, couple_every, fluid_kernels=0):
    dt = default_dt(s)
    perm_d = float(np.mean((2 * s.R) ** 3)) ** (1 / 3)
    p = cgdem.sample_params(s, dt, default_skin(s), couple_every=couple_every, fluid_mode=1, p_inlet=P_IN,
                            perm_d=perm_d)
    ctx = cgdem.Context([p], [len(s.R)], precision=prec, max_neighbors=64, fluid_tol=1e-14,
                        fluid_iters=5000, fluid_kernels=fluid_kernels)
    ctx.set_fluid_velocity(s.Us)
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=True)
    ctx.compute_forces()
    return ctx


def setup(prec, couple_every=5):
    s = with_velocities(small_cylinder(), 1e-3)
    dt = default_dt(s)
    perm_d = float(np.mean((2 * s.R) ** 3)) ** (1 / 3)
    ctx = gpu_context(s, prec, couple_every)
    op = oracle_params(s, dt, couple_every=couple_every)
    op.fluid_mode, op.p_inlet, op.perm_d = 1, P_IN, perm_d
    sim = O.Sim(op, s.x, s.v, s.w, s.R, s.Us)
    sim.bond_touching()
    sim.couple_fluid()
    sim.compute_forces()
    return s, ctx, sim


def field_check(s, ctx, sim):
    gp, gU, gG, gR, it = ctx.get_fluid(s.grid.ncell)
    op, oU, oG, oit = sim.fluid()
    assert it >= 0 and oit >= 0  # converged (0: the last pressure already solved the new porosity)
    assert np.abs(gp - op).max() <= 1e-9 * np.abs(op).max()
    assert np.abs(gU - oU).max() <= 1e-8 * np.abs(oU).max()
    assert np.abs(gG - oG).max() <= 1e-8 * np.abs(oG).max()
    return gU, oU, gR


def force_bound(s, sim, gU, oU, tau):
    """tau times the force scale, plus the drag's slope times the velocity
    difference of the grain's cell (|f| ~ |w|^(1..2): slope <= 2 |f| / |w|)."""
    cl = sim.closure_data()
    cell = cl[:, 9].astype(int)
    fd = np.linalg.norm(cl[:, 5:8], axis=1)
    slip = cl[:, 1]
    n = 1.0 - cl[:, 0]
    dU = np.linalg.norm(gU[cell] - oU[cell], axis=1) / np.maximum(n, 1e-3)
    return tau * sim.force_scale() + np.where(slip > 0, 2 * fd / np.maximum(slip, 1e-300), 0.0) * dU


@pytest.mark.parametrize("prec", [cgdem.FP64, cgdem.MIXED])
def test_darcy_flow_and_forces_match_the_oracle(prec):
    s, ctx, sim = setup(prec)
    assert ctx.get_fluid(s.grid.ncell)[4] > 0  # the first solve starts from zero pressure
    gU, oU, gR = field_check(s, ctx, sim)
    g, o = ctx.get_state(), sim.state()
    b = force_bound(s, sim, gU, oU, TOL[prec])
    e = np.linalg.norm(g["F"] - o["F"], axis=1)
    assert np.all(e <= b), (e / b).max()
    # the pressure force is a real part of the force: the flow pushes inwards
    assert np.abs(sim.fluid()[2]).max() > 0
    # drag reaction (Eq. 7): cell sums agree to the drag's accuracy
    oR = sim.reaction()
    fsum = np.zeros((s.grid.ncell, 3))
    cl = sim.closure_data()
    np.add.at(fsum, cl[:, 9].astype(int), np.abs(cl[:, 5:8]))
    slack = (1e-9 if prec == cgdem.FP64 else 1e-4) * fsum * 2.0 ** 60 + 64
    assert np.all(np.abs(gR - oR) <= slack)
    assert np.abs(oR).sum() > 0
    ctx.close()


@pytest.mark.parametrize("prec", [cgdem.FP64, cgdem.MIXED])
def test_darcy_steps_resolve_the_flow(prec):
    """20 steps, the flow solved again at every fifth (after the porosity
    update): fields, forces and (FP64) contacts against the oracle."""
    s, ctx, sim = setup(prec, couple_every=5)
    for n in (5, 15):
        ctx.step(n)
        sim.step(n)
        gU, oU, _ = field_check(s, ctx, sim)
        g, o = ctx.get_state(), sim.state()
        if prec == cgdem.FP64:
            gi, gj, gb = ctx.get_contacts()
            oi, oj, ob, _ = sim.contacts()
            assert np.array_equal(gi, oi) and np.array_equal(gj, oj) and np.array_equal(gb, ob)
            b = force_bound(s, sim, gU, oU, TOL[prec])
            e = np.linalg.norm(g["F"] - o["F"], axis=1)
            assert np.all(e <= b + 1e-9 * sim.force_scale())  # 20 steps: the trajectories' spread
        else:
            assert check_mixed_forces(s, g, o, sim, ctx.get_contacts(), TOL[prec]) <= 0.02 * len(s.R)
    ctx.close()


def test_one_launch_solve_equals_the_kernel_per_phase_form():
    """The solve in one cooperative launch and the solve as one kernel per
    phase in a WHILE node: the same system, summed in different orders, so
    the fields agree to the tolerance's rounding, over a first solve from
    zero pressure and warm-started solves after 10 steps."""
    s = with_velocities(small_cylinder(), 1e-3)
    a = gpu_context(s, cgdem.FP64, 5, fluid_kernels=0)
    b = gpu_context(s, cgdem.FP64, 5, fluid_kernels=1)
    for n in (0, 10):
        if n:
            a.step(n)
            b.step(n)
        pa, Ua, Ga, Ra, ia = a.get_fluid(s.grid.ncell)
        pb, Ub, Gb, Rb, ib = b.get_fluid(s.grid.ncell)
        assert ia >= 0 and ib >= 0 and abs(ia - ib) <= max(2, ib // 20)
        assert np.abs(pa - pb).max() <= 1e-11 * np.abs(pb).max()
        assert np.abs(Ua - Ub).max() <= 1e-10 * np.abs(Ub).max()
        fa, fb = a.get_state()["F"], b.get_state()["F"]
        assert np.abs(fa - fb).max() <= 1e-9 * np.abs(fb).max()
    a.close()
    b.close()

"""The preparation stages (Sec. 3.1) on the GPU against the oracle, both
precisions, through the C ABI.

* Original JKR (the generation stage, Fig. 1) on a moving periodic packing
  without initial bonds: contacts form when grains touch and separate at
  point S.  Contact lists with their contact flags bit-exact in FP64;
  forces within the per-step bar plus what the two runs' state difference
  moves them (tests/helpers.py), which near S grows with the curve's slope.
* Compression: the small cylinder, its outlet closed, under a
  stress-controlled top plate that starts on the bed's highest grain; the
  plate's height, velocity and stress follow the oracle's; then the
  touching pairs are bonded and the bed runs under the modified JKR.
* Perforation: the small cylinder, bonded (modified JKR), with a
  penetrometer driven by a force coming down from just above the bed; the
  tool's height and the force on it follow the oracle's.
"""
import copy

import numpy as np
import pytest

import oracle as O
from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import (check_mixed_forces, default_dt, default_skin, oracle_params, small_cylinder,
                           with_velocities)

pytestmark = pytest.mark.gpu

TAU = {cgdem.FP64: 1e-10, cgdem.MIXED: 1e-4}


def contexts(s, prec, jkr_mode, bond, skin=None, g=None):
    dt = default_dt(s)
    skin = default_skin(s) if skin is None else skin
    p = cgdem.sample_params(s, dt, skin, jkr_mode=jkr_mode)
    if g is not None:
        for i in range(3):
            p.g[i] = g[i]
    ctx = cgdem.Context([p], [len(s.R)], precision=prec, max_neighbors=64)
    ctx.set_fluid_velocity(s.Us)
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=bond)
    op = oracle_params(s, dt, g=g)
    op.jkr_mode = jkr_mode
    sim = O.Sim(op, s.x, s.v, s.w, s.R, s.Us)
    if bond:
        sim.bond_touching()
    sim.couple_fluid()
    return ctx, sim, skin


def compare(s, ctx, sim, prec, skin, **bound_kw):
    g, o = ctx.get_state(), sim.state()
    gc = ctx.get_contacts()
    oi, oj, ob, _ = sim.contacts()
    if prec == cgdem.FP64:
        assert np.array_equal(gc[0], oi) and np.array_equal(gc[1], oj) and np.array_equal(gc[2], ob)
    vf = (ctx.get_voidfrac(s.grid.ncell), sim.voidfrac())
    left = check_mixed_forces(s, g, o, sim, gc, TAU[prec], skin=skin, vf=vf, **bound_kw)
    assert left <= (0 if prec == cgdem.FP64 else 0.02 * len(s.R))
    return g, o


@pytest.mark.parametrize("prec", [cgdem.FP64, cgdem.MIXED])
def test_original_jkr_contacts_form_and_separate(prec):
    s = with_velocities(copy.copy(I.cached(I.small_periodic, 2000, 0)), 2e-2)
    # the original JKR keeps a pair until |delta_S|: twice the skin of the tests
    ctx, sim, skin = contexts(s, prec, 1, bond=False, skin=2 * default_skin(s))
    ctx.compute_forces()
    sim.compute_forces()
    compare(s, ctx, sim, prec, skin, orig=True)
    formed = broken = 0
    before = set(zip(*(a.tolist() for a in sim.contacts()[:2])))
    for n in (25, 25, 50):
        ctx.step(n)
        sim.step(n)
        compare(s, ctx, sim, prec, skin, orig=True)
        now = set(zip(*(a.tolist() for a in sim.contacts()[:2])))
        formed += len(now - before)
        broken += len(before - now)
        before = now
    assert formed > 0 and broken > 0  # both ends of Fig. 1's curve were exercised
    oi, oj, ob, _ = sim.contacts()
    assert np.all(ob == 1)  # under the original JKR every contact in force is a JKR contact
    ctx.close()


def bed_top(s):
    return float((s.x[:, 2] + s.R).max())


@pytest.mark.parametrize("prec", [cgdem.FP64, cgdem.MIXED])
def test_plate_compression_follows_the_oracle(prec):
    s = small_cylinder()
    ctx, sim, skin = contexts(s, prec, 1, bond=False, skin=2 * default_skin(s))
    H0 = bed_top(s)
    sigma = 2e4
    A = np.pi * s.domain["Rc"] ** 2
    kw = dict(jkr_mode=1, plate_mode=1, plate_H=H0, plate_stress=sigma, plate_gain=0.05 / sigma,
              plate_vmax=0.05, outlet_closed=1)
    ctx.set_stage(0, cgdem.stage(**kw))
    sim.set_stage(O.make_stage(**kw))
    ctx.compute_forces()
    sim.compute_forces()
    travel = 0.0
    for n in (50, 50, 100):
        ctx.step(n)
        sim.step(n)
        gb, ob = ctx.boundaries()[0], sim.boundaries()
        travel = H0 - ob["H"]
        tolH = (1e-9 if prec == cgdem.FP64 else 1e-3) * travel + 1e-15
        assert abs(gb["H"] - ob["H"]) <= tolH, (gb, ob)
        tolS = (1e-8 if prec == cgdem.FP64 else 1e-3) * sigma
        assert abs(gb["stress"] - ob["stress"]) <= tolS, (gb, ob)
        assert abs(gb["v_plate"] - ob["v_plate"]) <= 0.05 / sigma * tolS + 1e-15
        compare(s, ctx, sim, prec, skin, orig=True, H=ob["H"])
    assert travel > 0 and ob["stress"] > 0  # the plate came down and carries the bed
    assert ob["stress"] * A > 0
    # the compressed bed's touching pairs become the modified JKR's bonds,
    # the contacts in force keeping their springs; then steps under it
    ctx.bond_touching()
    sim.bond_touching()
    kw = dict(jkr_mode=0, outlet_closed=1)
    ctx.set_stage(0, cgdem.stage(**kw))
    sim.set_stage(O.make_stage(**kw))
    ctx.step(50)
    sim.step(50)
    compare(s, ctx, sim, prec, skin, H=ob["H"])
    assert (sim.contacts()[2] == 1).sum() > len(s.R)  # the bed is bonded
    ctx.close()


@pytest.mark.parametrize("prec", [cgdem.FP64, cgdem.MIXED])
def test_penetrometer_follows_the_oracle(prec):
    s = small_cylinder()
    ctx, sim, skin = contexts(s, prec, 0, bond=True)
    # a tool wider than the cavity over the outlet, starting with its
    # hemispherical end just above the first grain it will touch
    rp = 0.4 * s.domain["Rc"]
    r = np.hypot(s.x[:, 0], s.x[:, 1])
    under = r < rp + s.R
    top = float((s.x[under, 2] - rp + np.sqrt((rp + s.R[under]) ** 2 - r[under] ** 2)).max())
    kw = dict(jkr_mode=0, pen_mode=1, pen_radius=rp, pen_speed=0.5, pen_z_start=top + 1e-6,
              pen_z_stop=0.5 * top, pen_force=0.05)
    ctx.set_stage(0, cgdem.stage(**kw))
    sim.set_stage(O.make_stage(**kw))
    ctx.compute_forces()
    sim.compute_forces()
    Fmax = 0.0
    for n in (100, 100, 100):
        ctx.step(n)
        sim.step(n)
        gb, ob = ctx.boundaries()[0], sim.boundaries()
        assert gb["pen_dir"] == ob["pen_dir"] == -1
        travel = kw["pen_z_start"] - ob["pen_z"]
        assert abs(gb["pen_z"] - ob["pen_z"]) <= (1e-9 if prec == cgdem.FP64 else 2e-3) * travel + 1e-15
        Fmax = max(Fmax, ob["pen_force"])
        tolF = (1e-8 if prec == cgdem.FP64 else 2e-3) * max(abs(ob["pen_force"]), 1e-300) + 1e-12
        assert abs(gb["pen_force"] - ob["pen_force"]) <= tolF, (gb, ob)
        compare(s, ctx, sim, prec, skin, tool=(rp, ob["pen_z"]))
    assert Fmax > 0  # the tool met the bed
    ctx.close()


@pytest.mark.parametrize("prec", [cgdem.FP64, cgdem.MIXED])
def test_preparation_sequence(prec):
    """The whole sequence of Sec. 3.1 on a small whole bed (no cavity, 10,000
    grains, about eight grains deep):
    generation with the original JKR, compression to the target stress (the
    paper's overburden stress over Young's modulus, 5 kPa for these grains;
    a stress far above it, with the default driving force that follows from
    it, crushes grains between the tool and the bottom),
    bonds on the touching pairs, perforation by a force-driven penetrometer
    and its removal.  What each stage must leave: the stress reached with
    the plate at rest and the bed denser; every grain with bonds on average
    several; a perforation that broke bonds and, at its deepest, held the
    tool's path clear of grains (whether the hole stays open after the tool
    leaves depends on the cement's strength: reported, not asserted)."""
    from paper_2211_06142_gb300 import prep
    d = I.fine_diameters(10000, 21)
    s = I.cylinder_sample(d, 21, scale=0.35, nf=(14, 14, 7), U_in=0.0, name="prep", cavity=False)
    p = cgdem.sample_params(s, default_dt(s), default_skin(s), jkr_mode=1)
    ctx = cgdem.Context([p], [len(s.R)], precision=prec, max_neighbors=64)
    ctx.set_fluid_velocity(np.zeros_like(s.Us))
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=False)
    ctx.compute_forces()
    por0 = prep.porosity_under_plate(s.R, s.domain["Rc"], float((s.x[:, 2] + s.R).max()))
    sigma = prep.scaled_stress(s.material["E"])
    rec = prep.prepare(ctx, s, gen_steps=3000, stress=sigma, vmax=0.2, max_compress_steps=40000,
                       pen_radius=0.75e-3, pen_speed=0.5, chunk=200)
    print(rec)
    c, b, f = rec["compression"], rec["bonding"], rec["perforation"]
    assert c["converged"] and abs(c["stress"] - sigma) <= 0.02 * sigma
    assert c["porosity"] < por0 - 0.05
    assert b["per_grain_mean"] > 3
    assert f["removed"] and f["bonds_broken"] > 0.05 * b["bonds"]
    assert f["deepest_tip"] < 0.5 * c["H"]
    assert f["solid_fraction_in_path_at_depth"] < 0.02
    assert ctx.boundaries()[0]["pen_dir"] == 0
    ctx.close()

"""The library in the launch configurations the benchmark times, and at its
full sizes, against the FP64 oracle.

* cgdem_step of any length runs from CUDA graphs (blocks of steps_per_graph,
  powers of two below it, an opening and a closing part) and gives the
  same state as single steps; the kernel launches it reports add up.
* The FP64 diagnostics (kinetic energies, momentum, produced mass, active
  spheres, bonds) equal sums over the library's own state and agree with
  the oracle's within what the states' difference allows.
* A periodic packing of 100,000 spheres: the FP64 force kernel's grid spans
  several waves, so warps wait on pair results published by warps of an
  earlier wave; contacts bit-exact and forces within 1e-10 over 3 steps.
* The 2.0M-sphere cylinder of the benchmark at the autotuner's knobs (the
  same call the benchmark makes): forces and contacts of spheres well inside
  two sub-blocks of 100,000 spheres (one mid-bed, one at the outlet and the
  bottom wall) against the oracle run on each sub-block, at the first force
  evaluation and after 3 steps, in both precisions (mixed after 3 steps:
  within the per-step tolerance plus the first-order change of the forces
  that the two runs' state difference produces, tests/helpers.py).
* The benchmark's 4.29M-sphere periodic cube at the knobs it is timed with:
  the spheres well inside the 100,000 nearest its centre, the same checks.
* The 64-member ensemble of the benchmark at its autotuned knobs, with and
  without the per-member skins balanced by drift rate: every member against
  the oracle at the first evaluation, six members after 12 steps.
"""
import copy

import numpy as np
import pytest

import oracle as O
from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import (check_mixed_forces, default_dt, default_skin, normwise_error, oracle_params,
                           with_velocities)

pytestmark = pytest.mark.gpu

TOL = {cgdem.FP64: 1e-10, cgdem.MIXED: 1e-4}
PREC = [cgdem.FP64, cgdem.MIXED]


def context(s, prec, dt, skin, block=128, cell_scale=0.0, ppw=32, max_neighbors=64, **kw):
    p = cgdem.sample_params(s, dt, skin, **kw)
    ctx = cgdem.Context([p], [len(s.R)], precision=prec, max_neighbors=max_neighbors,
                        block_size=block, cell_scale=cell_scale, particles_per_warp=ppw)
    ctx.set_fluid_velocity(s.Us)
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=True)
    return ctx


@pytest.fixture(scope="module")
def periodic():
    return with_velocities(copy.copy(I.cached(I.small_periodic, 2000, 0)), 2e-3)


# ---------------------------------------------------------------------------
# graphs for any step count
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PREC)
def test_short_step_calls_run_from_graphs(periodic, prec):
    """step(n) for n = 1, 2, 3, 5, 20, 33 and 70 (every remainder path) with
    blocks of 32 steps per graph equals the same calls with blocks of 3
    (remainders of 2 and 1), bit for bit: each call is an opening half kick,
    n - 1 fused steps and a closing step whatever the graphs are cut into.
    The kernels each call reports add up: the opening part (3 kernels), one
    condition kernel per block plus one force kernel per step, and the
    closing part (condition, force, bookkeeping)."""
    s = periodic
    dt = default_dt(s)
    p = cgdem.sample_params(s, dt, default_skin(s))
    ctxs = []
    for U in (32, 3):
        c = cgdem.Context([p], [len(s.R)], precision=prec, max_neighbors=64, steps_per_graph=U)
        c.set_fluid_velocity(s.Us)
        c.init_particles(s.x, s.v, s.w, s.R, bond_touching=True)
        c.compute_forces()
        ctxs.append(c)
    for n in (1, 2, 3, 5, 20, 33, 70):
        for c in ctxs:
            U = c.cfg.steps_per_graph
            k0, _ = c.launch_counts()
            c.step(n)
            k1, body = c.launch_counts()
            blocks = (n - 1) // U + bin((n - 1) % U).count("1")
            assert k1 - k0 == 3 + blocks + (n - 1) + 3, (U, n, k1 - k0)
            assert body > 0
    ga, gb = ctxs[0].get_state(), ctxs[1].get_state()
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(ga[k], gb[k]), k
    ca, cb = ctxs[0].counters(), ctxs[1].counters()
    assert ca["steps"] == cb["steps"] == 134
    assert ca["rebuilds"] == cb["rebuilds"] > 1


# ---------------------------------------------------------------------------
# FP64 diagnostics accumulators
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PREC)
def test_diagnostics_against_own_state_and_oracle(prec):
    """Cylinder with walls, outlet and drag, 40 steps with a grain sent out
    through the outlet: the accumulators of cgdem_get_diagnostics equal the
    sums over the library's own state (1e-12), and the oracle's within the
    bound the two states' velocity difference gives: |dKE| <= sum m |v| |dv|
    + m |dv|^2 / 2, |dP| <= sum m |dv|; produced mass and active spheres
    equal; bonds equal (FP64) or within 0.5 % (mixed: the lists may differ
    at a threshold)."""
    from tests.helpers import small_cylinder, run_oracle
    s = with_velocities(small_cylinder(), 1e-3)
    s.x[0] = (0.0, 0.0, -1.9 * s.R[0])
    s.v[0] = (0.0, 0.0, -2.0)
    dt = default_dt(s)
    ctx = context(s, prec, dt, default_skin(s))
    ctx.compute_forces()
    sim = run_oracle(s, dt)
    for n in (10, 30):
        ctx.step(n)
        sim.step(n)
        g, o = ctx.get_state(), sim.state()
        dg, do = ctx.get_diagnostics()[0], sim.diagnostics()
        act = ctx.get_removed_step() < 0
        ma = s.material["rho"] * 4.0 / 3.0 * np.pi * s.R[act] ** 3
        Ia = 0.4 * ma * s.R[act] ** 2
        ke = 0.5 * float((ma * (g["v"][act] ** 2).sum(1)).sum())
        kr = 0.5 * float((Ia * (g["w"][act] ** 2).sum(1)).sum())
        P = (ma[:, None] * g["v"][act]).sum(0)
        assert dg["ke"] == pytest.approx(ke, rel=1e-12)
        assert dg["ke_rot"] == pytest.approx(kr, rel=1e-12)
        pscale = float((ma * np.linalg.norm(g["v"][act], axis=1)).sum())
        for c, k in enumerate(("px", "py", "pz")):
            assert abs(dg[k] - P[c]) <= 1e-12 * pscale
        assert dg["n_active"] == act.sum() == do["n_active"]
        assert dg["produced_mass"] == pytest.approx(do["produced_mass"], rel=1e-12, abs=0)
        assert do["produced_mass"] > 0
        dv = np.linalg.norm(g["v"][act] - o["v"][act], axis=1)
        dw = np.linalg.norm(g["w"][act] - o["w"][act], axis=1)
        vo = np.linalg.norm(o["v"][act], axis=1)
        wo = np.linalg.norm(o["w"][act], axis=1)
        bke = float((ma * (vo * dv + 0.5 * dv * dv)).sum()) + 1e-14 * do["ke"]
        bkr = float((Ia * (wo * dw + 0.5 * dw * dw)).sum()) + 1e-14 * do["ke_rot"]
        assert abs(dg["ke"] - do["ke"]) <= bke
        assert abs(dg["ke_rot"] - do["ke_rot"]) <= bkr
        bP = float((ma * dv).sum()) + 1e-14 * pscale
        for k in ("px", "py", "pz"):
            assert abs(dg[k] - do[k]) <= bP
        if prec == cgdem.FP64:
            assert dg["n_bonds"] == do["n_bonds"]
            assert abs(dg["ke"] - do["ke"]) <= 1e-8 * do["ke"]
        else:
            assert abs(dg["n_bonds"] - do["n_bonds"]) <= 0.005 * do["n_bonds"]
    ctx.close()


# ---------------------------------------------------------------------------
# the FP64 pair exchange across waves
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def periodic100k():
    return with_velocities(copy.copy(I.cached(I.tiled_periodic, 12_500, 2, 8)), 2e-3, seed=9)


@pytest.mark.parametrize("block", [128, 256])
def test_fp64_exchange_over_several_waves(periodic100k, block):
    s = periodic100k
    assert len(s.R) == 100_000
    dt = default_dt(s)
    skin = 0.02 * 2 * float(s.R.max())
    ctx = context(s, cgdem.FP64, dt, skin, block=block, cell_scale=0.5, max_neighbors=48)
    ctx.compute_forces()
    p = oracle_params(s, dt)
    sim = O.Sim(p, s.x, s.v, s.w, s.R, s.Us)
    sim.bond_touching()
    sim.couple_fluid()
    sim.compute_forces()
    for n in (0, 3):
        if n:
            ctx.step(n)
            sim.step(n)
        g, o = ctx.get_state(), sim.state()
        gi, gj, gb = ctx.get_contacts()
        oi, oj, ob, _ = sim.contacts()
        assert np.array_equal(gi, oi) and np.array_equal(gj, oj) and np.array_equal(gb, ob)
        scale = sim.force_scale()
        assert normwise_error(g["F"], o["F"], scale) <= 1e-10
        assert normwise_error(g["T"], o["T"], scale * s.R) <= 1e-10
    assert ctx.status() == 0
    ctx.close()


# ---------------------------------------------------------------------------
# the benchmark's 2.0M-sphere cylinder at the autotuned knobs
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big():
    import bench
    s = bench.make_workload(1)
    dt, skin = bench.step_params(s)
    from paper_2211_06142_gb300 import autotune as A
    tune = A.autotune([cgdem.sample_params(s, dt, skin)], [len(s.R)], (s.x, s.v, s.w, s.R), s.Us,
                      cgdem.MIXED)
    skin = tune["skin_frac"] * 2 * float(s.R.max())
    s = copy.copy(s)
    s.v = np.random.default_rng(3).normal(size=s.x.shape) * 1e-3
    return s, dt, skin, tune


def sub_block(s, centre, n):
    """The n spheres nearest centre, and the radius of that ball."""
    d2 = ((s.x - centre) ** 2).sum(1)
    idx = np.sort(np.argpartition(d2, n)[:n])
    return idx, float(np.sqrt(d2[idx].max()))


def sub_oracle(s, idx, dt, rel=0.0):
    v, w = s.v[idx], s.w[idx]
    if rel:
        rng = np.random.default_rng(99)
        v = v * (1 + rel * rng.standard_normal(v.shape))
    sim = O.Sim(oracle_params(s, dt), s.x[idx], v, w, s.R[idx], s.Us)
    sim.bond_touching()
    sim.couple_fluid()
    sim.compute_forces()
    return sim


@pytest.mark.parametrize("prec", PREC)
def test_full_size_cylinder_at_bench_knobs(big, prec):
    """Spheres count as inside a sub-block when every sphere their forces
    depend on after n steps lies in it: n + 1 hops of the larger of the
    candidate reach and a fluid cell's diagonal (a sphere's drag depends on
    every centre in its cell) from the ball's surface."""
    s, dt, skin, tune = big
    assert len(s.R) > 1_900_000
    ctx = context(s, prec, dt, skin, block=tune["block"], cell_scale=tune["cell_scale"],
                  ppw=tune["ppw"], max_neighbors=48)
    ctx.compute_forces()
    h = s.extra["h_bed"]
    Rc = s.domain["Rc"]
    centres = [np.array([0.5 * Rc, 0.0, 0.5 * h]), np.array([s.domain["r_out"] + 2.5e-3, 0.0, 0.0])]
    hop = max(2 * float(s.R.max()) + skin, float(np.linalg.norm(s.grid.h)))
    rel = 1e-15 if prec == cgdem.FP64 else 1e-7
    subs = []
    for c in centres:
        idx, rad = sub_block(s, c, 100_000)
        subs.append((idx, rad, sub_oracle(s, idx, dt), sub_oracle(s, idx, dt, rel), c))
    for steps in (0, 3):
        if steps:
            ctx.step(steps)
        g = ctx.get_state()
        gi, gj, gb = ctx.get_contacts()
        for idx, rad, sim, ref, c in subs:
            if steps:
                sim.step(steps)
                ref.step(steps)
            o, r = sim.state(), ref.state()
            inner = np.linalg.norm(s.x[idx] - c, axis=1) < rad - (steps + 1) * hop - 1e-4
            assert inner.sum() > 1000
            scale = sim.force_scale()[inner]
            loc = -np.ones(len(s.R), np.int64)
            loc[idx] = np.arange(len(idx))
            li, lj = loc[gi], loc[gj]
            both = (li >= 0) & (lj >= 0)
            if prec == cgdem.FP64 or steps == 0:
                spread = normwise_error(r["F"][inner], o["F"][inner], scale)
                e = normwise_error(g["F"][idx][inner], o["F"][inner], scale)
                assert e <= max(TOL[prec], 10 * spread), (steps, e, spread)
                tsc = scale * s.R[idx][inner]
                spread_t = normwise_error(r["T"][inner], o["T"][inner], tsc)
                et = normwise_error(g["T"][idx][inner], o["T"][inner], tsc)
                assert et <= max(TOL[prec], 10 * spread_t), (steps, et, spread_t)
            else:
                sub = copy.copy(s)
                sub.x, sub.v, sub.w, sub.R = s.x[idx], s.v[idx], s.w[idx], s.R[idx]
                gs = {q: g[q][idx] for q in ("x", "v", "w", "F", "T")}
                left = check_mixed_forces(sub, gs, o, sim, (li[both], lj[both], gb[both]), TOL[prec],
                                          rows=inner, skin=skin)
                assert left <= 0.02 * inner.sum()
            # contacts of the inner spheres, bit-exact (FP64; mixed at step 0)
            if prec == cgdem.FP64 or steps == 0:
                keep = both.copy()
                keep[keep] &= inner[li[keep]] & inner[lj[keep]]
                G = set(zip(li[keep].tolist(), lj[keep].tolist(), gb[keep].tolist()))
                oi, oj, ob, _ = sim.contacts()
                ko = inner[oi] & inner[oj]
                Oc = set(zip(oi[ko].tolist(), oj[ko].tolist(), ob[ko].tolist()))
                assert G == Oc
    assert ctx.status() == 0
    ctx.close()


@pytest.mark.parametrize("prec", PREC)
def test_scale_cube_at_bench_knobs(big, prec):
    """The benchmark's 4.29M-sphere periodic cube at the knobs it is timed
    with (the headline's autotuned ones): forces, torques and contacts of
    the spheres well inside the 100,000 nearest the cube's centre (far from
    the periodic wrap) against the oracle run on them, at the first force
    evaluation and after 3 steps, as in the cylinder test above."""
    import bench
    _, _, _, tune = big
    s = copy.copy(bench.make_scale_cube(1))
    assert len(s.R) > 4_000_000
    s.v = np.random.default_rng(4).normal(size=s.x.shape) * 1e-3
    dt, _ = bench.step_params(s)
    skin = tune["skin_frac"] * 2 * float(s.R.max())
    ctx = context(s, prec, dt, skin, block=tune["block"], cell_scale=tune["cell_scale"],
                  ppw=tune["ppw"], max_neighbors=48)
    ctx.compute_forces()
    c = 0.5 * np.asarray(s.domain["L"])
    idx, rad = sub_block(s, c, 100_000)
    assert rad < 0.4 * min(s.domain["L"])
    rel = 1e-15 if prec == cgdem.FP64 else 1e-7
    sim, ref = sub_oracle(s, idx, dt), sub_oracle(s, idx, dt, rel)
    hop = max(2 * float(s.R.max()) + skin, float(np.linalg.norm(s.grid.h)))
    loc = -np.ones(len(s.R), np.int64)
    loc[idx] = np.arange(len(idx))
    for steps in (0, 3):
        if steps:
            ctx.step(steps)
            sim.step(steps)
            ref.step(steps)
        g = ctx.get_state()
        gi, gj, gb = ctx.get_contacts()
        o, r = sim.state(), ref.state()
        inner = np.linalg.norm(s.x[idx] - c, axis=1) < rad - (steps + 1) * hop - 1e-4
        assert inner.sum() > 1000
        scale = sim.force_scale()[inner]
        li, lj = loc[gi], loc[gj]
        both = (li >= 0) & (lj >= 0)
        if prec == cgdem.FP64 or steps == 0:
            spread = normwise_error(r["F"][inner], o["F"][inner], scale)
            e = normwise_error(g["F"][idx][inner], o["F"][inner], scale)
            assert e <= max(TOL[prec], 10 * spread), (steps, e, spread)
            tsc = scale * s.R[idx][inner]
            spread_t = normwise_error(r["T"][inner], o["T"][inner], tsc)
            et = normwise_error(g["T"][idx][inner], o["T"][inner], tsc)
            assert et <= max(TOL[prec], 10 * spread_t), (steps, et, spread_t)
            keep = both.copy()
            keep[keep] &= inner[li[keep]] & inner[lj[keep]]
            G = set(zip(li[keep].tolist(), lj[keep].tolist(), gb[keep].tolist()))
            oi, oj, ob, _ = sim.contacts()
            ko = inner[oi] & inner[oj]
            assert G == set(zip(oi[ko].tolist(), oj[ko].tolist(), ob[ko].tolist()))
        else:
            sub = copy.copy(s)
            sub.x, sub.v, sub.w, sub.R = s.x[idx], s.v[idx], s.w[idx], s.R[idx]
            gs = {q: g[q][idx] for q in ("x", "v", "w", "F", "T")}
            left = check_mixed_forces(sub, gs, o, sim, (li[both], lj[both], gb[both]), TOL[prec],
                                      rows=inner, skin=skin)
            assert left <= 0.02 * inner.sum()
    assert ctx.status() == 0
    ctx.close()


# ---------------------------------------------------------------------------
# the benchmark's 64-member ensemble at its autotuned knobs
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def ensemble64():
    from paper_2211_06142_gb300 import autotune as A
    from paper_2211_06142_gb300 import workloads as Wl
    specs, samples = Wl.ensemble(64, 3)
    params = Wl.ensemble_params(specs, samples)
    counts = [len(s.R) for s in samples]
    state = tuple(np.concatenate([getattr(s, a) for s in samples]) for a in "xvwR")
    Us = np.concatenate([s.Us for s in samples])
    best = A.autotune(params, counts, state, Us, cgdem.MIXED)
    params = A.tuned_params(params, best)
    bal, fac = A.balance_skins(params, counts, state, Us, cgdem.MIXED, cell_scale=best["cell_scale"],
                               block=best["block"], ppw=best["ppw"])
    return specs, samples, params, bal, best, fac


@pytest.mark.parametrize("skins", ["tuned", "balanced"])
def test_ensemble_at_bench_knobs(ensemble64, skins):
    specs, samples, params, bal, best, fac = ensemble64
    pp = params if skins == "tuned" else bal
    if skins == "balanced":
        assert (fac > 1.0).any()
    counts = [len(s.R) for s in samples]
    ctx = cgdem.Context(pp, counts, precision=cgdem.MIXED, max_neighbors=48, block_size=best["block"],
                        cell_scale=best["cell_scale"], particles_per_warp=best["ppw"])
    ctx.set_fluid_velocity(np.concatenate([s.Us for s in samples]))
    ctx.init_particles(*(np.concatenate([getattr(s, a) for s in samples]) for a in "xvwR"),
                       bond_touching=True)
    ctx.compute_forces()
    offs = np.concatenate([[0], np.cumsum(counts)])
    coffs = np.concatenate([[0], np.cumsum([s.grid.ncell for s in samples])])
    order = np.argsort(counts)
    stepped = sorted({int(order[0]), int(order[-1]), 1, 2, 3, 4})  # smallest, largest, k mix, both kinds
    sims = {}
    g = ctx.get_state()
    vf = ctx.get_voidfrac(int(coffs[-1]))
    gi, gj, gb = ctx.get_contacts()
    for k, (sp, s, p) in enumerate(zip(specs, samples, pp)):
        o_p = oracle_params(s, p.dt, k=sp.k, scheme=1 if sp.k > 1 else 0)
        sim = O.Sim(o_p, s.x, s.v, s.w, s.R, s.Us)
        sim.bond_touching()
        sim.couple_fluid()
        sim.compute_forces()
        sl = slice(offs[k], offs[k + 1])
        assert normwise_error(g["F"][sl], sim.state()["F"], sim.force_scale()) <= TOL[cgdem.MIXED], k
        assert np.array_equal(vf[coffs[k]:coffs[k + 1]], sim.voidfrac()), k
        m = (gi >= offs[k]) & (gi < offs[k + 1])
        oi, oj, ob, _ = sim.contacts()
        assert np.array_equal(gi[m] - offs[k], oi) and np.array_equal(gj[m] - offs[k], oj), k
        assert np.array_equal(gb[m], ob), k
        if k in stepped:
            sims[k] = sim
    ctx.step(12)
    g = ctx.get_state()
    gi, gj, gb = ctx.get_contacts()
    for k, sim in sims.items():
        sim.step(12)
        sl = slice(offs[k], offs[k + 1])
        m = (gi >= offs[k]) & (gi < offs[k + 1])
        gk = {q: g[q][sl] for q in ("x", "v", "w", "F", "T")}
        left = check_mixed_forces(samples[k], gk, sim.state(), sim,
                                  (gi[m] - offs[k], gj[m] - offs[k], gb[m]), TOL[cgdem.MIXED], k=specs[k].k,
                                  skin=pp[k].skin)
        assert left <= 0.02 * counts[k], (k, left)
    assert ctx.status() == 0
    ctx.close()

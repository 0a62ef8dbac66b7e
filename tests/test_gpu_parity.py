"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Bars: contact pair lists and porosity cell sums bit-exact; per-step forces
normwise within 1e-10 (FP64) and 1e-4 (mixed) of the oracle, the norm being
the sum of the magnitudes of every force term on the particle.
"""
import re

import numpy as np
import pytest

from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import (check_mixed_forces, default_dt, default_skin, normwise_error, run_oracle,
                           small_cylinder, with_velocities)

pytestmark = pytest.mark.gpu

TOL = {cgdem.FP64: 1e-10, cgdem.MIXED: 1e-4}
PREC = [cgdem.FP64, cgdem.MIXED]


def gpu_context(samples, prec, dt=None, skin=None, max_neighbors=64, bond=True, ppw=32, **kw):
    params, counts = [], []
    for s in samples:
        params.append(cgdem.sample_params(s, dt if dt is not None else default_dt(s),
                                          skin if skin is not None else default_skin(s), **kw))
        counts.append(len(s.R))
    ctx = cgdem.Context(params, counts, precision=prec, max_neighbors=max_neighbors,
                        particles_per_warp=ppw)
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


def perturbed(s, rel, seed=99):
    """Copy of a sample with velocities perturbed by a relative amount rel."""
    import copy
    s2 = copy.copy(s)
    rng = np.random.default_rng(seed)
    s2.v = s.v * (1 + rel * rng.standard_normal(s.v.shape))
    s2.w = s.w * (1 + rel * rng.standard_normal(s.w.shape))
    return s2


def pair_deltas(s, x, pairs):
    """Overlap Ri + Rj - d of id pairs at positions x (minimum image)."""
    i, j = pairs[:, 0], pairs[:, 1]
    d = x[j] - x[i]
    if s.domain["kind"] == 0:
        L = s.domain["L"][0]
        d -= L * np.round(d / L)
    return s.R[i] + s.R[j] - np.sqrt((d * d).sum(1))


def check_contacts_near(ctx, sim, s, eps):
    """Contact lists of two slightly different trajectories: every pair in
    one list only must sit within eps (relative) of the touching or
    bond-break threshold in the oracle state."""
    gi, gj, gb = ctx.get_contacts()
    oi, oj, ob, _ = sim.contacts()
    G = {(a, b): c for a, b, c in zip(gi.tolist(), gj.tolist(), gb.tolist())}
    Oc = {(a, b): c for a, b, c in zip(oi.tolist(), oj.tolist(), ob.tolist())}
    diff = [k for k in set(G) ^ set(Oc)] + [k for k in set(G) & set(Oc) if G[k] != Oc[k]]
    if diff:
        x = sim.state()["x"]
        dl = pair_deltas(s, x, np.array(diff))
        S = s.R[np.array(diff)[:, 0]] + s.R[np.array(diff)[:, 1]]
        m = s.material
        Es = m["E"] / (2 * (1 - m["nu"] ** 2))
        Rs = s.R[np.array(diff)[:, 0]] * s.R[np.array(diff)[:, 1]] / S
        dC = -0.5723571212766659 * (np.pi ** 2 * m["gamma"] ** 2 * Rs / Es ** 2) ** (1 / 3)
        near = np.minimum(np.abs(dl), np.abs(dl - dC)) <= eps * S
        assert near.all(), (diff, dl)
    return len(diff)


def drift_bound(s, sim, n, dt, tau):
    """Position error after n steps that a force error of tau (normwise) per
    step produces at most: sum over steps of k dt^2 tau max(scale / m)."""
    m = s.material["rho"] * 4.0 / 3.0 * np.pi * s.R ** 3
    a = float(np.max(sim.force_scale() / m))
    return 0.5 * n * (n + 1) * dt * dt * tau * a


@pytest.mark.parametrize("prec", PREC)
def test_steps_periodic(periodic, prec):
    """Trajectories over 100 steps.  FP64: within ten times the oracle's own
    spread when its initial velocities are perturbed at rounding level (1e-15).
    Mixed: within the drift that the 1e-4 per-step force tolerance allows, or
    ten times the oracle's spread under a 1e-7 perturbation, whichever is larger."""
    s = periodic
    dt = default_dt(s)
    ctx = gpu_context([s], prec, dt=dt)
    ctx.compute_forces()
    sim = run_oracle(s, dt)
    rel = 1e-15 if prec == cgdem.FP64 else 1e-7
    ref = run_oracle(perturbed(s, rel), dt)
    L = s.domain["L"][0]
    done = 0
    for chunk in [1, 9, 40, 50]:
        ctx.step(chunk)
        sim.step(chunk)
        ref.step(chunk)
        done += chunk
        g, o, r = ctx.get_state(), sim.state(), ref.state()
        scale = sim.force_scale()
        spreadF = normwise_error(r["F"], o["F"], scale)
        dxr = r["x"] - o["x"]
        dxr -= L * np.round(dxr / L)
        spreadx = np.abs(dxr).max()
        if prec == cgdem.FP64:
            assert normwise_error(g["F"], o["F"], scale) <= max(TOL[prec], 10 * spreadF)
        else:
            assert check_mixed_forces(s, g, o, sim, ctx.get_contacts(), TOL[prec]) <= 0.02 * len(s.R)
        dx = g["x"] - o["x"]
        dx -= L * np.round(dx / L)
        bound = max(1e-13 * L, 10 * spreadx)
        if prec == cgdem.MIXED:
            bound = max(bound, drift_bound(s, sim, done, dt, TOL[prec]))
        assert np.abs(dx).max() <= bound
        if prec == cgdem.FP64:
            check_contacts(ctx, sim)
            assert np.array_equal(ctx.get_voidfrac(s.grid.ncell), sim.voidfrac())
        else:
            check_contacts_near(ctx, sim, s, eps=max(1e-9, 10 * spreadx / float(s.R.min())))
            gv, ov = ctx.get_voidfrac(s.grid.ncell), sim.voidfrac()
            assert int(gv.sum()) == int(ov.sum())
            # cells may differ only where a centre sits on a cell face
            assert (gv != ov).sum() <= 2 * 3 * np.count_nonzero(
                np.abs((o["x"] * s.grid.inv_h[0]) - np.round(o["x"] * s.grid.inv_h[0])) < 1e-6)


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
    rel = 1e-15 if prec == cgdem.FP64 else 1e-7
    ref = run_oracle(perturbed(s, rel), dt)
    ctx.step(20)
    sim.step(20)
    ref.step(20)
    g, o, r = ctx.get_state(), sim.state(), ref.state()
    scale = sim.force_scale()
    spreadx = np.abs(r["x"] - o["x"]).max()
    if prec == cgdem.FP64:
        check_contacts(ctx, sim)
    else:
        check_contacts_near(ctx, sim, s, eps=max(1e-9, 10 * spreadx / float(s.R.min())))
    if prec == cgdem.FP64:
        assert normwise_error(g["F"], o["F"], scale) <= max(TOL[prec], 10 * normwise_error(r["F"], o["F"], scale))
    else:
        assert check_mixed_forces(s, g, o, sim, ctx.get_contacts(), TOL[prec]) <= 0.02 * len(s.R)
    bound = max(1e-13, 10 * spreadx)
    if prec == cgdem.MIXED:
        bound = max(bound, drift_bound(s, sim, 20, dt, TOL[prec]))
    assert np.abs(g["x"] - o["x"]).max() <= bound
    # produced sand and removal steps agree (Eq. 40)
    np.testing.assert_array_equal(ctx.get_removed_step(), np.where(sim.removed_step() < 0, -1, sim.removed_step()))


@pytest.mark.parametrize("prec", PREC)
@pytest.mark.parametrize("domain", ["periodic", "cylinder"])
def test_sixteen_spheres_per_warp(periodic, cylinder, prec, domain):
    """The force kernel at 16 spheres per warp (record segments of 16
    spheres, lanes 16-31 evaluating entries only) against the oracle, with
    the checks of the 32-per-warp trajectory tests at the same step counts
    (1, 10, 50 and 100 steps): contacts bit-exact (FP64) or off only at
    thresholds (mixed), forces within the tolerance, same produced sand.
    The mixed trajectory's force error varies along the run (on the periodic
    packing it is 1.5e-4 at step 20 and 1.1e-5 at step 50 at both 16 and 32
    spheres per warp: position drift of ~3e-12 m near the touching and
    break thresholds), so the bound is checked where the 32-per-warp tests
    check it.  Both layouts also give the same forces up to the summation
    order of the contributions."""
    s = periodic if domain == "periodic" else cylinder
    dt = default_dt(s)
    ctx = gpu_context([s], prec, dt=dt, ppw=16)
    c32 = gpu_context([s], prec, dt=dt)
    ctx.compute_forces()
    c32.compute_forces()
    sim = run_oracle(s, dt)
    check_contacts(ctx, sim)
    assert np.array_equal(ctx.get_voidfrac(s.grid.ncell), sim.voidfrac())
    g, o = ctx.get_state(), sim.state()
    assert normwise_error(g["F"], o["F"], sim.force_scale()) <= TOL[prec]
    assert normwise_error(g["T"], o["T"], sim.force_scale() * s.R) <= TOL[prec]
    order = 1e-13 if prec == cgdem.FP64 else 1e-6  # summation order only
    assert normwise_error(g["F"], c32.get_state()["F"], sim.force_scale()) <= order
    rel = 1e-15 if prec == cgdem.FP64 else 1e-7
    ref = run_oracle(perturbed(s, rel), dt)
    done = 0
    for chunk in (1, 9, 40, 50):
        ctx.step(chunk)
        c32.step(chunk)
        sim.step(chunk)
        ref.step(chunk)
        done += chunk
        g, o, r = ctx.get_state(), sim.state(), ref.state()
        if done == 1:
            assert normwise_error(g["F"], c32.get_state()["F"], sim.force_scale()) <= order
        scale = sim.force_scale()
        dxr = r["x"] - o["x"]
        dx = g["x"] - o["x"]
        if domain == "periodic":
            L = s.domain["L"][0]
            dxr -= L * np.round(dxr / L)
            dx -= L * np.round(dx / L)
        spreadx = np.abs(dxr).max()
        if prec == cgdem.FP64:
            check_contacts(ctx, sim)
        else:
            check_contacts_near(ctx, sim, s, eps=max(1e-9, 10 * spreadx / float(s.R.min())))
        if prec == cgdem.FP64:
            assert normwise_error(g["F"], o["F"], scale) <= max(TOL[prec], 10 * normwise_error(r["F"], o["F"], scale))
        else:
            assert check_mixed_forces(s, g, o, sim, ctx.get_contacts(), TOL[prec]) <= 0.02 * len(s.R)
        bound = max(1e-13, 10 * spreadx)
        if prec == cgdem.MIXED:
            bound = max(bound, drift_bound(s, sim, done, dt, TOL[prec]))
        assert np.abs(dx).max() <= bound
    np.testing.assert_array_equal(ctx.get_removed_step(), np.where(sim.removed_step() < 0, -1, sim.removed_step()))


@pytest.mark.parametrize("prec", PREC)
def test_rebuild_every_step_carries_history(periodic, prec):
    """A candidate-list rebuild forced before each of 50 steps: the sphere
    order is re-sorted every step, so pair records (and, in FP64, the
    sphere that owns a pair and its inbox slots) change hands all the time;
    the tangential springs and bonds carried across must give the oracle's
    trajectory (contacts bit-exact in FP64, forces within the tolerance),
    checked after 10 and 50 steps as in the trajectory tests."""
    s = periodic
    dt = default_dt(s)
    ctx = gpu_context([s], prec, dt=dt)
    ctx.compute_forces()
    sim = run_oracle(s, dt)
    rel = 1e-15 if prec == cgdem.FP64 else 1e-7
    ref = run_oracle(perturbed(s, rel), dt)
    L = s.domain["L"][0]
    for chunk in (10, 40):
        for _ in range(chunk):
            ctx.build_contacts()
            ctx.step(1)
        sim.step(chunk)
        ref.step(chunk)
        g, o, r = ctx.get_state(), sim.state(), ref.state()
        scale = sim.force_scale()
        dxr = r["x"] - o["x"]
        dxr -= L * np.round(dxr / L)
        spreadx = np.abs(dxr).max()
        if prec == cgdem.FP64:
            check_contacts(ctx, sim)
        else:
            check_contacts_near(ctx, sim, s, eps=max(1e-9, 10 * spreadx / float(s.R.min())))
        tsc = scale * s.R
        if prec == cgdem.FP64:
            assert normwise_error(g["F"], o["F"], scale) <= max(TOL[prec], 10 * normwise_error(r["F"], o["F"], scale))
            assert normwise_error(g["T"], o["T"], tsc) <= max(TOL[prec], 10 * normwise_error(r["T"], o["T"], tsc))
        else:
            assert check_mixed_forces(s, g, o, sim, ctx.get_contacts(), TOL[prec]) <= 0.02 * len(s.R)
    assert ctx.counters()["rebuilds"] >= 51


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


@pytest.mark.parametrize("prec", PREC)
def test_cube_porosity_coarse_grains(prec):
    """Grains as large as a fluid cell (SSW k = 2 of the small cylinder) with
    the equal-volume cube spread of the porosity (vf_mode 1): cell sums
    bit-exact, contacts exact (FP64) and forces within the tolerance, before
    and after 10 steps, with couple_every = 2 so the rotating porosity
    buffers are exercised."""
    import oracle as O
    d = I.fine_diameters(6000, 23)
    dg, _ = O.cg_scale(d, 2, "ssw", 0.5)
    s = with_velocities(I.cylinder_sample(dg, 23, scale=0.3, nf=(12, 12, 6), U_in=0.05, name="cyl-k2"),
                        1e-3)
    dt = default_dt(s)
    kw = dict(k=2, scheme=1, vf_mode=1, couple_every=2)
    ctx = gpu_context([s], prec, dt=dt, **kw)
    ctx.compute_forces()
    sim = run_oracle(s, dt, **kw)
    assert np.array_equal(ctx.get_voidfrac(s.grid.ncell), sim.voidfrac())
    check_contacts(ctx, sim)
    g, o = ctx.get_state(), sim.state()
    assert normwise_error(g["F"], o["F"], sim.force_scale()) <= TOL[prec]
    rel = 1e-15 if prec == cgdem.FP64 else 1e-7
    ref = run_oracle(perturbed(s, rel), dt, **kw)
    ctx.step(10)
    sim.step(10)
    ref.step(10)
    g, o, r = ctx.get_state(), sim.state(), ref.state()
    scale = sim.force_scale()
    spread = normwise_error(r["F"], o["F"], scale)
    if prec == cgdem.FP64:
        assert normwise_error(g["F"], o["F"], scale) <= max(TOL[prec], 10 * spread)
    else:
        assert check_mixed_forces(s, g, o, sim, ctx.get_contacts(), TOL[prec], k=2) <= 0.02 * len(s.R)
    if prec == cgdem.FP64:
        check_contacts(ctx, sim)
        assert np.array_equal(ctx.get_voidfrac(s.grid.ncell), sim.voidfrac())


def test_init_rejects_a_bad_radius_or_state_by_the_lowest_index(periodic):
    """init_particles checks its inputs on the device before anything bins
    them: the lowest particle with a radius outside (0, r_max] or a
    non-finite state is named (the radius test first at equal index), the
    context stays uninitialised, and valid inputs then initialise it."""
    s = periodic
    ctx = cgdem.Context([cgdem.sample_params(s, default_dt(s), default_skin(s))], [len(s.R)],
                        precision=cgdem.MIXED, max_neighbors=64)
    ctx.set_fluid_velocity(s.Us)
    cases = []
    R = s.R.copy()
    R[700] = 2.0 * s.R.max()
    R[900] = -1.0
    cases.append(((s.x, s.v, s.w, R), cgdem.CGDEM_E_INVALID, 700))
    v = s.v.copy()
    v[500, 1] = np.nan
    cases.append(((s.x, v, s.w, R), cgdem.CGDEM_E_NONFINITE, 500))
    w = s.w.copy()
    w[300, 2] = np.inf
    R2 = s.R.copy()
    R2[300] = 0.0
    cases.append(((s.x, s.v, w, R2), cgdem.CGDEM_E_INVALID, 300))
    x = s.x.copy()
    x[len(s.R) - 1, 0] = -np.inf
    cases.append(((x, s.v, s.w, s.R), cgdem.CGDEM_E_NONFINITE, len(s.R) - 1))
    for args, code, idx in cases:
        with pytest.raises(cgdem.CgdemError) as e:
            ctx.init_particles(*args)
        assert e.value.code == code and re.search(rf"particle {idx}\b", str(e.value)), str(e.value)
        with pytest.raises(cgdem.CgdemError) as e:
            ctx.step(1)
        assert e.value.code == cgdem.CGDEM_E_STATE
    ctx.init_particles(s.x, s.v, s.w, s.R)
    ctx.step(3)
    assert np.isfinite(ctx.get_state()["x"]).all()
    ctx.close()


@pytest.mark.parametrize("prec", PREC)
def test_prepared_graphs_give_the_same_steps(periodic, prec):
    """A context that captured its step graphs at construction (prepare)
    steps bit-identically to one that captures them at its first step, and
    both read back into caller-provided arrays as into fresh ones."""
    s = periodic
    out = []
    for prep in (True, False):
        ctx = cgdem.Context([cgdem.sample_params(s, default_dt(s), default_skin(s))], [len(s.R)],
                            precision=prec, max_neighbors=64, prepare=prep)
        ctx.set_fluid_velocity(s.Us)
        ctx.init_particles(s.x, s.v, s.w, s.R)
        ctx.compute_forces()
        ctx.step(45)
        buf = {k: np.full((len(s.R), 3), np.nan) for k in ("x", "v", "w", "F", "T")}
        got = ctx.get_state(out=buf)
        assert all(got[k] is buf[k] for k in buf)
        fresh = ctx.get_state()
        for k in buf:
            assert np.array_equal(buf[k], fresh[k])
        out.append(fresh)
        ctx.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k

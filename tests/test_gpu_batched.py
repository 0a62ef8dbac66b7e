"""A batched ensemble in one library context, checked member by member
against the FP64 oracle run on each member alone.

The members differ in size, particle-size distribution, cohesion, domain
kind (periodic cube or cylinder with walls and outlet) and coarse-graining
ratio (k = 1 or SSW at k = 2, Sec. 2.4), as in a calibration sweep.  The
batch shares every array and launch; nothing of one member may leak into
another: contacts and porosity cells are compared exactly per member, forces
normwise within the per-step tolerance (or ten times the oracle's own spread
under a rounding-level perturbation, once trajectories have run).
"""
import copy

import numpy as np
import pytest

import oracle as O
from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import check_mixed_forces, default_dt, normwise_error, oracle_params, with_velocities

pytestmark = pytest.mark.gpu

TOL = {cgdem.FP64: 1e-10, cgdem.MIXED: 1e-4}
SSW = 1


def small_ensemble():
    """Four members (two periodic, two cylinders; k = 1 and 2), grains from
    the oracle's coarse-graining rule so that no input comes from the library."""
    specs = I.ensemble_specs(4, seed=5, n_lo=600, n_hi=1200, ks=(1, 2))
    grains = [O.cg_scale(sp.d_fine, sp.k, "ssw", sp.gamma)[0] for sp in specs]
    return specs, I.pack_ensemble(specs, grains, U=0.02, workers=1)


@pytest.fixture(scope="module")
def ensemble():
    specs, samples = I.cached(small_ensemble)
    samples = [with_velocities(copy.copy(s), 1e-3, seed=40 + i) for i, s in enumerate(samples)]
    assert {s.domain["kind"] for s in samples} == {0, 1}
    for sp, s in zip(specs, samples):  # packed: neighbours overlap by well under 5 % of a radius
        p = oracle_params(s, default_dt(s), k=sp.k, scheme=SSW if sp.k > 1 else 0)
        i, j = O.pairs_bruteforce(p, s.x, s.R, 0.0)
        d = s.x[j] - s.x[i]
        if s.domain["kind"] == 0:
            d -= s.domain["L"][0] * np.round(d / s.domain["L"][0])
        over = (s.R[i] + s.R[j] - np.linalg.norm(d, axis=1)) / np.minimum(s.R[i], s.R[j])
        assert over.max() < 0.05, (sp.index, over.max())
    return specs, samples


def skin(s):
    return 0.05 * 2 * float(s.R.max())


def batched_context(specs, samples, prec, ppw=32):
    params = [cgdem.sample_params(s, default_dt(s), skin(s), k=sp.k,
                                  scheme=SSW if sp.k > 1 else 0)
              for sp, s in zip(specs, samples)]
    ctx = cgdem.Context(params, [len(s.R) for s in samples], precision=prec, max_neighbors=64,
                        particles_per_warp=ppw)
    ctx.set_fluid_velocity(np.concatenate([s.Us for s in samples]))
    ctx.init_particles(*(np.concatenate([getattr(s, a) for s in samples]) for a in "xvwR"),
                       bond_touching=True)
    return ctx


def member_oracle(sp, s, rel=0.0, seed=99):
    s2 = copy.copy(s)
    if rel:
        rng = np.random.default_rng(seed)
        s2.v = s.v * (1 + rel * rng.standard_normal(s.v.shape))
        s2.w = s.w * (1 + rel * rng.standard_normal(s.w.shape))
    p = oracle_params(s2, default_dt(s2), k=sp.k, scheme=SSW if sp.k > 1 else 0)
    sim = O.Sim(p, s2.x, s2.v, s2.w, s2.R, s2.Us)
    sim.bond_touching()
    sim.couple_fluid()
    sim.compute_forces()
    return sim


def split_contacts(ctx, samples):
    gi, gj, gb = ctx.get_contacts()
    out, off = [], 0
    for s in samples:
        n = len(s.R)
        m = (gi >= off) & (gi < off + n)
        assert ((gj[m] >= off) & (gj[m] < off + n)).all()  # no pair across members
        out.append({(a - off, b - off): c for a, b, c in zip(gi[m].tolist(), gj[m].tolist(),
                                                              gb[m].tolist())})
        off += n
    assert sum(len(o) for o in out) == len(gi)
    return out


def oracle_contacts(sim):
    oi, oj, ob, _ = sim.contacts()
    return {(a, b): c for a, b, c in zip(oi.tolist(), oj.tolist(), ob.tolist())}


def near_threshold(s, x, pairs, eps, k):
    """Every pair lies within eps (relative) of touching or of bond break
    (grain surface energy k gamma, Eq. 24)."""
    pairs = np.array(pairs)
    i, j = pairs[:, 0], pairs[:, 1]
    d = x[j] - x[i]
    if s.domain["kind"] == 0:
        L = s.domain["L"][0]
        d -= L * np.round(d / L)
    S = s.R[i] + s.R[j]
    dl = S - np.sqrt((d * d).sum(1))
    m = s.material
    Es = m["E"] / (2 * (1 - m["nu"] ** 2))
    Rs = s.R[i] * s.R[j] / S
    gamma = m["gamma"] * k
    dC = -0.5723571212766659 * (np.pi ** 2 * gamma ** 2 * Rs / Es ** 2) ** (1 / 3)
    return (np.minimum(np.abs(dl), np.abs(dl - dC)) <= eps * S).all()


@pytest.mark.parametrize("prec,ppw", [(cgdem.FP64, 32), (cgdem.MIXED, 32), (cgdem.FP64, 16)])
def test_batched_members_match_oracle(ensemble, prec, ppw):
    """Members against their own oracle runs (at 16 spheres per warp, record
    segments also straddle members)."""
    specs, samples = ensemble
    ctx = batched_context(specs, samples, prec, ppw)
    ctx.compute_forces()
    sims = [member_oracle(sp, s) for sp, s in zip(specs, samples)]
    rel = 1e-15 if prec == cgdem.FP64 else 1e-7
    refs = [member_oracle(sp, s, rel) for sp, s in zip(specs, samples)]
    offs = np.concatenate([[0], np.cumsum([len(s.R) for s in samples])])
    coffs = np.concatenate([[0], np.cumsum([s.grid.ncell for s in samples])])
    for steps in (0, 12):
        if steps:
            ctx.step(steps)
            for a in sims + refs:
                a.step(steps)
        g = ctx.get_state()
        gc = split_contacts(ctx, samples)
        vf = ctx.get_voidfrac(int(coffs[-1]))
        diag = ctx.get_diagnostics()
        for k, (s, sim, ref) in enumerate(zip(samples, sims, refs)):
            sl = slice(offs[k], offs[k + 1])
            o, r = sim.state(), ref.state()
            scale = sim.force_scale()
            spread = normwise_error(r["F"], o["F"], scale)
            err = normwise_error(g["F"][sl], o["F"], scale)
            if prec == cgdem.FP64 or steps == 0:
                assert err <= max(TOL[prec], 10 * spread), (k, steps, err, spread)
            else:
                gk = {q: v for q, v in zip(["x", "v", "w", "F", "T"], [g[a][sl] for a in "xvwFT"])}
                ci = np.array([a for a, b in gc[k]], np.int64).reshape(-1)
                cj = np.array([b for a, b in gc[k]], np.int64).reshape(-1)
                cb = np.array([gc[k][q] for q in gc[k]], np.int64).reshape(-1)
                assert check_mixed_forces(s, gk, o, sim, (ci, cj, cb), TOL[prec], k=specs[k].k,
                                          skin=skin(s)) <= 0.02 * len(s.R)
            oc = oracle_contacts(sim)
            vk = vf[coffs[k]:coffs[k + 1]]
            if prec == cgdem.FP64 or steps == 0:
                assert gc[k] == oc, (k, steps)
                assert np.array_equal(vk, sim.voidfrac()), (k, steps)
            else:
                diff = [q for q in set(gc[k]) ^ set(oc)] + \
                       [q for q in set(gc[k]) & set(oc) if gc[k][q] != oc[q]]
                dx = r["x"] - o["x"]
                if s.domain["kind"] == 0:
                    dx -= s.domain["L"][0] * np.round(dx / s.domain["L"][0])
                eps = max(1e-9, 10 * np.abs(dx).max() / float(s.R.min()))
                assert not diff or near_threshold(s, o["x"], diff, eps, specs[k].k), (k, diff)
                assert int(vk.sum()) == int(sim.voidfrac().sum())
            od = sim.diagnostics()
            assert diag[k]["n_active"] == od["n_active"]
            assert diag[k]["produced_mass"] == pytest.approx(od["produced_mass"], rel=1e-12, abs=0)
    ctx.close()


def test_batched_member_removal_isolated(ensemble):
    """An outlet removal in one cylinder member changes no other member: the
    removal steps of each member equal those of the oracle on that member."""
    specs, samples = ensemble
    samples = [copy.deepcopy(s) for s in samples]
    for s in samples:
        if s.domain["kind"] == 1:  # one grain below the bed, over the outlet, moving out
            s.x[0] = (0.0, 0.0, -1.9 * s.R[0])
            s.v[0] = (0.0, 0.0, -2.0)
    ctx = batched_context(specs, samples, cgdem.FP64)
    ctx.compute_forces()
    sims = [member_oracle(sp, s) for sp, s in zip(specs, samples)]
    ctx.step(30)
    for sim in sims:
        sim.step(30)
    rs = ctx.get_removed_step()
    off = 0
    for s, sim in zip(samples, sims):
        n = len(s.R)
        ro = sim.removed_step().astype(np.int32)
        assert np.array_equal(rs[off:off + n], ro)
        assert (ro[0] >= 0) == (s.domain["kind"] == 1)
        off += n
    ctx.close()


def test_empty_and_single_sphere_members(ensemble):
    """Degenerate members beside a normal one: a member with no grains and a
    member with one grain (no contact; gravity, buoyancy and drag only).
    Every member matches the oracle run on it alone."""
    specs, samples = ensemble
    s = samples[2]
    one = copy.deepcopy(s)
    keep = np.array([0])
    one.x, one.v, one.w, one.R = s.x[keep], s.v[keep], s.w[keep], s.R[keep]
    none = copy.deepcopy(s)
    none.x, none.v, none.w, none.R = (np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)),
                                      np.zeros(0))
    members = [none, one, s]
    # the degenerate members take the time step, skin and largest radius of s
    params = [cgdem.sample_params(m, default_dt(s), skin(s), k=specs[2].k,
                                  scheme=SSW if specs[2].k > 1 else 0, r_max=float(s.R.max()))
              for m in members]
    ctx = cgdem.Context(params, [len(m.R) for m in members], precision=cgdem.FP64, max_neighbors=64)
    ctx.set_fluid_velocity(np.concatenate([m.Us for m in members]))
    ctx.init_particles(*(np.concatenate([getattr(m, a) for m in members]) for a in "xvwR"),
                       bond_touching=True)
    ctx.compute_forces()
    ctx.step(7)
    g = ctx.get_state()
    diag = ctx.get_diagnostics()
    assert diag[0]["n_active"] == 0 and diag[0]["ke"] == 0.0
    assert diag[1]["n_active"] == 1 and diag[1]["n_bonds"] == 0
    off = 0
    for m in members:
        n = len(m.R)
        if n:
            p = oracle_params(m, default_dt(s), k=specs[2].k, scheme=SSW if specs[2].k > 1 else 0)
            sim = O.Sim(p, m.x, m.v, m.w, m.R, m.Us)
            sim.bond_touching()
            sim.couple_fluid()
            sim.compute_forces()
            sim.step(7)
            o = sim.state()
            assert np.allclose(g["x"][off:off + n], o["x"], rtol=0, atol=1e-15 + 1e-12 * np.abs(o["x"]).max())
            assert normwise_error(g["F"][off:off + n], o["F"], sim.force_scale()) <= 1e-10
        off += n
    ctx.close()

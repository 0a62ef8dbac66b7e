"""Error of each precision against the FP64 oracle, quantity by quantity.

After the first force evaluation, one step and 100 steps on the 2,000-sphere
periodic packing and on the small cylinder (walls, outlet, drag), for the
FP64 and the mixed (FP32 contact physics, FP64 state) forms:

* F, per particle, normwise against two scales: the sum of the magnitudes
  of every force term (the one the parity bars use) and the sum of the
  magnitudes of the contact, wall and body force vectors;
* T, per particle, against the first scale times the radius;
* xi, the tangential spring of each active contact, against the largest
  spring of the sample;
* v and w against the largest speed (spin times radius) of the sample;
* x against the median grain diameter.

The bounds asserted are the per-step bars (1e-10 FP64, 1e-4 mixed) on F, T
and xi for the first evaluation and one step, and on v and x after one step
what those bars imply through the integrator (the 100-step trajectories are
bounded in tests/test_gpu_parity.py); with CGDEM_REPORT set, the measured
errors are written there as JSON.
"""
import copy
import json
import os

import numpy as np
import pytest

from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import default_dt, default_skin, run_oracle, small_cylinder, with_velocities

pytestmark = pytest.mark.gpu

REPORT = {}


def ctx_for(s, prec, dt):
    p = cgdem.sample_params(s, dt, default_skin(s))
    ctx = cgdem.Context([p], [len(s.R)], precision=prec, max_neighbors=64)
    ctx.set_fluid_velocity(s.Us)
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=True)
    ctx.compute_forces()
    return ctx


def errors(s, ctx, sim):
    g, o = ctx.get_state(), sim.state()
    out = {}
    for name, scale in (("F_termsum", sim.force_scale()), ("F_net", sim.force_scale_net())):
        e = np.linalg.norm(g["F"] - o["F"], axis=1) / np.maximum(scale, 1e-300)
        out[name] = {"max": float(e.max()), "median": float(np.median(e))}
    e = np.linalg.norm(g["T"] - o["T"], axis=1) / np.maximum(sim.force_scale() * s.R, 1e-300)
    out["T"] = {"max": float(e.max()), "median": float(np.median(e))}
    gi, gj, gx = ctx.get_contact_springs()
    oi, oj, ob, ox = sim.contacts()
    G = {(a, b): k for k, (a, b) in enumerate(zip(gi.tolist(), gj.tolist()))}
    both = [(G[(a, b)], k) for k, (a, b) in enumerate(zip(oi.tolist(), oj.tolist())) if (a, b) in G]
    xs = float(np.linalg.norm(ox, axis=1).max()) if len(ox) else 1.0
    if both and xs > 0:
        ig, io = (np.array(t) for t in zip(*both))
        e = np.linalg.norm(gx[ig] - ox[io], axis=1) / xs
        out["xi"] = {"max": float(e.max()), "median": float(np.median(e)), "pairs": len(both)}
    vs = float(np.linalg.norm(o["v"], axis=1).max())
    ws = float((np.linalg.norm(o["w"], axis=1) * s.R).max())
    ev = np.linalg.norm(g["v"] - o["v"], axis=1) / max(vs, 1e-300)
    ew = np.linalg.norm(g["w"] - o["w"], axis=1) * s.R / max(ws, 1e-300)
    dx = g["x"] - o["x"]
    if s.domain["kind"] == 0:
        L = s.domain["L"][0]
        dx -= L * np.round(dx / L)
    ex = np.linalg.norm(dx, axis=1) / float(np.median(2 * s.R))
    for k, e in (("v", ev), ("w", ew), ("x", ex)):
        out[k] = {"max": float(e.max()), "median": float(np.median(e))}
    out["v"]["abs_max"] = float(np.linalg.norm(g["v"] - o["v"], axis=1).max())
    out["x"]["abs_max"] = float(np.linalg.norm(dx, axis=1).max())
    return out


@pytest.fixture(scope="module", autouse=True)
def report():
    yield
    path = os.environ.get("CGDEM_REPORT")
    if path and REPORT:
        with open(path, "w") as f:
            json.dump(REPORT, f, indent=1)


@pytest.mark.parametrize("prec", [cgdem.FP64, cgdem.MIXED])
@pytest.mark.parametrize("kind", ["periodic", "cylinder"])
def test_error_per_quantity(kind, prec):
    s = (with_velocities(copy.copy(I.cached(I.small_periodic, 2000, 0)), 2e-3) if kind == "periodic"
         else with_velocities(small_cylinder(), 1e-3))
    dt = default_dt(s)
    ctx = ctx_for(s, prec, dt)
    sim = run_oracle(s, dt)
    m = s.material["rho"] * 4.0 / 3.0 * np.pi * s.R ** 3
    acc = float(np.max(sim.force_scale() / m))  # largest force-term scale over mass
    res = {"forces": errors(s, ctx, sim)}
    for n, label in ((1, "step1"), (99, "step100")):
        ctx.step(n)
        sim.step(n)
        res[label] = errors(s, ctx, sim)
    REPORT[f"{kind}-{'fp64' if prec == cgdem.FP64 else 'mixed'}"] = res
    tau = 1e-10 if prec == cgdem.FP64 else 1e-4
    for label in ("forces", "step1"):
        r = res[label]
        assert r["F_termsum"]["max"] <= tau and r["T"]["max"] <= tau, (label, r)
        assert r["xi"]["max"] <= tau, (label, r["xi"])
    # one step of the velocity Verlet moves v by dt F / m (two half kicks)
    # and x by dt v: a force error of tau times the scale gives at most
    # dt tau max(scale / m) in v and dt^2 tau max(scale / m) in x
    r = res["step1"]
    assert r["v"]["abs_max"] <= dt * tau * acc
    assert r["x"]["abs_max"] <= dt * dt * tau * acc
    ctx.close()


def test_fp64_newton_reciprocal_and_cube_root_match_cuda():
    """The FP64 contact law's reciprocal and cube root (Newton-Raphson from a
    single-precision seed) agree with CUDA's correctly rounded 1 / x and its
    cbrt to within 2 ulp, over the magnitudes the step meets and beyond
    (1e-40 to 1e40, where the seed falls back to the IEEE operations at the
    ends), both signs for the reciprocal."""
    rng = np.random.default_rng(5)
    x = 10.0 ** rng.uniform(-40, 40, 200_000) * rng.choice([-1.0, 1.0], 200_000)
    x = np.concatenate([x, [1.0, -1.0, 3.0, 1e-30, 1e30, 2.0 ** -60, 7.0 / 3.0]])
    r, r_ref, c, c_ref = cgdem.fp64_math_check(x)
    ulp_r = np.abs(r - r_ref) / np.spacing(np.abs(r_ref))
    ulp_c = np.abs(c - c_ref) / np.spacing(np.abs(c_ref))
    assert ulp_r.max() <= 2.0, (ulp_r.max(), x[ulp_r.argmax()])
    assert ulp_c.max() <= 2.0, (ulp_c.max(), x[ulp_c.argmax()])

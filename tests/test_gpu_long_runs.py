"""Long runs compared statistically (DEM is chaotic).

Eight seeded sand-production cylinders of 1,000 spheres (weak cohesion,
gamma = 0.02 J/m^2, strong radial inflow, so that the bonds at the outlet
break and sand is produced within a few thousand steps) run 9,000 steps:
on the GPU as one batched context in mixed precision, and each in the FP64
oracle.  Trajectories part after a few hundred steps, so the runs are
compared by their statistics: the produced mass (Eq. 40) at the end and the
time-mean kinetic energy over six read times, each by a two-sample
Kolmogorov-Smirnov test at the 5 % level and by the difference of the
means against three standard errors.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import default_dt, default_skin, oracle_params

pytestmark = pytest.mark.gpu

SEEDS = list(range(31, 39))
STEPS, READS = 9000, 6


def member(seed):
    d = I.fine_diameters(1000, seed)
    s = I.cylinder_sample(d, seed, scale=0.22, nf=(9, 9, 5), U_in=0.3, name=f"p12-{seed}")
    s.material = dict(s.material, gamma=0.02)
    return s


@pytest.fixture(scope="module")
def runs():
    samples = [member(sd) for sd in SEEDS]
    dts = [default_dt(s, 0.05) for s in samples]
    # GPU: all members in one batched context
    params = [cgdem.sample_params(s, dt, default_skin(s)) for s, dt in zip(samples, dts)]
    ctx = cgdem.Context(params, [len(s.R) for s in samples], precision=cgdem.MIXED, max_neighbors=64)
    ctx.set_fluid_velocity(np.concatenate([s.Us for s in samples]))
    ctx.init_particles(*(np.concatenate([getattr(s, a) for s in samples]) for a in "xvwR"),
                       bond_touching=True)
    ctx.compute_forces()
    g_ke = np.zeros((len(SEEDS), READS))
    for r in range(READS):
        ctx.step(STEPS // READS)
        g_ke[:, r] = [dg["ke"] for dg in ctx.get_diagnostics()]
    g_mass = np.array([dg["produced_mass"] for dg in ctx.get_diagnostics()])
    ctx.close()
    # oracle: each member on its own, on all host threads
    O.set_threads(os.cpu_count() or 1)
    o_ke = np.zeros((len(SEEDS), READS))
    o_mass = np.zeros(len(SEEDS))
    for k, (s, dt) in enumerate(zip(samples, dts)):
        sim = O.Sim(oracle_params(s, dt), s.x, s.v, s.w, s.R, s.Us)
        sim.bond_touching()
        sim.couple_fluid()
        sim.compute_forces()
        for r in range(READS):
            sim.step(STEPS // READS)
            o_ke[k, r] = sim.diagnostics()["ke"]
        o_mass[k] = sim.diagnostics()["produced_mass"]
    return g_mass, o_mass, g_ke.mean(1), o_ke.mean(1)


def same_distribution(a, b):
    from scipy.stats import ks_2samp
    p = ks_2samp(a, b).pvalue
    se = np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
    return p, abs(a.mean() - b.mean()), se


def test_produced_mass_statistics(runs):
    g_mass, o_mass, _, _ = runs
    assert (o_mass > 0).all() and (g_mass > 0).all()  # every member produced sand
    p, diff, se = same_distribution(g_mass, o_mass)
    assert p >= 0.05 and diff <= 3 * se, (g_mass, o_mass, p)


def test_kinetic_energy_statistics(runs):
    _, _, g_ke, o_ke = runs
    p, diff, se = same_distribution(g_ke, o_ke)
    assert p >= 0.05 and diff <= 3 * se, (g_ke, o_ke, p)

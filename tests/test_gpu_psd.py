"""Produced sand by size class (Sec. 3.4, Fig. 11) from the step's outlet.

A sand-producing cylinder (1,000 spheres, weak cohesion, strong inflow)
runs 6,000 steps with the eight Table 2 classes set: the library's class
counts and masses equal the sums over the grains it reports as removed
(cgdem_get_removed_step), class by class, to the last mass quantum; their
total equals the produced mass of the diagnostics; in FP64 the removals are
the oracle's, so the classes are too.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from paper_2211_06142_gb300 import sand as SD
from tests.helpers import default_dt, default_skin, oracle_params

pytestmark = pytest.mark.gpu


def sample():
    d = I.fine_diameters(1000, 31)
    s = I.cylinder_sample(d, 31, scale=0.22, nf=(9, 9, 5), U_in=0.3, name="psd")
    s.material = dict(s.material, gamma=0.02)
    return s


def expected(s, removed, edges):
    """Class counts and mass quanta of the removed grains, written out."""
    rho = s.material["rho"]
    rmax = float(s.R.max())
    mq = math.ldexp(rho * (4.0 / 3.0 * math.pi) * rmax * rmax * rmax, -40)
    nc = len(edges) - 1
    cnt = np.zeros(cgdem.PSD_MAX, np.int64)
    q = np.zeros(cgdem.PSD_MAX, np.int64)
    for i in np.flatnonzero(removed >= 0):
        R = float(s.R[i])
        c = int(np.clip(np.searchsorted(edges, 2 * R, side="right") - 1, 0, nc - 1))
        m = rho * (4.1887902047863905 * R * R * R)
        cnt[c] += 1
        q[c] += int(np.rint(m / mq))
    return cnt, q.astype(np.float64) * mq


@pytest.mark.parametrize("prec", [cgdem.FP64, cgdem.MIXED])
def test_psd_accumulators(prec):
    s = sample()
    dt = default_dt(s, 0.05)
    p = cgdem.sample_params(s, dt, default_skin(s))
    ctx = cgdem.Context([p], [len(s.R)], precision=prec, max_neighbors=64)
    ctx.set_fluid_velocity(s.Us)
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=True)
    edges = SD.table2_edges()
    ctx.set_psd_classes(edges)
    ctx.compute_forces()
    ctx.step(6000)
    mass, cnt = ctx.produced_psd()
    removed = ctx.get_removed_step()
    ec, em = expected(s, removed, edges)
    assert (removed >= 0).sum() > 20 and cnt[0].sum() == (removed >= 0).sum()
    assert np.array_equal(cnt[0], ec)
    assert np.array_equal(mass[0], em)
    assert mass[0].sum() == pytest.approx(ctx.get_diagnostics()[0]["produced_mass"], rel=1e-12)
    assert (cnt[0][len(edges) - 1:] == 0).all()
    if prec == cgdem.FP64:
        sim = O.Sim(oracle_params(s, dt), s.x, s.v, s.w, s.R, s.Us)
        sim.bond_touching()
        sim.couple_fluid()
        sim.compute_forces()
        sim.step(6000)
        ro = sim.removed_step()
        assert np.array_equal(np.where(ro < 0, -1, ro), removed)
    ctx.close()

"""Pins of the oracle's learned-closure hooks: corrections of one change
nothing, a uniform surface-energy correction c equals the plain model with
surface energy c gamma, the drag correction scales the drag term alone, and
the measured features equal the same quantities recomputed from the state
(contacts, overlaps, porosity cell sums, fluid velocity)."""
import copy
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import default_dt, oracle_params, with_velocities


@pytest.fixture(scope="module")
def sample():
    s = copy.deepcopy(I.cached(I.small_periodic, 400, 0))
    return with_velocities(s, 2e-3)


def sim_of(s, gamma_scale=1.0, closure=False, k_feat=2.0, steps=0):
    p = oracle_params(s, default_dt(s))
    p.gamma *= gamma_scale
    sim = O.Sim(p, s.x, s.v, s.w, s.R, s.Us)
    sim.bond_touching()
    sim.couple_fluid()
    if closure:
        sim.set_closure(True, k_feat)
    sim.compute_forces()
    if steps:
        sim.step(steps)
    return sim


def test_unit_corrections_change_nothing(sample):
    a = sim_of(sample, steps=5)
    b = sim_of(sample, closure=True, steps=5)
    sa, sb = a.state(), b.state()
    for k in ("x", "v", "F", "T"):
        assert np.array_equal(sa[k], sb[k])


@pytest.mark.parametrize("c", [4.0, 0.25])
def test_uniform_cohesion_correction_is_a_surface_energy(sample, c):
    ref = sim_of(sample, gamma_scale=c, steps=0)
    sim = sim_of(sample, closure=True)
    sim.set_corrections(np.ones(sim.n), np.full(sim.n, c))
    sim.compute_forces()  # re-evaluate with gamma sqrt(c c) = c gamma (c c and its root exact)
    ref.compute_forces()
    assert np.array_equal(sim.state()["F"], ref.state()["F"])
    assert np.array_equal(sim.state()["T"], ref.state()["T"])


def test_pair_cohesion_uses_geometric_mean(sample):
    """c_g = 4 on one sphere of each pair, 1 on the other: the pair sees
    gamma sqrt(4) = 2 gamma, which equals a plain run at 2 gamma when every
    contact joins a corrected and an uncorrected sphere; checked on the
    contacts of sphere 0 with its partners' corrections set so."""
    s = sample
    base = sim_of(s)
    i, j, b, _ = base.contacts()
    mine = (i == 0) | (j == 0)
    partners = np.where(i[mine] == 0, j[mine], i[mine])
    assert len(partners) >= 2
    # corrections: 4 on sphere 0, 1 everywhere else -> its pairs see 2 gamma
    cg = np.ones(base.n)
    cg[0] = 4.0
    sim = sim_of(s, closure=True)
    sim.set_corrections(np.ones(base.n), cg)
    sim.compute_forces()
    ref = sim_of(s, gamma_scale=2.0)
    ref.compute_forces()
    plain = sim_of(s)
    plain.compute_forces()
    # sphere 0's force: all of its contacts at 2 gamma
    Fs, Fr, Fp = sim.state()["F"][0], ref.state()["F"][0], plain.state()["F"][0]
    assert np.allclose(Fs, Fr, rtol=0, atol=1e-12 * np.abs(Fr).max())
    assert not np.allclose(Fs, Fp, rtol=0, atol=1e-6 * np.abs(Fp).max())


def test_drag_correction_scales_the_drag_alone(sample):
    a = sim_of(sample, closure=True)
    b = sim_of(sample, closure=True)
    b.set_corrections(np.full(b.n, 2.0), np.ones(b.n))
    b.compute_forces()
    a.compute_forces()
    da, db = a.closure_data(), b.closure_data()
    assert np.array_equal(db[:, 5:8], 2.0 * da[:, 5:8])
    dF = b.state()["F"] - a.state()["F"]
    assert np.allclose(dF, da[:, 5:8], rtol=1e-9, atol=1e-12 * np.abs(a.state()["F"]).max())


def test_features_match_the_state(sample):
    s = sample
    sim = sim_of(s, closure=True, k_feat=3.0, steps=3)
    sim.compute_forces()
    D = sim.closure_data()
    st = sim.state()
    x, v = st["x"], st["v"]
    n = len(s.R)
    i, j, b, _ = sim.contacts()
    # coordination and mean overlap from the active contacts
    Z = np.bincount(i, minlength=n) + np.bincount(j, minlength=n)
    assert np.array_equal(D[:, 3], Z.astype(float))
    d = x[j] - x[i]
    L = s.domain["L"][0]
    d -= L * np.round(d / L)
    delta = s.R[i] + s.R[j] - np.sqrt((d * d).sum(1))
    dsum = np.bincount(i, weights=delta, minlength=n) + np.bincount(j, weights=delta, minlength=n)
    want = np.where(Z > 0, dsum / np.maximum(Z, 1) / (2 * s.R), 0.0)
    assert np.allclose(D[:, 4], want, rtol=1e-9, atol=1e-15)
    # bond capacity: half of 3 pi gamma R* over bonded contacts
    Rs = s.R[i] * s.R[j] / (s.R[i] + s.R[j])
    capk = 0.5 * 3 * math.pi * s.material["gamma"] * Rs * (b > 0)
    cap = np.bincount(i, weights=capk, minlength=n) + np.bincount(j, weights=capk, minlength=n)
    assert np.allclose(D[:, 8], cap, rtol=1e-12, atol=0)
    # solid fraction and slip speed from the cell sums and the fluid field
    vf = sim.voidfrac()
    cell = D[:, 9].astype(int)
    g = s.grid
    c3 = np.clip(np.floor((x - np.array(g.lo)) * np.array(g.inv_h)), 0, np.array(g.nf) - 1).astype(int)
    assert np.array_equal(cell, (c3[:, 2] * g.nf[1] + c3[:, 1]) * g.nf[0] + c3[:, 0])
    nc = np.clip(1.0 - vf[cell].astype(float) * 2.0 ** -40, 0.2, 1.0)
    assert np.allclose(D[:, 0], 1.0 - nc, rtol=1e-15, atol=1e-16)
    slip = s.Us[cell] / nc[:, None] - v
    assert np.allclose(D[:, 1], np.linalg.norm(slip, axis=1), rtol=1e-14)
    assert np.all(D[:, 2] == 3.0)


def test_step_closure_applies_network_and_range_fallback(sample):
    s = sample
    theta = M.init_params(0)
    mu, isg, layers = M.unpack(theta)
    layers[3] = (np.zeros((2, 64)), np.array([math.log(2.0), math.log(0.5)]))
    theta = M.pack(mu, isg, layers)
    sim = sim_of(s, closure=True, k_feat=2.0)
    lo = np.array([0.0, 0.0, 1.0, 0.0, -1.0])
    hi = np.array([1.0, 10.0, 3.0, 4.0, 1.0])  # coordination above 4 -> fallback
    sim.step_closure(theta, 2, lo, hi, 3.0, math.log(4.0))
    D = sim.closure_data()  # the second evaluation used the first one's corrections
    cd, cg = D[:, 10], D[:, 11]
    assert set(np.unique(cd)) <= {1.0, 2.0} and set(np.unique(cg)) <= {1.0, 0.5}
    assert (cd == 2.0).sum() > 0 and (cd == 1.0).sum() > 0
    assert np.array_equal(cd == 2.0, cg == 0.5)

"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_printed.json), closed forms, limits,
invariants, an independent ODE integration or brute force in numpy.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
from paper_2211_06142_gb300 import inputs as I

E, NU = 1e8, 0.3
ES = E / (2 * (1 - NU * NU))


def base_params(**kw):
    d = dict(rho=2650.0, E=E, nu=NU, e=0.5, mu=0.5, gamma=0.5, rho_f=998.2, mu_f=1e-3,
             use_drag=0, use_buoyancy=0, kind=0, L=(1.0, 1.0, 1.0), dt=1e-7,
             nf=(1, 1, 1), f_lo=(0, 0, 0), hf=(1, 1, 1), inv_hf=(1, 1, 1), V_cell=1.0, n_min=0.2)
    d.update(kw)
    return O.make_params(**d)


# ---------------------------------------------------------------- Table 1 (P4)

@pytest.mark.parametrize("Rs,gamma", [(6e-5, 0.5), (1.2e-4, 2.0), (3e-5, 30.0)])
def test_table1_points(Rs, gamma, printed):
    """F, delta, a at points C, A, B of Table 1 from Eq. 12-13 and the bisection solver."""
    t1 = printed["table1"]
    xi = (math.pi ** 2 * gamma ** 2 * Rs / ES ** 2) ** (1 / 3)
    unit_a3 = math.pi * gamma * Rs ** 2 / ES
    for pt in "CAB":
        a = (t1[pt]["contact_radius_cubed_over_pi_gamma_Rs2_over_Es"] * unit_a3) ** (1 / 3)
        F = O.jkr_force(a, Rs, ES, gamma) / (math.pi * gamma * Rs)
        d = O.jkr_overlap(a, Rs, ES, gamma) / xi
        # printed to two decimals
        assert abs(F - t1[pt]["force_over_pi_gamma_Rs"]) <= 0.005 + 1e-12, (pt, F)
        assert abs(d - t1[pt]["overlap_over_xi"]) <= 0.005 + 1e-12, (pt, d)
    # exact forms: -3, -8/3, 0 and (81/16)^(1/3) - 12^(1/3), 0, 81^(1/3) - 24^(1/3)
    exact = {"C": (-3.0, (81 / 16) ** (1 / 3) - 12 ** (1 / 3)), "A": (-8 / 3, 0.0),
             "B": (0.0, 81 ** (1 / 3) - 24 ** (1 / 3))}
    for pt, (fx, dx) in exact.items():
        a = (t1[pt]["contact_radius_cubed_over_pi_gamma_Rs2_over_Es"] * unit_a3) ** (1 / 3)
        assert O.jkr_force(a, Rs, ES, gamma) / (math.pi * gamma * Rs) == pytest.approx(fx, abs=1e-12)
        assert O.jkr_overlap(a, Rs, ES, gamma) / xi == pytest.approx(dx, abs=1e-12)
        # inverting Eq. 13 at the point's overlap returns its contact radius
        assert O.jkr_contact_radius(dx * xi, Rs, ES, gamma) == pytest.approx(a, rel=1e-12)
    assert O.delta_c(Rs, ES, gamma) / xi == pytest.approx(exact["C"][1], rel=1e-13)
    # the jump at A is 8/9 of the pull-off force (Sec. 2.3)
    assert (8 / 3) / 3 == pytest.approx(printed["jkr_jump_fraction_of_FC"]["value"])


def test_bond_break_threshold():
    """The break test fires exactly below the Table 1 point-C overlap."""
    Rs, g = 6e-5, 0.5
    dC = O.delta_c(Rs, ES, g)
    assert O.bond_breaks(dC * (1 + 1e-9), Rs, ES, g)
    assert not O.bond_breaks(dC * (1 - 1e-9), Rs, ES, g)
    assert not O.bond_breaks(0.0, Rs, ES, g)
    assert not O.bond_breaks(1e-7, Rs, ES, g)
    # gamma = 0: delta_C = 0, any separation breaks
    assert O.bond_breaks(-1e-15, Rs, ES, 0.0)


# ---------------------------------------------------------------- Hertz limit (P3)

def test_hertz_limit():
    Rs, delta = 6e-5, 2e-7
    a = O.jkr_contact_radius(delta, Rs, ES, 0.0)
    assert a == pytest.approx(math.sqrt(Rs * delta), rel=1e-14)
    FH = 4.0 / 3.0 * ES * math.sqrt(Rs) * delta ** 1.5
    assert O.jkr_force(a, Rs, ES, 0.0) == pytest.approx(FH, rel=1e-14)
    # with cohesion, at fixed overlap, the sqrt(gamma) terms of Eq. 12 and Eq. 13
    # cancel to first order, so the force tends to Hertz linearly in gamma
    diffs = []
    for g in [1e-6, 4e-6, 16e-6]:
        ag = O.jkr_contact_radius(delta, Rs, ES, g)
        diffs.append(abs(O.jkr_force(ag, Rs, ES, g) - FH))
    assert diffs[1] / diffs[0] == pytest.approx(4.0, rel=2e-2)
    assert diffs[2] / diffs[1] == pytest.approx(4.0, rel=2e-2)


# ---------------------------------------------------------------- work of adhesion (P6)

@pytest.mark.parametrize("Rs,gamma", [(6e-5, 0.5), (1.15e-4, 30.0)])
def test_work_of_adhesion(Rs, gamma, printed):
    """Eq. 25-26: integral of F between points A and C."""
    dC = O.delta_c(Rs, ES, gamma)

    def F(delta):
        return O.jkr_force(O.jkr_contact_radius(delta, Rs, ES, gamma), Rs, ES, gamma)

    W, _ = quad(F, 0.0, dC, epsabs=0, epsrel=1e-12, limit=200)
    unit = (gamma ** 5 * Rs ** 4 / ES ** 2) ** (1 / 3)
    coeff = W / unit
    assert abs(coeff - printed["eq26_work_coefficient"]["value"]) < 0.005
    # exact coefficient of the closed form
    assert coeff == pytest.approx(11.120068109434463, rel=1e-6)


# ---------------------------------------------------------------- pull-off and modified JKR (P5)

def test_pull_off_and_break_then_hertz():
    """Kinematic separation of a bonded pair: the tensile force peaks at
    -3 pi gamma R* (Table 1 C), the bond breaks just beyond delta_C and
    does not reform; a new contact is Hertz with no jump to -8/9 F_C."""
    R, g = 1e-4, 0.5
    p = base_params(gamma=g, e=1.0, mu=0.0, kind=1)
    m = 2650.0 * 4 / 3 * math.pi * R ** 3
    Rs = R / 2
    FC = 3 * math.pi * g * Rs
    dC = O.delta_c(Rs, ES, g)
    xi_s = (math.pi ** 2 * g ** 2 * Rs / ES ** 2) ** (1 / 3)
    z = np.zeros(3)
    bonded, hist = True, np.zeros(3)
    Fmin, broke_at = 0.0, None
    deltas = np.linspace(1.44 * xi_s, 1.2 * dC, 4001)
    for d in deltas:
        xj = np.array([2 * R - d, 0, 0])
        act, Fi, Ti, Tj, Fne, a, delta, hist, bonded = O.pair_contact(
            p, z, z, z, R, m, xj, z, z, R, m, hist, bonded)
        if act:
            Fmin = min(Fmin, Fne)
        if not bonded and broke_at is None:
            broke_at = d
            assert not act and np.all(Fi == 0)
    assert Fmin == pytest.approx(-FC, rel=1e-6)
    assert broke_at is not None and broke_at < dC and broke_at > dC - 2 * (deltas[0] - deltas[1])
    # re-approach: unbonded, zero force until contact, then Hertz
    for d in [0.5 * dC, -1e-12, 1e-9, 5e-8]:
        xj = np.array([2 * R - d, 0, 0])
        act, Fi, Ti, Tj, Fne, a, delta, hist, bonded = O.pair_contact(
            p, z, z, z, R, m, xj, z, z, R, m, hist, bonded)
        assert not bonded
        if d <= 0:
            assert not act
        else:
            assert act and Fne == pytest.approx(4 / 3 * ES * math.sqrt(Rs) * d ** 1.5, rel=1e-9)


# ---------------------------------------------------------------- restitution (P7)

def _rk4_restitution(e, R, rho, v0):
    """Independent integration of the normal-impact ODE of two equal spheres:
    m* x'' = -(4/3) E* sqrt(R*) x^(3/2) - 2 sqrt(5/6) beta sqrt(2 E* sqrt(R* x) m*) x'."""
    m = rho * 4 / 3 * math.pi * R ** 3
    ms, Rs = m / 2, R / 2
    beta = -math.log(e) / math.sqrt(math.log(e) ** 2 + math.pi ** 2)

    def acc(x, v):
        if x <= 0:
            return 0.0
        a = math.sqrt(Rs * x)
        return (-(4 / 3) * ES * math.sqrt(Rs) * x ** 1.5
                - 2 * math.sqrt(5 / 6) * beta * math.sqrt(2 * ES * a * ms) * v) / ms

    x, v = 0.0, v0
    tc = 2.94 * (ms ** 2 / (ES ** 2 * Rs * v0)) ** 0.2  # Hertz contact time scale
    h = tc / 20000
    while True:
        k1x, k1v = v, acc(x, v)
        k2x, k2v = v + 0.5 * h * k1v, acc(x + 0.5 * h * k1x, v + 0.5 * h * k1v)
        k3x, k3v = v + 0.5 * h * k2v, acc(x + 0.5 * h * k2x, v + 0.5 * h * k2v)
        k4x, k4v = v + h * k3v, acc(x + h * k3x, v + h * k3v)
        x += h / 6 * (k1x + 2 * k2x + 2 * k3x + k4x)
        v += h / 6 * (k1v + 2 * k2v + 2 * k3v + k4v)
        if x < 0 and v < 0:
            return -v / v0


@pytest.mark.parametrize("e", [0.5, 0.8])
def test_restitution_head_on(e):
    R, rho = 1e-4, 2650.0
    out = []
    for v0 in [0.05, 0.2]:
        m = rho * 4 / 3 * math.pi * R ** 3
        ms = m / 2
        tc = 2.94 * (ms ** 2 / (ES ** 2 * (R / 2) * v0)) ** 0.2
        dt = tc / 4000
        p = base_params(gamma=0.0, e=e, mu=0.0, kind=1, Rc=1.0, H=1.0, r_out=0.0, g=(0, 0, 0),
                        dt=dt, nf=(1, 1, 1), f_lo=(-1, -1, -1), hf=(2, 2, 2), inv_hf=(0.5, 0.5, 0.5),
                        V_cell=8.0)
        x = np.array([[0.0, 0.0, 0.5], [2 * R + 1e-9, 0.0, 0.5]])
        v = np.array([[v0 / 2, 0, 0], [-v0 / 2, 0, 0]])
        s = O.Sim(p, x, v, np.zeros((2, 3)), np.array([R, R]))
        s.compute_forces()
        for _ in range(20000):
            s.step(1)
            st = s.state()
            if st["x"][1, 0] - st["x"][0, 0] > 2 * R and st["v"][1, 0] - st["v"][0, 0] > 0:
                break
        st = s.state()
        e_meas = (st["v"][1, 0] - st["v"][0, 0]) / v0
        e_ode = _rk4_restitution(e, R, rho, v0)
        assert e_meas == pytest.approx(e_ode, rel=2e-3), (e, v0)
        out.append(e_meas)
    # this damping form gives a restitution coefficient independent of impact speed
    assert out[0] == pytest.approx(out[1], rel=2e-3)
    # and close to the nominal e (beta of Eq. 33 derives from a linear spring)
    assert abs(out[0] - e) < 0.1


# ---------------------------------------------------------------- drag (P10)

def test_drag_limits():
    rho_f, mu_f, d = 998.2, 1e-3, 2e-4
    v = np.zeros(3)
    # Stokes-like limit Re -> 0: f -> 2.88 pi mu d w n^-3.7
    w = 1e-9
    for n in [1.0, 0.45]:
        f = O.drag(rho_f, mu_f, d, [w, 0, 0], v, n)
        assert f[0] == pytest.approx(2.88 * math.pi * mu_f * d * w * n ** -3.7, rel=1e-3)
        assert f[1] == 0 and f[2] == 0
    # at Re = 10^1.5 the porosity exponent is 3.7 - 0.65 = 3.05 (Eq. 10)
    w = 10 ** 1.5 * mu_f / (rho_f * d)
    f1 = O.drag(rho_f, mu_f, d, [0, w, 0], v, 0.8)[1]
    f2 = O.drag(rho_f, mu_f, d, [0, w, 0], v, 0.4)[1]
    assert math.log(f2 / f1) / math.log(2.0) == pytest.approx(3.05, rel=1e-12)
    # Newton regime Re -> inf: C_d -> 0.63^2 and chi -> 3.7
    w = 1e7
    f = O.drag(rho_f, mu_f, d, [0, 0, -w], v, 1.0)[2]
    newton = -0.63 ** 2 / 8 * rho_f * math.pi * d * d * w * w
    assert f == pytest.approx(newton, rel=3 * 4.8 / 0.63 / math.sqrt(rho_f * d * w / mu_f))
    # drag is along u - v and vanishes with the slip
    assert np.all(O.drag(rho_f, mu_f, d, [0.1, 0.2, 0.3], [0.1, 0.2, 0.3], 0.5) == 0)


# ---------------------------------------------------------------- coarse-graining identities (P9)

@pytest.mark.parametrize("k", [2.0, 3.0])
@pytest.mark.parametrize("bonded", [True, False])
def test_cg_pair_force_scaling(k, bonded):
    """Eq. 22, 24, 28-35: at (kR, k gamma, k delta, k xi, k dt, the same
    velocities and surface speeds, i.e. omega / k) every contact force is k^2
    times the fine one; torques k^3."""
    rho = 2605.0
    Ri, Rj = 1.1e-4, 0.8e-4
    gamma = 0.7
    rng = np.random.default_rng(3)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    delta = 3e-7 if not bonded else -0.2 * (math.pi ** 2 * gamma ** 2 * (Ri * Rj / (Ri + Rj)) / ES ** 2) ** (1 / 3)
    vi, vj = rng.normal(size=3) * 1e-3, rng.normal(size=3) * 1e-3
    wi, wj = rng.normal(size=3), rng.normal(size=3)
    hist = np.cross(n, rng.normal(size=3)) * 1e-9
    outs = []
    for kk in [1.0, k]:
        p = base_params(gamma=kk * gamma, e=0.6, mu=0.4, kind=1, dt=1e-8 * kk, rho=rho)
        mi = rho * 4 / 3 * math.pi * (kk * Ri) ** 3
        mj = rho * 4 / 3 * math.pi * (kk * Rj) ** 3
        xi_pos = np.zeros(3)
        xj_pos = n * (kk * (Ri + Rj) - kk * delta)
        outs.append(O.pair_contact(p, xi_pos, vi, wi / kk, kk * Ri, mi, xj_pos, vj, wj / kk,
                                   kk * Rj, mj, kk * hist, bonded))
    f, c = outs
    assert f[0] and c[0]
    np.testing.assert_allclose(c[1], k ** 2 * f[1], rtol=1e-12, atol=1e-30)
    np.testing.assert_allclose(c[2], k ** 3 * f[2], rtol=1e-12, atol=1e-30)
    assert c[4] == pytest.approx(k ** 2 * f[4], rel=1e-12)   # elastic normal force
    assert c[5] == pytest.approx(k * f[5], rel=1e-12)        # contact radius, Eq. 30
    np.testing.assert_allclose(c[7], k * f[7], rtol=1e-10, atol=1e-25)  # spring, Eq. 29


def test_cg_closed_form_scalings(printed):
    t3 = printed["table3"]
    Rs, g = 6e-5, 30.0
    for k in [2.0, 3.0]:
        # F_C (Table 1) ~ k^2 with gamma_g = k gamma (Eq. 23-24)
        assert (3 * math.pi * k * g * k * Rs) / (3 * math.pi * g * Rs) == pytest.approx(k ** 2)
        assert O.delta_c(k * Rs, ES, k * g) == pytest.approx(k * O.delta_c(Rs, ES, g), rel=1e-13)
        aC = lambda R, gg: (9 * math.pi * gg * R ** 2 / (4 * ES)) ** (1 / 3)
        assert aC(k * Rs, k * g) == pytest.approx(k * aC(Rs, g), rel=1e-13)
        # Rayleigh step ~ k (Eq. 37)
        assert O.rayleigh_dt(k * 1e-4, 2605, 2e10, 0.3) == pytest.approx(k * O.rayleigh_dt(1e-4, 2605, 2e10, 0.3), rel=1e-14)
    # Table 3: N 270000 -> 33750 and gamma 30 -> 60 at k = 2; mass kept (Eq. 17-20)
    rng = np.random.default_rng(0)
    d = I.table2_diameters(t3["N_k1"], rng)
    for scheme in ["ssw", "ssp"]:
        dg, gg = O.cg_scale(d, 2, scheme, t3["gamma_k1"])
        assert len(dg) == t3["N_k2"]
        assert gg == t3["gamma_k2"]
    dg, _ = O.cg_scale(d, 2, "ssp", 30.0)
    assert float((dg ** 3).sum()) == pytest.approx(float((d ** 3).sum()), rel=1e-12)
    dg, _ = O.cg_scale(d, 2, "ssw", 30.0)
    np.testing.assert_allclose(np.unique(dg) * 1e3, np.array(printed["table2"]["d_ssw_mm"])[np.isin(
        printed["table2"]["d_ssw_mm"], np.unique(dg) * 1e3)], rtol=1e-12)


def test_table2_ssp_diameter_and_time_step(printed):
    """SSP diameter = k x volume-mean diameter of Table 2 (printed 0.46 mm);
    Eq. 37-38 with that mean gives 1e-8 s = 4.4 % of the Rayleigh step."""
    t2 = printed["table2"]
    w = np.array(t2["mass_fraction"])
    d = np.array(t2["d_original_mm"]) * 1e-3
    dbar = (w.sum() / (w / d ** 3).sum()) ** (1 / 3)
    assert round(2 * dbar * 1e3, 2) == t2["d_ssp_mm"]
    t3 = printed["table3"]
    dtc = O.rayleigh_dt(dbar / 2, t3["rho"], t3["E"], t3["nu"])
    frac = printed["sec31_time_step"]["dt_dem"] / dtc
    assert round(frac * 100, 1) == round(printed["sec31_time_step"]["fraction_of_rayleigh"] * 100, 1)
    # cells per mean diameter (Sec. 3.1): 1.5 mm / dbar ~ 6.52, coarse k = 2 ~ 3.26
    cells = printed["sec31_cells"]
    assert 1.5e-3 / dbar == pytest.approx(cells["ratio_fine"], rel=5e-3)
    assert 1.5e-3 / (2 * dbar) == pytest.approx(cells["ratio_coarse"], rel=5e-3)


# ---------------------------------------------------------------- pair search (P1)

def _numpy_pairs(x, R, L, skin, periodic=True):
    d = x[None, :, :] - x[:, None, :]
    if periodic:
        d = np.where(d > 0.5 * L, d - L, np.where(d < -0.5 * L, d + L, d))
    d2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]
    S = R[:, None] + R[None, :] + skin
    m = d2 < S * S
    i, j = np.nonzero(np.triu(m, 1))
    return set(zip(i.tolist(), j.tolist()))


def test_contact_search_matches_brute_force():
    s = I.cached(I.small_periodic, 600, 11)
    L = s.domain["L"][0]
    p = base_params(kind=0, L=(L, L, L), gamma=0.0)
    sim = O.Sim(p, s.x, s.v, s.w, s.R)
    sim.compute_forces()
    i, j, b, _ = sim.contacts()
    assert set(zip(i.tolist(), j.tolist())) == _numpy_pairs(s.x, s.R, L, 0.0)
    pi, pj = O.pairs_bruteforce(p, s.x, s.R, 1e-5)
    assert set(zip(pi.tolist(), pj.tolist())) == _numpy_pairs(s.x, s.R, L, 1e-5)


def test_contact_search_periodic_wrap_and_exact_tie():
    L = 2.0 ** -10
    r = 2.0 ** -13
    R = np.array([r, r, r, r])
    # 0-1 overlap across the x boundary; 2-3 touch exactly (d = S in binary, excluded)
    x = np.array([[0.5 * r, 4 * r, 4 * r], [L - 1.25 * r, 4 * r, 4 * r],
                  [4 * r, r, 2 * r], [4 * r, r, 4 * r]])
    p = base_params(kind=0, L=(L, L, L), gamma=0.0)
    sim = O.Sim(p, x, np.zeros((4, 3)), np.zeros((4, 3)), R)
    sim.compute_forces()
    i, j, b, _ = sim.contacts()
    assert list(zip(i.tolist(), j.tolist())) == [(0, 1)]
    assert _numpy_pairs(x, R, L, 0.0) == {(0, 1)}


# ---------------------------------------------------------------- void fraction (P2)

def test_voidfrac_centroid_bruteforce_and_sum():
    s = I.cached(I.small_periodic, 600, 11)
    L = s.domain["L"][0]
    nf = 6
    hf = L / nf
    p = base_params(kind=0, L=(L, L, L), nf=(nf,) * 3, hf=(hf,) * 3, inv_hf=(1 / hf,) * 3,
                    V_cell=hf ** 3)
    S = O.voidfrac(p, s.x, s.R)
    inv_q = 2.0 ** 40 / (hf ** 3)
    V = 4.0 / 3.0 * math.pi * s.R * s.R * s.R
    q = np.rint(V * inv_q).astype(np.uint64)
    c = np.clip(np.floor(s.x * (1 / hf)), 0, nf - 1).astype(np.int64)
    cell = (c[:, 2] * nf + c[:, 1]) * nf + c[:, 0]
    ref = np.zeros(nf ** 3, np.uint64)
    np.add.at(ref, cell, q)
    assert np.array_equal(S, ref)
    assert int(S.sum()) == int(q.sum())
    # porosity: 1 - S 2^-40 equals 1 - (solid volume in the cell)/V_cell to quantum accuracy
    solid = np.zeros(nf ** 3)
    np.add.at(solid, cell, V)
    np.testing.assert_allclose(S.astype(np.float64) * 2.0 ** -40, solid / hf ** 3, atol=1e-11)


def test_voidfrac_cube_overlap_conserves_volume():
    s = I.cached(I.small_periodic, 600, 11)
    L = s.domain["L"][0]
    nf = 8
    hf = L / nf
    p = base_params(kind=0, L=(L, L, L), nf=(nf,) * 3, hf=(hf,) * 3, inv_hf=(1 / hf,) * 3,
                    V_cell=hf ** 3, vf_mode=1)
    S = O.voidfrac(p, s.x, s.R)
    V = 4.0 / 3.0 * math.pi * s.R ** 3
    # each part rounds to one quantum: total within n_parts/2 quanta of the exact volume
    total = float(S.sum()) * hf ** 3 * 2.0 ** -40
    assert total == pytest.approx(V.sum(), rel=1e-9)
    # a cube well inside one cell puts its whole volume there
    x1 = np.array([[0.5 * hf, 0.5 * hf, 0.5 * hf]])
    S1 = O.voidfrac(p, x1, np.array([0.1 * hf]))
    assert np.count_nonzero(S1) == 1 and S1[0] > 0


@pytest.mark.parametrize("case", ["vertex", "face", "quarter", "wide"])
def test_voidfrac_cube_spread_splits_by_the_overlap_fractions(case):
    """The equal-volume cube's spread (R16) puts into each cell the fraction
    of the sphere's volume that the cell cuts from the cube, worked out by
    hand for symmetric placements: centred on a grid vertex, 1/8 in each of
    8 cells; centred on a face, 1/2 and 1/2; a quarter side off a face, 3/4
    and 1/4; a cube 1.5 cells wide centred in a cell, 1/6, 2/3, 1/6 along
    each axis (27 cells, products of those).  Each part is rounded to one
    quantum of 2^-40 cell volumes."""
    nf, hf = 8, 1e-3
    p = base_params(kind=0, L=(nf * hf,) * 3, nf=(nf,) * 3, hf=(hf,) * 3, inv_hf=(1 / hf,) * 3,
                    V_cell=hf ** 3, vf_mode=1)
    side = {"wide": 1.5 * hf}.get(case, 0.6 * hf)
    R = (3.0 / (4.0 * math.pi)) ** (1 / 3) * side  # the sphere whose volume is side^3
    V = side ** 3
    h = hf
    if case == "vertex":
        x, want = (3 * h, 3 * h, 3 * h), {(i, j, k): 1 / 8 for i in (2, 3) for j in (2, 3) for k in (2, 3)}
    elif case == "face":
        x, want = (3 * h, 3.5 * h, 3.5 * h), {(2, 3, 3): 0.5, (3, 3, 3): 0.5}
    elif case == "quarter":
        x, want = (3 * h - side / 4, 3.5 * h, 3.5 * h), {(2, 3, 3): 0.75, (3, 3, 3): 0.25}
    else:
        f = {2: 1 / 6, 3: 2 / 3, 4: 1 / 6}
        x = (3.5 * h,) * 3
        want = {(i, j, k): f[i] * f[j] * f[k] for i in f for j in f for k in f}
    S = O.voidfrac(p, np.array([x]), np.array([R]))
    q = V / hf ** 3 * 2.0 ** 40  # the sphere's volume in quanta
    got = {}
    for c in np.flatnonzero(S):
        iz, rem = divmod(int(c), nf * nf)
        iy, ix = divmod(rem, nf)
        got[(ix, iy, iz)] = int(S[c])
    assert set(got) == set(want), (sorted(got), sorted(want))
    for cell, frac in want.items():
        assert abs(got[cell] - frac * q) <= 1.0, (cell, got[cell], frac * q)


# ---------------------------------------------------------------- whole-step invariants (P8)

def test_momentum_conservation_periodic():
    s = I.cached(I.small_periodic, 600, 11)
    L = s.domain["L"][0]
    rng = np.random.default_rng(1)
    v = rng.normal(size=s.x.shape) * 1e-3
    w = rng.normal(size=s.x.shape) * 1.0
    dtc = O.rayleigh_dt(s.R.mean(), 2650.0, E, NU)
    p = base_params(kind=0, L=(L, L, L), g=(0, 0, 0), dt=0.2 * dtc, gamma=0.5)
    sim = O.Sim(p, s.x, v, w, s.R)
    sim.bond_touching()
    sim.compute_forces()
    m = 2650.0 * 4 / 3 * math.pi * s.R ** 3
    P0 = (m[:, None] * v).sum(0)
    scale = (m[:, None] * np.abs(v)).sum()
    sim.step(200)
    st = sim.state()
    P1 = (m[:, None] * st["v"]).sum(0)
    assert np.abs(P1 - P0).max() <= 1e-13 * scale
    # Newton's third law: contact forces sum to zero
    assert np.abs(st["F"].sum(0)).max() <= 1e-12 * np.abs(st["F"]).sum()
    d = sim.diagnostics()
    assert d["n_bonds"] > 0


def test_gravity_buoyancy_free_fall():
    """One isolated sphere: a = g (1 - rho_f/rho) without drag (Eq. 1)."""
    R = 1e-4
    p = base_params(kind=0, L=(1.0, 1.0, 1.0), g=(0, 0, -9.81), dt=1e-5, use_buoyancy=1)
    sim = O.Sim(p, [[0.5, 0.5, 0.5]], [[0, 0, 0]], [[0, 0, 0]], [R])
    sim.compute_forces()
    sim.step(100)
    v = sim.state()["v"][0, 2]
    assert v == pytest.approx(-9.81 * (1 - 998.2 / 2650.0) * 1e-3, rel=1e-12)


# ------------------------------------------- tangential law, walls, outlet

def _pair_at(overlap, R=1e-4, hist=None, p=None):
    """Two equal unbonded spheres at rest along x with the given overlap."""
    p = p or base_params(gamma=0.0)
    m = 2650.0 * 4 / 3 * math.pi * R ** 3
    return O.pair_contact(p, [0, 0, 0], [0, 0, 0], [0, 0, 0], R, m,
                          [2 * R - overlap, 0, 0], [0, 0, 0], [0, 0, 0], R, m, hist=hist)


def test_tangential_to_normal_stiffness_is_mindlin_ratio():
    """For two identical elastic spheres the tangential contact stiffness
    over the normal one is 2 (1 - nu) / (2 - nu) (Mindlin), whatever the
    overlap: the normal stiffness by central differences of F_ne(delta),
    the tangential one from a spring set in the tangent plane at rest."""
    for delta in (1e-8, 1e-7, 1e-6):
        h = 1e-4 * delta
        kn = (_pair_at(delta + h)[4] - _pair_at(delta - h)[4]) / (2 * h)
        s = 1e-12  # far below the Coulomb limit
        Fi = _pair_at(delta, hist=[0.0, s, 0.0])[1]
        kt = Fi[1] / s
        assert kt / kn == pytest.approx(2 * (1 - NU) / (2 - NU), rel=1e-6)


def test_coulomb_cap_saturates_at_mu_times_normal_force():
    """A stretched spring beyond the Coulomb limit gives |F_t| = mu F_ne
    exactly, along the spring, and the stored spring shrinks to F_t / k_t
    (Eq. 35, R4)."""
    p = base_params(gamma=0.0, mu=0.3)
    delta = 1e-7
    act, Fi, _, _, Fne, _, _, hist, _ = _pair_at(delta, hist=[0.0, 0.0, 1e-6], p=p)
    assert act and Fne > 0
    assert abs(Fi[2]) == pytest.approx(0.3 * Fne, rel=1e-12) and Fi[2] > 0 and Fi[1] == 0.0
    # at rest the spring force is k_t xi: the shrunk spring reproduces the capped force
    Fi2 = _pair_at(delta, hist=list(hist), p=p)[1]
    assert Fi2[2] == pytest.approx(Fi[2], rel=1e-12)


@pytest.mark.parametrize("wall", ["bottom", "side", "top"])
def test_sphere_resting_on_a_wall_has_the_hertz_overlap(wall):
    """One sphere pushed onto a wall of the cylinder by gravity (pointing at
    that wall) and buoyancy comes to rest (damping, e = 0.5) at the overlap
    where the Hertz force of a sphere on a flat, (4/3) E* sqrt(R)
    delta^(3/2), carries its apparent weight m g (1 - rho_f / rho)."""
    R, rho, rho_f, g = 1e-4, 2650.0, 998.2, 9.81
    Rc, H = 0.1, 0.1
    if wall == "bottom":
        gv, x0, k = (0, 0, -g), [0.05, 0.0, R], 2
    elif wall == "side":
        gv, x0, k = (g, 0, 0), [Rc - R, 0.0, 0.05], 0
    else:
        gv, x0, k = (0, 0, g), [0.05, 0.0, H - R], 2
    p = base_params(kind=1, Rc=Rc, H=H, r_out=1e-3, g=gv, dt=1e-6, use_buoyancy=1, gamma=0.0)
    sim = O.Sim(p, [x0], [[0, 0, 0]], [[0, 0, 0]], [R])
    sim.compute_forces()
    sim.step(60000)
    st = sim.state()
    m = rho * 4 / 3 * math.pi * R ** 3
    W = m * g * (1 - rho_f / rho)
    delta = (3 * W / (4 * ES * math.sqrt(R))) ** (2 / 3)
    if wall == "bottom":
        ov = R - st["x"][0, 2]
    elif wall == "side":
        ov = math.hypot(st["x"][0, 0], st["x"][0, 1]) + R - Rc
    else:
        ov = st["x"][0, 2] + R - H
    assert ov == pytest.approx(delta, rel=1e-6)
    assert abs(st["v"][0, k]) < 1e-9 * math.sqrt(g * R)


def test_outlet_removes_a_falling_sphere_on_time():
    """A sphere released above the outlet hole falls freely (velocity
    Verlet is exact under a constant force) and leaves at the first step
    whose position is below -2R (Eq. 40), adding its mass to the produced
    sand."""
    R, rho, rho_f, g, dt = 1e-4, 2650.0, 998.2, 9.81, 1e-5
    z0 = 3e-3
    p = base_params(kind=1, Rc=1.0, H=1.0, r_out=2e-3, g=(0, 0, -g), dt=dt, use_buoyancy=1,
                    gamma=0.0)
    sim = O.Sim(p, [[0.0, 0.0, z0]], [[0, 0, 0]], [[0, 0, 0]], [R])
    sim.compute_forces()
    a = g * (1 - rho_f / rho)
    n = 1
    while z0 - 0.5 * a * (n * dt) ** 2 >= -2 * R:
        n += 1
    sim.step(n + 5)
    assert sim.removed_step()[0] == n
    assert sim.diagnostics()["produced_mass"] == pytest.approx(rho * 4 / 3 * math.pi * R ** 3, rel=1e-14)


def test_cohesive_coulomb_limit_stays_positive_on_the_jkr_branch():
    """Under cohesion the Coulomb limit is F_ne + 2 F_C (R5).  JKR theory
    puts the smallest normal force of the stable branch at -F_C (the
    pull-off force 3 pi gamma R*, Table 1), so the limit never drops below
    F_C even where the bond pulls; a stretched spring saturates at mu times
    it."""
    R, g, mu = 1e-4, 0.5, 0.3
    p = base_params(gamma=g, mu=mu, e=1.0)
    m = 2650.0 * 4 / 3 * math.pi * R ** 3
    Rs = R / 2
    FC = 3 * math.pi * g * Rs
    dC = O.delta_c(Rs, ES, g)
    z = np.zeros(3)
    for frac in (0.999, 0.5, 0.0, -0.5):  # from just above break to compression
        d = frac * dC if frac > 0 else -frac * abs(dC)
        act, Fi, _, _, Fne, _, _, _, bonded = O.pair_contact(
            p, z, z, z, R, m, np.array([2 * R - d, 0, 0]), z, z, R, m, [0.0, 0.0, 1e-5], True)
        assert act and bonded
        assert Fne >= -FC * (1 + 1e-9)
        assert abs(Fi[2]) == pytest.approx(mu * (Fne + 2 * FC), rel=1e-12)
        assert abs(Fi[2]) >= mu * FC * (1 - 1e-9)


# ------------------------------------- tangential dynamics (walls, springs)

def _resting_on_floor(R, rho=2650.0, g=9.81):
    """Overlap of a sphere resting on a flat under its weight (Hertz, sphere on
    a flat: (4/3) E* sqrt(R) delta^(3/2) = m g)."""
    m = rho * 4 / 3 * math.pi * R ** 3
    return (3 * m * g / (4 * ES * math.sqrt(R))) ** (2 / 3), m


@pytest.mark.parametrize("mu", [0.3, 0.8])
def test_sliding_sphere_rolls_at_five_sevenths(mu):
    """A sphere launched along the bottom wall of the cylinder at v0 without
    spin slides, friction at the contact spins it up, and it ends up rolling
    at v = (5/7) v0 whatever the friction coefficient: friction acts at the
    contact point, so the angular momentum about the contact line,
    m R v_x + I w_y with I = (2/5) m R^2, keeps its initial value m R v0 at
    every step; rolling (v_x = R w_y) then fixes v.  Pins the walls'
    tangential law: its sign, its torque arm R and the contact velocity
    v - R w x n it acts on."""
    R, v0 = 1e-4, 1e-3
    delta, m = _resting_on_floor(R)
    I_ = 0.4 * m * R * R
    p = base_params(kind=1, Rc=0.1, H=0.1, r_out=1e-3, g=(0, 0, -9.81), dt=2e-8, gamma=0.0, mu=mu)
    sim = O.Sim(p, [[0.05, 0.0, R - delta]], [[v0, 0, 0]], [[0, 0, 0]], [R])
    sim.compute_forces()
    L0 = m * R * v0
    for _ in range(60):
        sim.step(1000)
        st = sim.state()
        L = m * R * st["v"][0, 0] + I_ * st["w"][0, 1]
        assert L == pytest.approx(L0, rel=1e-11)
    st = sim.state()
    assert st["v"][0, 0] == pytest.approx(5 / 7 * v0, rel=1e-4)
    assert R * st["w"][0, 1] == pytest.approx(st["v"][0, 0], rel=1e-4)


def _rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


@pytest.mark.parametrize("bonded", [False, True])
def test_contact_law_is_frame_indifferent(bonded):
    """A rigid rotation Q of a whole pair (positions, velocities, spins and
    the stored spring, here not in the tangent plane) rotates the forces,
    the torques and the updated spring by Q and changes nothing else: the
    law may depend on the frame only through its vectors (Eq. 3-5, 12-13,
    32-35 are written in vectors)."""
    rng = np.random.default_rng(5)
    R1, R2 = 1.1e-4, 0.8e-4
    m1, m2 = (2650.0 * 4 / 3 * math.pi * r ** 3 for r in (R1, R2))
    p = base_params(gamma=0.5 if bonded else 0.0, mu=0.5)
    x1 = rng.normal(size=3) * 1e-4
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    x2 = x1 + n * (R1 + R2 - 2e-7)
    v1, v2 = rng.normal(size=3) * 1e-3, rng.normal(size=3) * 1e-3
    w1, w2 = rng.normal(size=3), rng.normal(size=3)
    hist = rng.normal(size=3) * 2e-9
    ref = O.pair_contact(p, x1, v1, w1, R1, m1, x2, v2, w2, R2, m2, hist=hist, bonded=bonded)
    Q = _rot(rng.normal(size=3), 1.234)
    rot = O.pair_contact(p, Q @ x1, Q @ v1, Q @ w1, R1, m1, Q @ x2, Q @ v2, Q @ w2, R2, m2,
                         hist=Q @ hist, bonded=bonded)
    assert ref[0] and rot[0] and ref[8] == rot[8] == bonded
    for k in (1, 2, 3, 7):  # Fi, Ti, Tj, updated spring
        scale = np.linalg.norm(ref[k])
        np.testing.assert_allclose(rot[k], Q @ ref[k], rtol=0, atol=1e-12 * scale)
    for k in (4, 5, 6):  # F_ne, contact radius, overlap
        assert rot[k] == pytest.approx(ref[k], rel=1e-12)


def test_spring_follows_the_tangent_plane_keeping_its_length():
    """With no relative motion the stored spring only turns with the contact:
    after one evaluation it lies in the current tangent plane, has kept its
    length, and lies in the plane of its old direction and the normal (it is
    turned, not twisted).  A spring turned the wrong way, or not rescaled,
    fails one of these."""
    R = 1e-4
    m = 2650.0 * 4 / 3 * math.pi * R ** 3
    p = base_params(gamma=0.0, mu=10.0)
    z = np.zeros(3)
    n = np.array([1.0, 0.0, 0.0])
    for tilt in (0.0, 0.05, 0.4):
        hist = np.array([math.sin(tilt), math.cos(tilt), 0.0]) * 3e-10  # tilted out of the plane
        act, Fi, _, _, Fne, a, delta, h, _ = O.pair_contact(p, z, z, z, R, m, n * (2 * R - 1e-7), z, z, R, m,
                                                            hist=hist)
        assert act
        assert abs(h @ n) <= 1e-15 * np.linalg.norm(h)
        assert np.linalg.norm(h) == pytest.approx(np.linalg.norm(hist), rel=1e-14)
        assert abs(np.cross(hist, n) @ h) <= 1e-15 * np.linalg.norm(h) * np.linalg.norm(hist)


def test_tangential_oscillation_on_a_wall_decays_at_the_dashpot_rate():
    """A sphere at rest on the bottom wall, its contact point given a small
    sideways velocity (no slip: mu = 10), oscillates in the tangent plane
    under the spring k_t = 8 G* a and the dashpot g_t = 2 sqrt(5/6) beta
    sqrt(k_t m) (R6) of that contact.  The slip velocity u' = v_x - R w_y obeys
    u'' + g_t u' / m_e + k_t u / m_e = 0 with 1 / m_e = 1 / m + R^2 / I (the
    force acts on translation and, through the arm R, on spin): its zero
    crossings come every half period pi / (w0 sqrt(1 - z^2)) and its peaks
    shrink by exp(-z w0 t), w0^2 = k_t / m_e, z = g_t / (2 sqrt(k_t m_e))."""
    R = 1e-4
    delta, m = _resting_on_floor(R)
    a = math.sqrt(R * delta)
    G = E / (2 * (1 + NU))
    Gs = G / (2 * (2 - NU))
    le = math.log(0.5)
    beta = -le / math.sqrt(le * le + math.pi ** 2)
    kt = 8 * Gs * a
    gt = 2 * math.sqrt(5 / 6) * beta * math.sqrt(kt * m)
    me = 1.0 / (1.0 / m + R * R / (0.4 * m * R * R))
    w0 = math.sqrt(kt / me)
    zeta = gt / (2 * math.sqrt(kt * me))
    wd = w0 * math.sqrt(1 - zeta * zeta)
    dt = 2 * math.pi / w0 / 4000
    p = base_params(kind=1, Rc=0.1, H=0.1, r_out=1e-3, g=(0, 0, -9.81), dt=dt, gamma=0.0, mu=10.0)
    u0 = 1e-7  # slip velocity kick, all in translation
    sim = O.Sim(p, [[0.05, 0.0, R - delta]], [[u0, 0, 0]], [[0, 0, 0]], [R])
    sim.compute_forces()
    t, u = [], []
    for k in range(int(2.2 * 2 * math.pi / wd / dt / 10)):
        sim.step(10)
        st = sim.state()
        t.append((k + 1) * 10 * dt)
        u.append(st["v"][0, 0] - R * st["w"][0, 1])
    t, u = np.array(t), np.array(u)
    # zero crossings by linear interpolation
    s = np.flatnonzero(np.sign(u[:-1]) != np.sign(u[1:]))
    tz = t[s] - u[s] * (t[s + 1] - t[s]) / (u[s + 1] - u[s])
    half = np.diff(tz)
    assert len(half) >= 3
    assert np.median(half) == pytest.approx(math.pi / wd, rel=2e-3)
    # decay of the extrema between successive half periods
    peaks = [np.abs(u[s[i]:s[i + 1]]).max() for i in range(len(s) - 1)]
    ratio = np.array(peaks[1:]) / np.array(peaks[:-1])
    assert np.median(ratio) == pytest.approx(math.exp(-zeta * w0 * math.pi / wd), rel=1e-2)


def test_oracle_threads_change_no_bit():
    """The oracle on one host thread and on all of them: identical states,
    forces and contacts after 30 steps of a cylinder with walls, outlet and
    drag (the pair evaluations run in parallel, their sums in pair order)."""
    from tests.helpers import run_oracle, small_cylinder, default_dt, with_velocities
    s = with_velocities(small_cylinder(), 1e-3)
    out = []
    nmax = O.set_threads(0)
    for t in (1, nmax):
        O.set_threads(t)
        sim = run_oracle(s, default_dt(s), steps=30)
        out.append((sim.state(), sim.contacts(), sim.force_scale(), sim.force_scale_net()))
    O.set_threads(nmax)
    (a, ca, fa, na), (b, cb, fb, nb) = out
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(a[k], b[k]), k
    for u, v in zip(ca, cb):
        assert np.array_equal(u, v)
    assert np.array_equal(fa, fb) and np.array_equal(na, nb)

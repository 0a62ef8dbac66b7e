"""Pins of the oracle's sample-preparation stages (Sec. 3.1): the original
JKR contact of the generation stage (Fig. 1), the top plate that compresses
the sample to an overburden stress, and the penetrometer.

* Original JKR: two particles brought together touch at point A, where the
  force drops to -8/9 F_C (Table 1: -2.67 pi gamma R*); pulled apart they
  follow Eq. 12-13 past the pull-off point C to the turning point S of a
  displacement-driven contact, delta_S = -(3/4) (pi^2 w^2 R* / E*^2)^(1/3)
  with the work of adhesion w = 2 gamma of Eq. 12, where the force is
  -(5/6) pi w R* = -5/9 F_C, and separate there; touching again forms a new
  contact.  A quasi-static cycle dissipates the area of the adhesive lobe
  between S and A, which integrates in closed form.
* Top plate under a stress servo: one sphere between the bottom and the
  plate comes to rest where the plate's force, the target stress times the
  plate area, is the Hertz force of the sphere on each flat.
* Penetrometer (a cylinder with a hemispherical end): the nearest point of
  the tool against a brute-force search along its axis; the stroke (down at constant speed, back up, removed);
  a sphere squeezed under the tip against the bottom carries the Hertz
  force of its overlap, which the tool reports; driven by a force, the tool
  comes to rest where the grains push back with that force, and pulled
  back it goes up from there.
"""
import math

import numpy as np
import pytest

import oracle as O

E, NU = 1e8, 0.3
ES = E / (2 * (1 - NU * NU))


def params(**kw):
    d = dict(rho=2650.0, E=E, nu=NU, e=0.5, mu=0.5, gamma=0.5, rho_f=998.2, mu_f=1e-3,
             use_drag=0, use_buoyancy=0, kind=1, L=(1.0, 1.0, 1.0), Rc=1e-3, H=1e-3, r_out=0.0,
             dt=1e-7, nf=(1, 1, 1), f_lo=(-1e-3, -1e-3, 0), hf=(2e-3, 2e-3, 1e-3),
             inv_hf=(500.0, 500.0, 1000.0), V_cell=4e-9, n_min=0.2, jkr_mode=1)
    d.update(kw)
    return O.make_params(**d)


def pair_force(p, d, R, hist, bonded):
    """Two equal spheres at rest with overlap d (kinematic, no velocity)."""
    z = np.zeros(3)
    m = 2650.0 * 4 / 3 * math.pi * R ** 3
    xj = np.array([2 * R - d, 0.0, 0.0])
    act, Fi, Ti, Tj, Fne, a, delta, hist, bonded = O.pair_contact(p, z, z, z, R, m, xj, z, z, R, m,
                                                                  hist, bonded)
    return act, Fne, hist, bonded


@pytest.mark.parametrize("R,gamma", [(1e-4, 0.5), (2e-4, 5.0)])
def test_original_jkr_forms_at_A_and_separates_at_S(R, gamma, printed):
    p = params(gamma=gamma)
    Rs = R / 2
    FC = 3 * math.pi * gamma * Rs
    xi = (math.pi ** 2 * gamma ** 2 * Rs / ES ** 2) ** (1 / 3)
    w = 2 * gamma
    dS = -0.75 * (math.pi ** 2 * w ** 2 * Rs / ES ** 2) ** (1 / 3)
    assert O.delta_s(Rs, ES, gamma) == pytest.approx(dS, rel=1e-13)
    hist, bonded = np.zeros(3), False
    # approach: no force while apart
    act, Fne, hist, bonded = pair_force(p, -1e-3 * xi, R, hist, bonded)
    assert not act and not bonded
    # touching: point A, the jump to -8/9 F_C (Table 1: -2.67 pi gamma R*)
    act, Fne, hist, bonded = pair_force(p, 1e-12 * xi, R, hist, bonded)
    assert act and bonded
    A = printed["table1"]["A"]["force_over_pi_gamma_Rs"]
    assert round(Fne / (math.pi * gamma * Rs), 2) == A
    assert Fne == pytest.approx(-printed["jkr_jump_fraction_of_FC"]["value"] * FC, rel=1e-6)
    # pulled apart past C: still in contact, the force rises back towards -5/9 F_C
    for d in np.linspace(0.0, dS * (1 - 1e-9), 200):
        act, Fne, hist, bonded = pair_force(p, d, R, hist, bonded)
        assert act and bonded and Fne >= -FC * (1 + 1e-9)
    assert Fne == pytest.approx(-(5 / 6) * math.pi * w * Rs, rel=1e-3)
    # beyond S: separated, no force
    act, Fne, hist, bonded = pair_force(p, dS * (1 + 1e-9), R, hist, bonded)
    assert not act and not bonded
    # separation test right at S, decided without a cube root
    assert O.contact_separates(dS * (1 + 1e-12), Rs, ES, gamma)
    assert not O.contact_separates(dS * (1 - 1e-12), Rs, ES, gamma)
    # touching again forms a new contact at A (the modified JKR would give Hertz)
    act, Fne, hist, bonded = pair_force(p, 1e-12 * xi, R, hist, bonded)
    assert act and bonded and Fne < -0.88 * FC
    q = params(gamma=gamma, jkr_mode=0)
    act, Fne, _, b0 = pair_force(q, 1e-12 * xi, R, np.zeros(3), False)
    assert act and not b0 and 0.0 <= Fne < 1e-12 * FC


def lobe_area(R, gamma):
    """Area of the adhesive lobe of Eq. 12-13 between S and A, -int F d(delta),
    in closed form: with a = c u, u^3 = pi gamma R*^2 / E*, the integral of
    F(a) d(delta)/da is pi gamma u^2 (8 c^5 / 15 - 8 c^(7/2) / 3 + 2 c^2);
    c_A = 4^(1/3) (delta = 0), c_S = 4^(-1/3) (d delta / da = 0)."""
    Rs = R / 2
    u = (math.pi * gamma * Rs ** 2 / ES) ** (1 / 3)

    def Wc(c):
        return 8 * c ** 5 / 15 - 8 * c ** 3.5 / 3 + 2 * c * c

    return math.pi * gamma * u * u * (Wc(4 ** (-1 / 3)) - Wc(4 ** (1 / 3)))


def test_original_jkr_cycle_dissipates_the_lobe():
    """A quasi-static approach to 2 xi of overlap and back: the work of the
    normal force around the cycle is the lobe between S and A (loading and
    unloading follow the same curve above A)."""
    R, gamma = 1e-4, 0.5
    p = params(gamma=gamma)
    Rs = R / 2
    xi = (math.pi ** 2 * gamma ** 2 * Rs / ES ** 2) ** (1 / 3)
    n = 200_000
    path = np.concatenate([np.linspace(-0.2 * xi, 2 * xi, n), np.linspace(2 * xi, -1.4 * xi, n)[1:]])
    hist, bonded = np.zeros(3), False
    F = np.zeros(len(path))
    for k, d in enumerate(path):
        act, Fne, hist, bonded = pair_force(p, d, R, hist, bonded)
        F[k] = Fne if act else 0.0
    # work done on the pair around the cycle, the repulsive force times the
    # overlap's change: what the cycle dissipates
    W = float(np.sum(0.5 * (F[1:] + F[:-1]) * np.diff(path)))
    assert W == pytest.approx(lobe_area(R, gamma), rel=2e-3)


def test_plate_servo_rests_at_the_hertz_overlap():
    """One sphere between the bottom and the top plate, no gravity: the plate
    stops where its force, sigma pi Rc^2, is the Hertz force (4/3) E*
    sqrt(R) delta^(3/2) of the sphere on each flat."""
    R, Rc = 1e-4, 1e-3
    F = 1e-3
    sigma = F / (math.pi * Rc * Rc)
    p = params(Rc=Rc, H=2 * R + 1e-7, gamma=0.0, jkr_mode=0)
    sim = O.Sim(p, [[5e-4, 0.0, R]], [[0, 0, 0]], [[0, 0, 0]], [R])
    A = math.pi * Rc * Rc
    k = 1.5 * F / ((3 * F / (4 * ES * math.sqrt(R))) ** (2 / 3))  # Hertz stiffness at F
    gain = A / (1e-4 * k)  # servo time constant 1e-4 s
    sim.set_stage(O.make_stage(jkr_mode=0, plate_mode=1, plate_stress=sigma, plate_gain=gain,
                               plate_vmax=1.0))
    sim.compute_forces()
    sim.step(30_000)
    b = sim.boundaries()
    delta = (3 * F / (4 * ES * math.sqrt(R))) ** (2 / 3)
    assert b["stress"] == pytest.approx(sigma, rel=1e-6)
    assert abs(b["v_plate"]) <= gain * 1e-6 * sigma
    assert b["H"] == pytest.approx(2 * R - 2 * delta, abs=1e-6 * delta)
    st = sim.state()
    assert st["x"][0, 2] == pytest.approx(R - delta, abs=1e-6 * delta)


def tool_bruteforce(x, rp, zt):
    """Nearest point of the tool's surface to x by a dense search over its
    axis: the tool is every point within rp of the axis from zt + rp up, so
    its surface point nearest to x lies rp from the nearest axis point,
    towards x."""
    zs = np.linspace(zt + rp, zt + rp + 6e-3, 600001)
    dd = np.sqrt(x[0] ** 2 + x[1] ** 2 + (zs - x[2]) ** 2)
    k = int(np.argmin(dd))
    a = np.array([0.0, 0.0, zs[k]])
    return dd[k] - rp, a + rp * (x - a) / dd[k]


def test_penetrometer_nearest_point_against_brute_force():
    rng = np.random.default_rng(5)
    rp, zt, R = 0.85e-3, 2e-3, 1e-4
    # beside the tool, under its tip on and off the axis, around the rim
    cases = [(1.2e-3, 0.3, 3e-3), (0.3e-3, 1.0, 1.9e-3), (0.95e-3, 2.0, 1.95e-3), (1.0e-3, -2.5, 2.0e-3),
             (1e-9, 0.0, 1.85e-3)]
    for _ in range(6):
        cases.append((rng.uniform(0.9e-3, 1.2e-3), rng.uniform(-np.pi, np.pi), rng.uniform(1.8e-3, 3.6e-3)))
    for r, a, z in cases:
        x = np.array([r * math.cos(a), r * math.sin(a), z])
        ov, n = O.tool_overlap(x, R, rp, zt)
        dist, q = tool_bruteforce(x, rp, zt)
        assert R - ov == pytest.approx(dist, abs=2e-10)
        u = (q - x) / np.linalg.norm(q - x)
        assert np.linalg.norm(n) == pytest.approx(1.0, abs=1e-12)
        assert np.dot(n, u) > 1 - 1e-9


def test_penetrometer_stroke():
    """Down at constant speed to the stop height, back up at the same speed,
    removed at the start height; a tip speed of 1e-3 m/s over 1e-7 s steps
    moves it 1e-10 m a step."""
    p = params(gamma=0.0, jkr_mode=0)
    sim = O.Sim(p, [[9e-4, 0.0, 5e-4]], [[0, 0, 0]], [[0, 0, 0]], [1e-4])
    z0, z1, v = 8e-4, 7.9e-4, 1e-3
    sim.set_stage(O.make_stage(pen_mode=1, pen_radius=5e-5, pen_speed=v, pen_z_start=z0, pen_z_stop=z1))
    sim.compute_forces()
    n_down = round((z0 - z1) / (v * p.dt))
    zs, dirs = [], []
    for _ in range(2 * n_down + 5):
        sim.step(1)
        b = sim.boundaries()
        zs.append(b["pen_z"])
        dirs.append(b["pen_dir"])
    dirs = np.array(dirs)
    turn = int(np.argmax(dirs > 0))
    assert abs(turn + 1 - n_down) <= 1
    assert zs[turn] == pytest.approx(z1, abs=2 * v * p.dt)
    gone = int(np.argmax(dirs == 0))
    assert abs(gone + 1 - 2 * n_down) <= 2 and zs[gone] >= z0
    assert np.all(np.diff(zs[:turn]) < 0) and np.all(np.diff(zs[turn:gone + 1]) > 0)


def test_penetrometer_squeezes_a_sphere_onto_the_bottom():
    """The tip comes down slowly onto a sphere resting on the bottom (no
    gravity) and turns back where the sphere is squeezed by d on each flat:
    the force the tool reports there is the Hertz force of that overlap."""
    R = 1e-4
    d = 2e-7
    p = params(gamma=0.0, jkr_mode=0, e=0.3, Rc=2e-3, H=2e-3)
    sim = O.Sim(p, [[0.0, 0.0, R]], [[0, 0, 0]], [[0, 0, 0]], [R])
    z0, z1, v = 2 * R + 1e-7, 2 * R - 2 * d, 2e-4
    sim.set_stage(O.make_stage(pen_mode=1, pen_radius=0.5e-3, pen_speed=v, pen_z_start=z0, pen_z_stop=z1))
    sim.compute_forces()
    Fmax = 0.0
    while True:
        sim.step(1)
        b = sim.boundaries()
        Fmax = max(Fmax, b["pen_force"])
        if b["pen_dir"] > 0:
            break
    F = 4 / 3 * ES * math.sqrt(R) * d ** 1.5
    assert b["pen_force"] == pytest.approx(F, rel=0.03)
    assert Fmax == pytest.approx(F, rel=0.03)


def test_driven_penetrometer_stops_at_its_driving_force():
    """With a driving force, the tip slows as the grains push back and comes
    to rest where the push equals the driving force: on a sphere lying on the
    bottom, where the sphere's Hertz force on each flat is that force."""
    R = 1e-4
    Fd = 5e-3
    p = params(gamma=0.0, jkr_mode=0, e=0.3, Rc=2e-3, H=2e-3)
    sim = O.Sim(p, [[0.0, 0.0, R]], [[0, 0, 0]], [[0, 0, 0]], [R])
    sim.set_stage(O.make_stage(pen_mode=1, pen_radius=0.5e-3, pen_speed=2e-2, pen_z_start=2 * R + 1e-7,
                               pen_z_stop=0.0, pen_force=Fd))
    sim.compute_forces()
    sim.step(40_000)
    b = sim.boundaries()
    delta = (3 * Fd / (4 * ES * math.sqrt(R))) ** (2 / 3)
    assert b["pen_dir"] == -1  # still pressing: it never reached the stop
    assert b["pen_force"] == pytest.approx(Fd, rel=1e-4)
    assert b["pen_z"] == pytest.approx(2 * R - 2 * delta, abs=1e-4 * delta)
    # pulled back from where it stands: up at its speed, removed at the start height
    z = b["pen_z"]
    sim.set_stage(O.make_stage(pen_mode=2, pen_radius=0.5e-3, pen_speed=2e-2, pen_z_start=2 * R + 1e-7,
                               pen_z_stop=0.0, pen_force=Fd))
    sim.step(10)
    b = sim.boundaries()
    assert b["pen_dir"] == 1 and b["pen_z"] == pytest.approx(z + 10 * 2e-2 * p.dt, rel=1e-9)
    sim.step(5000)
    assert sim.boundaries()["pen_dir"] == 0

"""Shared set-up for tests: the same seeded sample fed to the CUDA library and
to the FP64 oracle (which never sees any output of the CUDA path)."""
import math

import numpy as np

import oracle as O
from paper_2211_06142_gb300 import inputs as I


def grain_gamma(material, k, scheme):
    """gamma as the oracle sees it: the paper's grain-level k * gamma (Eq. 24)."""
    return material["gamma"] * (k if scheme != 0 else 1.0)


def oracle_params(s, dt, k=1.0, scheme=0, use_drag=1, use_buoyancy=1, coulomb_mode=0, vf_mode=0,
                  couple_every=1, n_min=0.2, g=None):
    m = s.material
    d = s.domain
    return O.make_params(
        rho=m["rho"], E=m["E"], nu=m["nu"], e=m["e"], mu=m["mu"],
        gamma=grain_gamma(m, k, scheme), rho_f=s.fluid["rho_f"], mu_f=s.fluid["mu_f"],
        use_drag=use_drag, use_buoyancy=use_buoyancy, kind=d["kind"], L=d["L"], Rc=d["Rc"],
        H=d["H"], r_out=d["r_out"], g=s.g if g is None else g, dt=dt, coulomb_mode=coulomb_mode,
        nf=s.grid.nf, f_lo=s.grid.lo, hf=s.grid.h, inv_hf=s.grid.inv_h, V_cell=s.grid.V_cell,
        n_min=n_min, vf_mode=vf_mode, couple_every=couple_every)


def default_dt(s, frac=0.2):
    """0.2 x Rayleigh step of the volume-mean radius (Eq. 37-38), written out here."""
    m = s.material
    Rbar = float(np.mean(s.R ** 3)) ** (1 / 3)
    G = m["E"] / (2 * (1 + m["nu"]))
    beta = 0.8766 + 0.163 * m["nu"]
    return frac * math.pi * Rbar / beta * math.sqrt(m["rho"] / G)


def default_skin(s):
    return 0.05 * 2 * float(s.R.max())


def with_velocities(s, scale, seed=7):
    rng = np.random.default_rng(seed)
    s.v = rng.normal(size=s.x.shape) * scale
    s.w = rng.normal(size=s.x.shape) * scale / float(s.R.mean())
    return s


def small_cylinder(n=3000, seed=21):
    """A scaled-down sand-production cylinder: radius 12 d50, height 10 d50,
    outlet 3 d50, same PSD, radial inflow."""
    d = I.fine_diameters(n, seed)
    return I.cylinder_sample(d, seed, scale=0.3, nf=(12, 12, 6), U_in=0.05, name="cyl-small")


def run_oracle(s, dt, steps=0, bond=True, **kw):
    p = oracle_params(s, dt, **kw)
    sim = O.Sim(p, s.x, s.v, s.w, s.R, s.Us)
    if bond:
        sim.bond_touching()
    sim.couple_fluid()
    sim.compute_forces()
    if steps:
        sim.step(steps)
    return sim


def normwise_error(Fg, Fo, scale):
    """max over particles of |F_gpu - F_oracle| / (sum of force-term magnitudes)."""
    err = np.linalg.norm(Fg - Fo, axis=1)
    return float(np.max(err / np.maximum(scale, 1e-300)))


# ---------------------------------------------------------------------------
# mixed precision over several steps
# ---------------------------------------------------------------------------
#
# One evaluation of the mixed step on the same state is within 1e-4 of the
# oracle (normwise, per particle).  After n steps the two trajectories sit at
# slightly different states, so their forces also differ by what the state
# difference changes: that part is bounded here to first order from the
# oracle's contacts -- normal and tangential stiffness times the position
# differences of the pair, normal and tangential damping times their
# velocity differences (surface velocities included), the drag's slope times
# the velocity difference, the walls likewise -- with a factor of 2 for the
# second-order terms and the tangential history.  The mixed step also takes
# each contact's geometry from positions and radii rounded to a fixed-point
# quantum dq (the library's shadow of the positions), so an overlap carries
# an error of up to (sqrt(3) + 1) dq: its stiffness times that is added (it
# dominates for a contact that has only just formed, a few nm deep).  A
# particle whose contact
# set (with bond flags) differs between the two runs has crossed a touching
# or bond-break threshold in one of them; those are checked separately (every
# differing pair must sit at a threshold) and left out of the force check.

def jkr_radius_np(delta, Rs, Es, gamma, orig=False):
    """Contact radius on the stable branch of Eq. 13 (from point C, or from
    point S for the original JKR), by Newton on the reduced quartic
    (test-side, for a bound)."""
    aA = (4 * np.pi * gamma * Rs * Rs / Es) ** (1 / 3)
    dA = aA * aA / Rs
    D = delta / dA
    u = np.where(D >= 0, (np.maximum(D, 0) + 1) ** 0.25 + 0.05, 1.0)
    for _ in range(60):
        u = u - (u ** 4 - u - D) / (4 * u ** 3 - 1)
    u = np.maximum(u, 0.25 ** (1 / 3) if orig else 0.75 ** (1 / 3))
    return u * u * aA


def tool_overlap_np(x, R, rp, zt):
    """Overlap of each sphere with the penetrometer, a cylinder of radius rp
    ending in a hemisphere with its lowest point at zt (test-side, for a
    bound)."""
    dz = np.maximum(zt + rp - x[:, 2], 0.0)
    return R + rp - np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2 + dz ** 2)


def state_diff(s, g, o):
    dx = g["x"] - o["x"]
    if s.domain["kind"] == 0:
        L = s.domain["L"][0]
        dx -= L * np.round(dx / L)
    return (np.linalg.norm(dx, axis=1), np.linalg.norm(g["v"] - o["v"], axis=1),
            np.linalg.norm(g["w"] - o["w"], axis=1))


def fixed_quantum(s, skin):
    """The fixed-point quantum of the mixed step's position shadow: L / 2^32
    in a periodic cube, else the power of two that puts the largest
    candidate distance 2 r_max + skin below 2^30 quanta."""
    if s.domain["kind"] == 0:
        return s.domain["L"][0] / 2.0 ** 32
    reach = 2 * float(s.R.max()) + skin
    return 2.0 ** math.ceil(math.log2(reach / 2.0 ** 30))


def force_bound(s, o, sim, g, tau, k=1.0, dq=0.0, orig=False, H=None, tool=None, vf=None):
    """Per-particle bounds on |F_gpu - F_oracle| and |T_gpu - T_oracle| after
    several mixed steps (see above); orig: the original JKR's branch for
    the contacts in force; H: the top plate's height, if it moved; tool:
    (radius, tip height) of a penetrometer, if one is in; vf: the two runs'
    porosity cell sums, whose difference (a grain on the other side of a
    cell face in one run) moves the drag of every grain in the cell by at
    most (chi + 2) |dn| / n of it (Eq. 8-11: n^-chi, and u = U / n)."""
    m = s.material
    Es = m["E"] / (2 * (1 - m["nu"] ** 2))
    Gs = m["E"] / (2 * (1 + m["nu"])) / (2 * (2 - m["nu"]))
    le = np.log(m["e"])
    beta = -le / np.sqrt(le * le + np.pi ** 2)
    cd = 2 * np.sqrt(5 / 6) * beta
    gamma = m["gamma"] * k
    R = s.R
    mass = m["rho"] * 4 / 3 * np.pi * R ** 3
    dx, dv, dw = state_diff(s, g, o)
    n = len(R)
    B = np.zeros(n)
    oi, oj, ob, _ = sim.contacts()
    if len(oi):
        d = o["x"][oj] - o["x"][oi]
        if s.domain["kind"] == 0:
            L = s.domain["L"][0]
            d -= L * np.round(d / L)
        dist = np.linalg.norm(d, axis=1)
        Ri, Rj = R[oi], R[oj]
        Rs = Ri * Rj / (Ri + Rj)
        ms = mass[oi] * mass[oj] / (mass[oi] + mass[oj])
        delta = Ri + Rj - dist
        bond = ob.astype(bool) & (gamma > 0)
        a = np.sqrt(Rs * np.maximum(delta, 0))
        kn = 2 * Es * a
        if bond.any():
            ab = jkr_radius_np(delta[bond], Rs[bond], Es, gamma, orig)
            dFda = 4 * Es * ab ** 2 / Rs[bond] - 1.5 * np.sqrt(16 * np.pi * gamma * Es * ab)
            ddda = 2 * ab / Rs[bond] - np.sqrt(np.pi * gamma / (Es * ab))
            a[bond] = ab
            kn[bond] = np.abs(dFda) / np.maximum(ddda, 1e-300)
        kt = 8 * Gs * a
        gn = cd * np.sqrt(2 * Es * a * ms)
        gt = cd * np.sqrt(kt * ms)
        # the dashpots of a Hertz contact grow as delta^(1/4) (Eq. 32 with
        # a = sqrt(R* delta)): at a fresh, small overlap their force moves by
        # (gn |vn| + gt |vt|) / (4 delta) per unit of overlap
        vr = o["v"][oj] - o["v"][oi]
        nrm = d / np.maximum(dist, 1e-300)[:, None]
        vn = np.abs((vr * nrm).sum(1))
        vt = np.linalg.norm(vr - (vr * nrm).sum(1)[:, None] * nrm, axis=1) + Ri * np.linalg.norm(o["w"][oi], axis=1) \
            + Rj * np.linalg.norm(o["w"][oj], axis=1)
        ddamp = np.where(~bond & (delta > 0), (gn * vn + gt * vt) / (4 * np.maximum(delta, 1e-300)), 0.0)
        t = (kn + kt + ddamp) * (dx[oi] + dx[oj] + (math.sqrt(3) + 1) * dq) + \
            (gn + gt) * (dv[oi] + dv[oj] + Ri * dw[oi] + Rj * dw[oj])
        np.add.at(B, oi, t)
        np.add.at(B, oj, t)
    if s.domain["kind"] == 1:
        x = o["x"]
        r = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)
        dom = s.domain
        walls = [r + R - dom["Rc"], np.where(r >= dom["r_out"], R - x[:, 2], -1.0),
                 x[:, 2] + R - (dom["H"] if H is None else H)]
        if tool is not None:
            walls.append(tool_overlap_np(x, R, *tool))
        for dw_ in walls:
            aw = np.sqrt(R * np.maximum(dw_, 0))
            kw = (2 * Es + 8 * Gs) * aw
            gw = cd * (np.sqrt(2 * Es * aw * mass) + np.sqrt(8 * Gs * aw * mass))
            B += np.where(dw_ > 0, kw * dx + gw * (dv + R * dw), 0.0)
    cl = sim.closure_data()
    fd = np.linalg.norm(cl[:, 5:8], axis=1)
    slip = cl[:, 1]
    B += np.where(slip > 0, 2 * fd / np.maximum(slip, 1e-300), 0.0) * dv
    if vf is not None:
        n_min = 0.2
        ng, no = (np.clip(1.0 - a.astype(np.float64) * 2.0 ** -40, n_min, 1.0) for a in vf)
        cell = cl[:, 9].astype(np.int64)
        B += 6.0 * fd * np.abs(ng[cell] - no[cell]) / no[cell]
    scale = sim.force_scale()
    bF = tau * scale + 2 * B
    return bF, R * bF


def agreeing_particles(n, gc, oc):
    """Particles whose contacts (partner and bond flag) agree between the runs.
    gc, oc: (i, j, bonded) arrays."""
    G = set(zip(*(a.tolist() for a in gc)))
    Oc = set(zip(*(a.tolist() for a in oc)))
    ok = np.ones(n, bool)
    for i, j, _ in G ^ Oc:
        ok[i] = ok[j] = False
    return ok


def check_mixed_forces(s, g, o, sim, gc, tau, k=1.0, rows=None, skin=None, **bound_kw):
    """Forces and torques after several mixed steps within force_bound for
    the particles (of `rows`, default all) whose contacts agree; returns the
    number of particles left out."""
    oi, oj, ob, _ = sim.contacts()
    ok = agreeing_particles(len(s.R), gc, (oi, oj, ob))
    if rows is not None:
        ok &= rows
    dq = fixed_quantum(s, default_skin(s) if skin is None else skin)
    bF, bT = force_bound(s, o, sim, g, tau, k, dq, **bound_kw)
    eF = np.linalg.norm(g["F"] - o["F"], axis=1)
    eT = np.linalg.norm(g["T"] - o["T"], axis=1)
    bad = ok & ((eF > bF) | (eT > bT))
    if bad.any():
        b = np.flatnonzero(bad)[:3]
        scale = sim.force_scale()
        info = [dict(i=int(i), eF=float(eF[i]), bF=float(bF[i]), eT=float(eT[i]), bT=float(bT[i]),
                     scale=float(scale[i]), R=float(s.R[i]), x=o["x"][i].tolist(),
                     Fo=o["F"][i].tolist(), Fg=g["F"][i].tolist(),
                     contacts=int(((oi == i) | (oj == i)).sum()),
                     bonds=int((((oi == i) | (oj == i)) & (ob > 0)).sum())) for i in b]
        raise AssertionError(f"mixed forces beyond the bound: {info}")
    return int((~ok).sum() if rows is None else (rows & ~ok).sum())

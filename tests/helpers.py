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

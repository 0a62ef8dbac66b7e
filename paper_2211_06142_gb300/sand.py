"""Produced sand of the fine and the coarse-grained models (Sec. 3.3).

A model of the sand-production cylinder runs for a physical time T; the
cumulative produced mass (Eq. 40: the mass of the grains that left through
the outlet) is read at n equally spaced times.  A coarse model is compared
with the fine one by

* the root-mean-square relative error over the times where the fine model
  has produced sand (Eq. 41, read as 100 sqrt(mean(((M_f - M_c) / M_f)^2)));
* the relative error of the mass produced by the end of the run.

The prescribed radial inflow stands in for the paper's CFD solution
(Sec. 3.1); with it the bonds near the outlet break, and sand is produced
within a few milliseconds, once the inflow velocity at the cylinder wall is
about 0.02 m/s.  Drag on the smallest grains next to the outlet is stiff at
that velocity, so these runs take a time step of 0.02 of the Rayleigh time
(Eq. 37-38) instead of 0.2.

With ``closure`` the learned correction runs in the coarse model's force
kernel; ``record`` keeps the per-particle closure data at every read time
(for training it, see closure.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import cgdem
from . import inputs as I

U_SAND = 0.02      # inflow velocity at the cylinder wall [m/s]
# Sec. 3.4 reads the produced PSD over 0-0.003, 0.003-0.015 and
# 0.015-0.04 s of a 0.04 s run: the same fractions of the run time here
WINDOW_FRACTIONS = (0.075, 0.375, 1.0)


def table2_edges():
    """Size classes of the produced-sand PSD: the eight diameter classes of
    Table 2, each taking the diameters nearer to it than to its neighbours
    (edges at the midpoints) [m]."""
    d = I.TABLE2_DIAMETER_MM * 1e-3
    mid = 0.5 * (d[1:] + d[:-1])
    return np.concatenate([[0.0], mid, [1.0]])
DT_FRAC = 0.02     # time step / Rayleigh time of the volume-mean grain
SKIN_FRAC = 0.04   # candidate-list skin / largest grain diameter


@dataclass
class Production:
    times: np.ndarray      # [n] s
    mass: np.ndarray       # [n] kg, cumulative produced mass
    steps: int
    data: list = field(default_factory=list)  # recorded closure rows per time
    nf: tuple = ()
    psd: np.ndarray = None  # [n, classes] kg, cumulative produced mass per Table 2 class


def rayleigh_dt(s, frac=DT_FRAC):
    m = s.material
    Rbar = float(np.mean(s.R ** 3)) ** (1 / 3)
    return frac * cgdem.cgdem_rayleigh_dt(Rbar, m["rho"], m["E"], m["nu"])


def run(s, k=1, scheme=cgdem.CG_NONE, U_ref=1e-4, T=0.004, n_times=40, precision=cgdem.MIXED,
        closure=None, record=False, device="cuda:0", vf_mode=0, skin_frac=SKIN_FRAC):
    """Run sample s (its field built for an inflow of U_ref, rescaled to
    U_SAND) for time T; returns the produced mass at n_times times."""
    dt = rayleigh_dt(s)
    skin = skin_frac * 2 * float(s.R.max())
    p = cgdem.sample_params(s, dt, skin, k=k, scheme=scheme if k > 1 else cgdem.CG_NONE, vf_mode=vf_mode)
    use_cl = closure is not None or record
    ctx = cgdem.Context([p], [len(s.R)], precision=precision, max_neighbors=64, closure=use_cl,
                        device=device, particles_per_warp=cgdem.spheres_per_warp_for(len(s.R), device))
    try:
        ctx.set_fluid_velocity(s.Us * (U_SAND / U_ref))
        ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=True)
        edges = table2_edges()
        ctx.set_psd_classes(edges)
        if closure is not None:
            theta, lo, hi, cd_max, cg_max = closure
            ctx.set_closure(theta, lo, hi, cd_max, cg_max)
        if record:
            ctx.closure_record(True)
        ctx.compute_forces()
        times = T * np.arange(1, n_times + 1) / n_times
        mass, data, psd, done = [], [], [], 0
        for t in times:
            n = int(round(t / dt)) - done
            if n > 0:
                ctx.step(n)
                done += n
            mass.append(ctx.get_diagnostics()[0]["produced_mass"])
            psd.append(ctx.produced_psd()[0][0, :len(edges) - 1])
            if record:
                data.append(ctx.closure_data().copy())
        return Production(times, np.array(mass), done, data, tuple(int(v) for v in s.grid.nf),
                          np.array(psd))
    finally:
        ctx.close()


def rmsre(ref: Production, mod: Production):
    """Eq. 41 (as read): percent RMS of the relative error over the times
    where the reference has produced sand; None if it produced none."""
    ok = ref.mass > 0
    if not ok.any():
        return None
    r = (ref.mass[ok] - mod.mass[ok]) / ref.mass[ok]
    return float(100.0 * np.sqrt(np.mean(r * r)))


def rmsre_late(ref: Production, mod: Production, frac=0.1):
    """Eq. 41 over the times after the reference has produced frac of its
    final mass (the onset, where a few grains make the relative error, is
    left out)."""
    if not ref.mass[-1] > 0:
        return None
    ok = ref.mass >= frac * ref.mass[-1]
    r = (ref.mass[ok] - mod.mass[ok]) / ref.mass[ok]
    return float(100.0 * np.sqrt(np.mean(r * r)))


def final_error(ref: Production, mod: Production):
    if not ref.mass[-1] > 0:
        return None
    return float(abs(mod.mass[-1] - ref.mass[-1]) / ref.mass[-1])


def normalized_curve(prod: Production):
    """Eq. 39-40: t_d = t / t_end and M_d = cumulative produced mass over its
    value at t_end (None if nothing was produced)."""
    if not prod.mass[-1] > 0:
        return None
    return prod.times / prod.times[-1], prod.mass / prod.mass[-1]


def rmsre_normalized(ref: Production, mod: Production):
    """Eq. 41 (square restored) on the normalised curves of Eq. 40, over the
    read times where the reference's M_d is positive."""
    a, b = normalized_curve(ref), normalized_curve(mod)
    if a is None or b is None:
        return None
    ok = a[1] > 0
    r = (a[1][ok] - b[1][ok]) / a[1][ok]
    return float(100.0 * np.sqrt(np.mean(r * r)))


def psd_windows(prod: Production, fractions=WINDOW_FRACTIONS):
    """Produced mass per Table 2 class in each time window ending at the
    given fractions of the run time (Sec. 3.4, Fig. 11): [windows, classes]."""
    out, prev = [], np.zeros(prod.psd.shape[1])
    for f in fractions:
        i = int(np.argmin(np.abs(prod.times - f * prod.times[-1])))
        out.append(prod.psd[i] - prev)
        prev = prod.psd[i]
    return np.array(out)

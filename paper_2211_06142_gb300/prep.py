"""The paper's sample preparation (Sec. 3.1) as a sequence of library stages.

Generation: the grains settle under gravity with the original JKR contact
(Fig. 1) and Hertz walls, the outlet closed.  Compression: the top plate,
started on the highest grain, moves under a stress servo until the stress
on it is the overburden stress (1 MPa in the paper).  Bonding: the pairs
touching at the end of the compression become the modified JKR's bonds.
Perforation: a penetrometer (1.7 mm in diameter in the paper) goes down the
axis, driven by a constant force at a bounded speed (the paper adjusted its
constant moving force for a gradual perforation), until its tip is one
grain above the bottom or stalls, then back up, and is removed.  The outlet
opens for the sand production.

Every stage runs in the library (cgdem_set_stage, cgdem_step); this module
only sequences them and reads back what they left.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import cgdem

PAPER_STRESS = 1.0e6          # overburden stress of the compression [Pa] (Sec. 3.1)
PAPER_PEN_DIAMETER = 1.7e-3   # penetrometer diameter [m] (Sec. 3.1)
PAPER_E = 2.0e10              # Young's modulus of the grains [Pa] (Table 3)


def scaled_stress(E):
    """The paper's overburden stress for grains of Young's modulus E: the
    same stress over modulus, so that the compression strains the contacts
    as much as in the paper."""
    return PAPER_STRESS * E / PAPER_E


def porosity_under_plate(R, Rc, H):
    """1 - solid volume / volume of the cylinder under the plate."""
    return 1.0 - float((4.0 / 3.0 * math.pi * np.asarray(R) ** 3).sum()) / (math.pi * Rc * Rc * H)


def bonds_per_grain(ctx, n):
    i, j, b = ctx.get_contacts()
    cnt = np.zeros(n, np.int64)
    np.add.at(cnt, i[b > 0], 1)
    np.add.at(cnt, j[b > 0], 1)
    return cnt


def _run(ctx, torch, steps, stage):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.step(steps)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    st = ctx.status()
    if st:
        raise cgdem.CgdemError(st, f"{stage}: {cgdem.lib().cgdem_last_error(ctx.h).decode()}")
    return sec


def prepare(ctx, s, sample=0, gen_steps=2000, stress=PAPER_STRESS, vmax=0.05, gain=None, tol=0.02,
            max_compress_steps=20000, pen_radius=0.5 * PAPER_PEN_DIAMETER, pen_speed=0.2, pen_force=None,
            pen_z_stop=None, max_pen_steps=400000, chunk=500):
    """Run the preparation stages on one cylinder sample of a context made
    with jkr_mode 1 and initialised without bonds.  The penetrometer is
    driven by a force (by default 10 times the overburden stress on its
    cross-section) and turns back at pen_z_stop (by default one largest
    grain diameter above the bottom), or where it stalls against the grains
    under its tip.  The stress should keep the paper's ratio to Young's
    modulus (scaled_stress): far above it, the default driving force that
    follows from it crushes grains between the tool and the bottom.  Returns
    what each stage did (steps, seconds, particle-steps/s, and the stage's
    own figures)."""
    import torch

    n = len(s.R)
    Rc = s.domain["Rc"]
    rec = {}
    # generation: settle with the original JKR, the outlet closed, the plate at the top
    ctx.set_stage(sample, cgdem.stage(jkr_mode=1, outlet_closed=1))
    sec = _run(ctx, torch, gen_steps, "generation")
    ke = ctx.get_diagnostics()[sample]["ke"]
    rec["generation"] = dict(steps=gen_steps, seconds=sec, value=n * gen_steps / sec, ke=ke)
    # compression: the plate from the highest grain down to the overburden stress
    st = ctx.get_state()
    top = min(float((st["x"][:, 2] + s.R).max()), s.domain["H"])
    gain = gain if gain is not None else vmax / (0.5 * stress)
    ctx.set_stage(sample, cgdem.stage(jkr_mode=1, outlet_closed=1, plate_mode=1, plate_H=top,
                                      plate_stress=stress, plate_gain=gain, plate_vmax=vmax))
    steps, sec = 0, 0.0
    while steps < max_compress_steps:
        sec += _run(ctx, torch, chunk, "compression")
        steps += chunk
        b = ctx.boundaries()[sample]
        if abs(b["stress"] - stress) <= tol * stress and abs(b["v_plate"]) <= tol * vmax:
            break
    b = ctx.boundaries()[sample]
    rec["compression"] = dict(steps=steps, seconds=sec, value=n * steps / sec, stress=b["stress"],
                              target=stress, H=b["H"], H_start=top,
                              porosity=porosity_under_plate(s.R, Rc, b["H"]),
                              converged=bool(abs(b["stress"] - stress) <= tol * stress))
    # bonding: the modified JKR's bonds on the pairs touching now (the contacts
    # in force keep their state and springs), the plate held
    ctx.bond_touching()
    ctx.set_stage(sample, cgdem.stage(jkr_mode=0, outlet_closed=1))
    ctx.compute_forces()
    bonds0 = bonds_per_grain(ctx, n)
    rec["bonding"] = dict(bonds=int(bonds0.sum() // 2), per_grain_mean=float(bonds0.mean()),
                          per_grain_max=int(bonds0.max()))
    # perforation: down the axis to the bottom, back up, removed
    H = b["H"]
    pen_force = pen_force if pen_force is not None else 10.0 * stress * math.pi * pen_radius ** 2
    tool = dict(jkr_mode=0, outlet_closed=1, pen_radius=pen_radius, pen_speed=pen_speed, pen_z_start=H,
                pen_z_stop=2.0 * float(s.R.max()) if pen_z_stop is None else pen_z_stop, pen_force=pen_force)
    ctx.set_stage(sample, cgdem.stage(pen_mode=1, **tool))
    def fill(zlo):
        # solid fraction of the space the tool fills with its tip at zlo, up to
        # the plate (a cylinder ending in a hemisphere): the grains whose
        # centres lie inside it
        x = ctx.get_state()["x"]
        az = np.maximum(x[:, 2], zlo + pen_radius)
        dist = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2 + (az - x[:, 2]) ** 2)
        inside = (dist < pen_radius) & (x[:, 2] < H)
        vol = math.pi * pen_radius ** 2 * max(H - zlo - pen_radius, 0.0) + 2.0 / 3.0 * math.pi * pen_radius ** 3
        return float((4.0 / 3.0 * math.pi * s.R[inside] ** 3).sum()) / vol

    steps, sec, fmax, zmin, stalled, at_depth = 0, 0.0, 0.0, H, 0, None
    while steps < max_pen_steps:
        sec += _run(ctx, torch, chunk, "perforation")
        steps += chunk
        b = ctx.boundaries()[sample]
        fmax = max(fmax, b["pen_force"])
        if b["pen_dir"] == 0:
            break
        if b["pen_dir"] < 0:  # a descent that no longer advances turns back
            stalled = stalled + 1 if b["pen_z"] > zmin - 1e-3 * pen_radius else 0
            zmin = min(zmin, b["pen_z"])
            if stalled >= 4:
                at_depth = fill(b["pen_z"])
                ctx.set_stage(sample, cgdem.stage(pen_mode=2, **tool))
        elif at_depth is None:  # turned at the stop height
            at_depth = fill(b["pen_z"])
    bonds1 = bonds_per_grain(ctx, n)
    vol_in = fill(zmin)  # the hole the tool left, between its deepest tip and the plate
    rec["perforation"] = dict(steps=steps, seconds=sec, value=n * steps / sec, removed=bool(b["pen_dir"] == 0),
                              deepest_tip=float(zmin), driving_force=float(pen_force), max_force=float(fmax),
                              bonds_after=int(bonds1.sum() // 2),
                              bonds_broken=int((bonds0.sum() - bonds1.sum()) // 2),
                              solid_fraction_in_path_at_depth=at_depth, solid_fraction_in_hole=vol_in)
    # sand production starts with the outlet open
    ctx.set_stage(sample, cgdem.stage(jkr_mode=0, outlet_closed=0))
    return rec

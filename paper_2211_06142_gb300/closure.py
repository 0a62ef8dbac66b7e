"""Training data, targets and training of the learned closure.

The closure corrects the two terms of a coarse-grained run whose scaling the
paper leaves approximate (Sec. 2.4, Sec. 3): the drag on the parcels
(Eq. 8-11) and their cohesion (Eq. 12-13, surface energy gamma_g = k gamma,
Eq. 24).  Its targets come from runs the library itself makes:

1. a fine run (k = 1) and a plain coarse run (SSW at ratio k) of the same
   domain and fluid field record, at the same physical times, the drag
   force and bond capacity of every particle and the fluid cell it sits in
   (cgdem_closure_record);
2. per fluid cell and time, D = |sum of drag forces| and B = sum of bond
   capacities; the targets of every coarse parcel in the cell are
   y = (ln D_fine / D_coarse, ln B_fine / B_coarse), masked where a sum
   vanishes;
3. the network (cgdem.Closure: tensor-core training kernels) is fitted to
   the parcels' recorded inputs (solid fraction, slip speed, k,
   coordination number, mean overlap / diameter);
4. the coarse run with the closure enabled multiplies each parcel's drag by
   c_d = exp(o_1) and pairs use gamma_g sqrt(c_g,i c_g,j), c_g = exp(o_2).

Every computation runs in the CUDA library; this module moves arrays.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cgdem

COL_FEAT = slice(0, 5)
COL_DRAG = slice(5, 8)
COL_CAP = 8
COL_CELL = 9


@dataclass
class Run:
    """Recorded rows (one [N, 12] array per time), the produced mass and
    the fluid grid's dimensions."""
    data: list
    times: list
    produced: list
    nf: tuple


def make_context(s, dt, skin, k, precision=cgdem.MIXED, max_neighbors=64, scheme=cgdem.CG_SSW,
                 device="cuda:0", **sample_kw):
    p = cgdem.sample_params(s, dt, skin, k=k, scheme=scheme if k > 1 else cgdem.CG_NONE, **sample_kw)
    ctx = cgdem.Context([p], [len(s.R)], precision=precision, max_neighbors=max_neighbors,
                        closure=True, device=device)
    ctx.set_fluid_velocity(s.Us)
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=True)
    return ctx


def record_run(ctx, s, dt, times, closure=None):
    """Step to each time of `times` (seconds, increasing), recording the
    closure data of the last force evaluation before each."""
    if closure is not None:
        theta, lo, hi, cd_max, cg_max = closure
        ctx.set_closure(theta, lo, hi, cd_max, cg_max)
    ctx.closure_record(True)
    ctx.compute_forces()
    done = 0
    data, produced = [], []
    for t in times:
        n = int(round(t / dt)) - done
        if n > 0:
            ctx.step(n)
            done += n
        data.append(ctx.closure_data().copy())
        produced.append(ctx.get_diagnostics()[0]["produced_mass"])
    return Run(data, list(times), produced, tuple(int(v) for v in s.grid.nf))


def _region(cell, nf, merge):
    """Index of the block of merge^3 fluid cells holding each cell."""
    nx, ny, _ = nf
    x, y, z = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    mx, my = -(-nx // merge), -(-ny // merge)
    return ((z // merge) * my + y // merge) * mx + x // merge


def _nregion(nf, merge):
    return int(np.prod([-(-n // merge) for n in nf]))


def cell_sums(rows, nf, merge=1):
    """(D, B, parcels) per block of merge^3 fluid cells from one recorded
    array: D = |sum of drag forces|, B = sum of bond capacities."""
    act = rows[:, 2] > 0  # the k input is positive on every active particle
    reg = _region(rows[act, COL_CELL].astype(np.int64), nf, merge)
    nr = _nregion(nf, merge)
    D = np.zeros((nr, 3))
    np.add.at(D, reg, rows[act][:, COL_DRAG].astype(np.float64))
    B = np.bincount(reg, weights=rows[act, COL_CAP].astype(np.float64), minlength=nr)
    n = np.bincount(reg, minlength=nr)
    return np.linalg.norm(D, axis=1), B, n


def targets(fine: Run, coarse: Run, min_parcels=2, merge=1):
    """Inputs X, targets Y and mask M of every active coarse parcel at every
    recorded time (ratios over blocks of merge^3 fluid cells)."""
    Xs, Ys, Ms = [], [], []
    for rf, rc in zip(fine.data, coarse.data):
        Df, Bf, _ = cell_sums(rf, fine.nf, merge)
        Dc, Bc, nc = cell_sums(rc, coarse.nf, merge)
        okd = (Df > 0) & (Dc > 0) & (nc >= min_parcels)
        okb = (Bf > 0) & (Bc > 0) & (nc >= min_parcels)
        y1 = np.where(okd, np.log(np.where(okd, Df, 1.0) / np.where(okd, Dc, 1.0)), 0.0)
        y2 = np.where(okb, np.log(np.where(okb, Bf, 1.0) / np.where(okb, Bc, 1.0)), 0.0)
        act = rc[:, 2] > 0
        reg = _region(rc[act, COL_CELL].astype(np.int64), coarse.nf, merge)
        Xs.append(rc[act][:, COL_FEAT].astype(np.float64))
        Ys.append(np.stack([y1[reg], y2[reg]], 1))
        Ms.append(np.stack([okd[reg], okb[reg]], 1).astype(np.float64))
    return np.concatenate(Xs), np.concatenate(Ys), np.concatenate(Ms)


def standardisation(X):
    mu = X.mean(0)
    sd = X.std(0)
    return mu, np.where(sd > 1e-12 * np.maximum(1.0, np.abs(mu)), 1.0 / np.maximum(sd, 1e-300), 1.0)


def input_range(X, margin=0.05):
    lo, hi = X.min(0), X.max(0)
    w = np.maximum(hi - lo, 1e-6 * np.maximum(1.0, np.abs(hi)))
    return lo - margin * w, hi + margin * w


def init_theta(mu, inv_sigma, seed, out_bias=(0.0, 0.0)):
    """He-uniform hidden layers, small output layer, zero hidden biases; the
    output biases start at the given values (the mean targets)."""
    rng = np.random.default_rng(seed)
    parts = [np.asarray(mu, np.float64), np.asarray(inv_sigma, np.float64)]
    sizes = [(5, 64), (64, 64), (64, 64), (64, 2)]
    for li, (i, o) in enumerate(sizes):
        bound = np.sqrt(6.0 / i) if li < 3 else 0.1 * np.sqrt(1.0 / i)
        b = np.zeros(o) if li < 3 else np.asarray(out_bias, np.float64)
        parts += [rng.uniform(-bound, bound, size=o * i), b]
    return np.concatenate(parts).astype(np.float32)


def fit(X, Y, M, steps=1000, lr=3e-3, seed=0, device="cuda:0"):
    """Fit the network on the GPU (full-batch Adam); returns (theta, loss
    history).  The output biases start at the masked mean targets."""
    mu, isg = standardisation(X)
    mean = (Y * M).sum(0) / np.maximum(M.sum(0), 1.0)
    net = cgdem.Closure(init_theta(mu, isg, seed, mean), device=device)
    hist = net.train(X, Y, M, steps, lr)
    return net.params(), hist


def cell_drag_error(fine: Run, coarse: Run, min_parcels=2, merge=1):
    """Mean over blocks of merge^3 cells and times of |ln D_coarse / D_fine|
    (blocks holding at least min_parcels parcels and drag on both sides)."""
    errs = []
    for rf, rc in zip(fine.data, coarse.data):
        Df, _, _ = cell_sums(rf, fine.nf, merge)
        Dc, _, nc = cell_sums(rc, coarse.nf, merge)
        ok = (Df > 0) & (Dc > 0) & (nc >= min_parcels)
        errs.append(np.abs(np.log(Dc[ok] / Df[ok])))
    return float(np.mean(np.concatenate(errs)))


def total_drag_error(fine: Run, coarse: Run):
    """Mean over times of |ln sum_cells D_coarse / sum_cells D_fine| (the
    drag magnitude the fluid sees from the whole bed)."""
    errs = []
    for rf, rc in zip(fine.data, coarse.data):
        Df, _, _ = cell_sums(rf, fine.nf)
        Dc, _, _ = cell_sums(rc, coarse.nf)
        errs.append(abs(np.log(Dc.sum() / Df.sum())))
    return float(np.mean(errs))


def cell_bond_error(fine: Run, coarse: Run, min_parcels=2, merge=1):
    errs = []
    for rf, rc in zip(fine.data, coarse.data):
        _, Bf, _ = cell_sums(rf, fine.nf, merge)
        _, Bc, nc = cell_sums(rc, coarse.nf, merge)
        ok = (Bf > 0) & (Bc > 0) & (nc >= min_parcels)
        errs.append(np.abs(np.log(Bc[ok] / Bf[ok])))
    return float(np.mean(np.concatenate(errs)))

"""Project-written autotuner for the step: search-cell size, threads per
block of the fused force kernel, spheres per warp of that kernel (32, or 16
for samples too small to fill the GPU), and the candidate-list skin.

Coordinate search (each knob in turn, the others held at the best so far),
each trial timing a short run of ``cgdem_step`` with CUDA events after a
warm-up; the two fastest settings are then timed again with longer runs.
Results are cached in JSON keyed by a signature of the workload (sphere
counts, domain kinds, largest radii, precision), so a workload is
tuned once per machine.  Every trial computes the same physics: the skin and
the cells only change which candidate pairs are listed, never which pairs
touch.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import cgdem

CELL_SCALES = (0.25, 0.35, 0.5, 0.75, 1.0)
BLOCKS = (64, 128, 256)
SKIN_FRACS = (0.01, 0.02, 0.04, 0.06, 0.09)
PPWS = (32, 16)


def _cache_path():
    root = os.environ.get("CGDEM_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cgdem"))
    return os.path.join(root, "autotune.json")


def signature(params, counts, precision):
    h = hashlib.sha1()
    h.update(repr((2, list(map(int, counts)), int(precision))).encode())
    for p in params:
        h.update(repr((p.kind, round(p.r_max, 12), p.nf[0], p.nf[1], p.nf[2])).encode())
    return h.hexdigest()[:16]


def _with_skin(params, frac):
    out = []
    for p in params:
        q = cgdem.SampleParams()
        C = type(p)
        for name, _ in C._fields_:
            v = getattr(p, name)
            if hasattr(v, "__len__"):
                for i in range(len(v)):
                    getattr(q, name)[i] = v[i]
            else:
                setattr(q, name, v)
        q.skin = frac * 2 * p.r_max
        out.append(q)
    return out


def trial(params, counts, state, Us, precision, cell_scale, block, steps=600, warm=50,
          device="cuda:0", max_neighbors=48, ppw=32):
    import torch
    ctx = cgdem.Context(params, counts, precision=precision, max_neighbors=max_neighbors,
                        block_size=block, cell_scale=cell_scale, device=device,
                        particles_per_warp=ppw)
    try:
        ctx.set_fluid_velocity(Us)
        ctx.init_particles(*state, bond_touching=True)
        ctx.compute_forces()
        ctx.step(warm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.step(steps)
        e1.record()
        torch.cuda.synchronize()
        ctx.status()
        return e0.elapsed_time(e1) / steps
    finally:
        ctx.close()


def autotune(params, counts, state, Us, precision=cgdem.MIXED, device="cuda:0", use_cache=True,
             steps=600, log=None):
    """Return {"cell_scale", "block", "skin_frac", "ppw", "ms_per_step", "trials"} for the
    workload."""
    key = signature(params, counts, precision)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return dict(cache[key], cached=True)
    best = {"cell_scale": 0.35, "block": 128, "skin_frac": 0.02, "ppw": 32}
    trials = []

    def run(cs, b, sf, pw, n=steps):
        try:
            ms = trial(_with_skin(params, sf), counts, state, Us, precision, cs, b, steps=n,
                       device=device, ppw=pw)
        except cgdem.CgdemError as e:  # e.g. a skin below the bond-break separation
            ms = float("inf")
            if log:
                log(f"trial cs={cs} block={b} skin={sf} ppw={pw}: {e}")
        trials.append({"cell_scale": cs, "block": b, "skin_frac": sf, "ppw": pw, "ms_per_step": ms})
        return ms

    best_ms = run(best["cell_scale"], best["block"], best["skin_frac"], best["ppw"])
    for knob, values in (("cell_scale", CELL_SCALES), ("block", BLOCKS), ("skin_frac", SKIN_FRACS),
                         ("ppw", PPWS)):
        for v in values:
            if v == best[knob]:
                continue
            cand = dict(best, **{knob: v})
            ms = run(cand["cell_scale"], cand["block"], cand["skin_frac"], cand["ppw"])
            if ms < best_ms:
                best, best_ms = cand, ms
    # the short trials carry a few per cent of noise: the two fastest distinct
    # settings are timed again, twice each with runs twice as long
    keys = ("cell_scale", "block", "skin_frac", "ppw")
    ranked, seen = [], set()
    for t in sorted(trials, key=lambda t: t["ms_per_step"]):
        k = tuple(t[x] for x in keys)
        if k not in seen and t["ms_per_step"] < float("inf"):
            seen.add(k)
            ranked.append(dict(zip(keys, k)))
    if len(ranked) > 1:
        mean = {}
        for c in ranked[:2]:
            mean[tuple(c[x] for x in keys)] = sum(
                run(c["cell_scale"], c["block"], c["skin_frac"], c["ppw"], 2 * steps) for _ in range(2)) / 2
        k = min(mean, key=mean.get)
        best, best_ms = dict(zip(keys, k)), mean[k]
    res = dict(best, ms_per_step=best_ms, trials=trials)
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            cache[key] = res
            tmp = path + ".tmp.%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
    return dict(res, cached=False)


def tuned_params(params, result):
    return _with_skin(params, result["skin_frac"])


def skin_factors(rates, quantile=0.75, max_factor=2.5):
    """Per-sample skin multipliers from each sample's drift rate (largest
    speed x dt / skin): a rebuild of the ensemble is due when any member has
    moved half its skin, so members that drift faster than the given
    quantile of the ensemble get a proportionally larger skin (at most
    max_factor), and the ensemble rebuilds at the pace of the bulk of its
    members instead of its fastest one."""
    rates = np.asarray(rates, float)
    ref = float(np.quantile(rates, quantile)) if len(rates) else 0.0
    if not ref > 0.0:
        return np.ones(len(rates))
    return np.clip(rates / ref, 1.0, max_factor)


def balance_skins(params, counts, state, Us, precision=cgdem.MIXED, cell_scale=0.0, block=128, ppw=32,
                  steps=300, device="cuda:0", max_neighbors=48, **kw):
    """Run the ensemble for `steps` steps, measure each member's drift rate
    and return its parameters with skins scaled by `skin_factors` (and the
    factors)."""
    ctx = cgdem.Context(params, counts, precision=precision, max_neighbors=max_neighbors,
                        block_size=block, cell_scale=cell_scale, device=device, particles_per_warp=ppw)
    try:
        ctx.set_fluid_velocity(Us)
        ctx.init_particles(*state, bond_touching=True)
        ctx.compute_forces()
        ctx.step(steps)
        v = ctx.get_state()["v"]
    finally:
        ctx.close()
    rates, off = [], 0
    for p, n in zip(params, counts):
        vm = float(np.sqrt((v[off:off + n] ** 2).sum(1)).max()) if n else 0.0
        off += n
        rates.append(vm * p.dt / p.skin if p.skin > 0 else 0.0)
    f = skin_factors(rates, **kw)
    out = []
    for p, fk in zip(params, f):
        q = _with_skin([p], p.skin / (2 * p.r_max))[0]
        q.skin = p.skin * float(fk)
        out.append(q)
    return out, f

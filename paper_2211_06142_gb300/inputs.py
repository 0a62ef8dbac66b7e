"""Seeded synthetic inputs for the coarse-grained CFD-DEM step.

This module only draws inputs: particle size distributions, packed
positions, initial velocities and the prescribed superficial fluid-velocity
field, plus the workload descriptions they belong to.  It holds none of the
method's arithmetic (no contact law, no coarse-graining rule, no time-step
rule), so both the CUDA library and the CPU oracle can be fed from it.

Workloads stand in for the paper's reservoir-sand sample (Sec. 3.1, Table 2);
there is no public dataset, so every array here is drawn from a seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# fluid properties of Table 4 (water)
WATER_RHO = 998.2
WATER_MU = 1.0e-3

# Table 2: mass fraction per diameter class of the original particles [mm]
TABLE2_MASS_FRACTION = np.array([0.058, 0.075, 0.088, 0.1216, 0.2264, 0.1705, 0.121, 0.1395])
TABLE2_DIAMETER_MM = np.array([0.15, 0.18, 0.2, 0.22, 0.25, 0.275, 0.3, 0.355])


def lognormal_diameters(n: int, d50: float, sigma_ln: float, dmin: float, dmax: float,
                        rng: np.random.Generator) -> np.ndarray:
    """Diameters with a log-normal distribution truncated to [dmin, dmax].

    d50 is read as the MASS median (sieve analyses such as Table 2 are by
    mass); the number median of a log-normal with log-standard deviation
    sigma is then d50 * exp(-3 sigma^2).
    """
    mu = math.log(d50) - 3.0 * sigma_ln ** 2
    out = np.empty(0)
    while out.size < n:
        d = np.exp(rng.normal(mu, sigma_ln, size=2 * (n - out.size) + 16))
        d = d[(d >= dmin) & (d <= dmax)]
        out = np.concatenate([out, d])
    return out[:n].copy()


def table2_diameters(n: int, rng: np.random.Generator) -> np.ndarray:
    """Diameters drawn from the 8 classes of Table 2 (by mass) [m]."""
    d = TABLE2_DIAMETER_MM * 1e-3
    w = TABLE2_MASS_FRACTION / d ** 3
    idx = rng.choice(len(d), size=n, p=w / w.sum())
    return d[idx]


# ---------------------------------------------------------------------------
# packing: random placement, then overlap removal (geometry only)
# ---------------------------------------------------------------------------

_PACKER = None


def _packer():
    """Load (compiling on first use) the C overlap-removal packer."""
    global _PACKER
    if _PACKER is None:
        import ctypes
        import os
        import subprocess

        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "gen", "packer.c")
        out_dir = os.path.join(here, "_build")
        lib = os.path.join(out_dir, "libcgdem_packer.so")
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            os.makedirs(out_dir, exist_ok=True)
            tmp = lib + ".tmp.%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
            os.replace(tmp, lib)
        L = ctypes.CDLL(lib)
        pd = ctypes.POINTER(ctypes.c_double)
        L.gen_pack.restype = ctypes.c_int
        L.gen_pack.argtypes = [ctypes.c_int64, pd, pd, ctypes.c_int, pd, ctypes.c_int, ctypes.c_double]
        _PACKER = L
    return _PACKER


def _pack(x, R, kind, geo, iters, tol):
    import ctypes

    pd = ctypes.POINTER(ctypes.c_double)
    x = np.ascontiguousarray(x, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    g = np.ascontiguousarray(geo, dtype=np.float64)
    _packer().gen_pack(len(R), x.ctypes.data_as(pd), R.ctypes.data_as(pd), kind,
                       g.ctypes.data_as(pd), iters, tol)
    return x


def pack_periodic(R: np.ndarray, L: float, rng: np.random.Generator, iters: int = 2000,
                  tol: float = 0.01, squeeze: float = 0.005) -> np.ndarray:
    """Positions of spheres of radii R in the periodic cube [0, L)^3.

    The spheres are packed with radii R (1 - squeeze) and returned at full
    size, so that neighbours closer than squeeze (Ri + Rj) overlap slightly,
    as in a compressed sample.
    """
    x = rng.uniform(0.0, L, size=(len(R), 3))
    x = _pack(x, np.asarray(R) * (1.0 - squeeze), 0, [L], iters, tol)
    return np.mod(x, L)


def pack_cylinder(R: np.ndarray, Rc: float, r_out: float, h_bed: float, rng: np.random.Generator,
                  iters: int = 2000, tol: float = 0.01, squeeze: float = 0.005) -> np.ndarray:
    """Positions of spheres inside the annulus r_out < r < Rc, 0 < z < h_bed.

    The central cavity r < r_out (left by the perforation stage) is empty.
    Packed at radii R (1 - squeeze) as in pack_periodic.
    """
    n = len(R)
    u = rng.uniform(0, 1, n)
    rr = np.sqrt(r_out ** 2 + u * (Rc ** 2 - r_out ** 2))
    th = rng.uniform(0, 2 * math.pi, n)
    z = rng.uniform(0, h_bed, n)
    x = np.stack([rr * np.cos(th), rr * np.sin(th), z], 1)
    return _pack(x, np.asarray(R) * (1.0 - squeeze), 1, [Rc, r_out, h_bed], iters, tol)


# ---------------------------------------------------------------------------
# prescribed superficial fluid velocity on a Cartesian grid
# ---------------------------------------------------------------------------

@dataclass
class FluidGrid:
    nf: tuple
    lo: tuple
    h: tuple

    @property
    def inv_h(self):
        return tuple(1.0 / v for v in self.h)

    @property
    def V_cell(self):
        return self.h[0] * self.h[1] * self.h[2]

    @property
    def ncell(self):
        return self.nf[0] * self.nf[1] * self.nf[2]

    def centres(self):
        idx = np.indices(self.nf[::-1]).reshape(3, -1)[::-1].T  # x fastest
        return np.asarray(self.lo) + (idx + 0.5) * np.asarray(self.h)


def uniform_field(grid: FluidGrid, U) -> np.ndarray:
    return np.tile(np.asarray(U, dtype=np.float64), (grid.ncell, 1))


def radial_inflow_field(grid: FluidGrid, U_in: float, Rc: float, r_out: float,
                        h_bed: float) -> np.ndarray:
    """Superficial velocity of a radial inflow towards a central perforation.

    Outside the cavity: U_s = -U_in (Rc / r) e_r (volume flux through every
    cylinder r = const is the same).  Inside the cavity (r < r_out) the
    collected flux leaves downwards through the outlet: u_z grows linearly
    with depth below the bed top, u_z = -2 Rc U_in (h_bed - z) / r_out^2.
    """
    c = grid.centres()
    r = np.sqrt(c[:, 0] ** 2 + c[:, 1] ** 2)
    U = np.zeros_like(c)
    out = r >= r_out
    s = -U_in * Rc / np.maximum(r[out], 1e-300)
    U[out, 0] = s * c[out, 0] / np.maximum(r[out], 1e-300)
    U[out, 1] = s * c[out, 1] / np.maximum(r[out], 1e-300)
    cav = ~out
    depth = np.clip(h_bed - c[cav, 2], 0.0, h_bed)
    U[cav, 2] = -2.0 * Rc * U_in * depth / r_out ** 2
    return U


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

@dataclass
class Sample:
    """One packed sample, grain level, plus the description of its setting."""
    name: str
    x: np.ndarray          # [N,3] m
    v: np.ndarray          # [N,3] m/s
    w: np.ndarray          # [N,3] rad/s
    R: np.ndarray          # [N] m
    material: dict         # rho, E, nu, e, mu, gamma (grain level)
    domain: dict           # kind, L, Rc, H, r_out
    grid: FluidGrid
    Us: np.ndarray         # [ncell,3] superficial fluid velocity
    fluid: dict = field(default_factory=lambda: dict(rho_f=WATER_RHO, mu_f=WATER_MU))
    g: tuple = (0.0, 0.0, -9.81)
    extra: dict = field(default_factory=dict)


def fine_diameters(n: int, seed: int, d50: float = 0.25e-3, sigma_ln: float = 0.4,
                   dmin: float = 0.1e-3, dmax: float = 0.6e-3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return lognormal_diameters(n, d50, sigma_ln, dmin, dmax, rng)


def periodic_sample(d: np.ndarray, phi: float, seed: int, nf: int = 8, U=(0.0, 0.0, 0.01),
                    material=None, name="periodic", vel_scale=0.0) -> Sample:
    """Spheres of diameters d packed to solid fraction phi in a periodic cube."""
    rng = np.random.default_rng(seed + 1000)
    R = 0.5 * np.asarray(d, dtype=np.float64)
    Vs = float((4.0 / 3.0 * math.pi * R ** 3).sum())
    L = (Vs / phi) ** (1.0 / 3.0)
    x = pack_periodic(R, L, rng)
    v = rng.normal(0.0, 1.0, size=x.shape) * vel_scale
    w = np.zeros_like(x)
    h = L / nf
    grid = FluidGrid((nf, nf, nf), (0.0, 0.0, 0.0), (h, h, h))
    mat = material or dict(rho=2650.0, E=1e8, nu=0.3, e=0.5, mu=0.5, gamma=0.5)
    dom = dict(kind=0, L=(L, L, L), Rc=0.0, H=0.0, r_out=0.0)
    return Sample(name, x, v, w, R, dict(mat), dom, grid, uniform_field(grid, U))


def cylinder_sample(d: np.ndarray, seed: int, d50: float = 0.25e-3, scale: float = 1.0,
                    phi: float = 0.55, U_in: float = 0.01, nf=(40, 40, 20), material=None,
                    name="cylinder", cavity: bool = True) -> Sample:
    """Sand-production sample: cylinder Rc = 40 d50, H = 30 d50 (x scale),
    central perforation outlet r_out = 3 d50 on the lower face, bed packed from
    z = 0 to the height that holds the spheres at solid fraction phi, with the
    perforation over the outlet left empty (cavity) or the bed whole (for the
    preparation stages, whose penetrometer makes the perforation)."""
    rng = np.random.default_rng(seed + 2000)
    R = 0.5 * np.asarray(d, dtype=np.float64)
    Rc = 40.0 * d50 * scale
    H = 30.0 * d50 * scale
    r_out = 3.0 * d50
    r_cav = r_out if cavity else 0.0
    Vs = float((4.0 / 3.0 * math.pi * R ** 3).sum())
    h_bed = Vs / (phi * math.pi * (Rc ** 2 - r_cav ** 2))
    if not h_bed <= H:
        raise ValueError(f"{name}: the cylinder (Rc {Rc:.3g}, H {H:.3g}, cavity {r_cav:.3g}) cannot hold "
                         f"the grains at solid fraction {phi}")
    x = pack_cylinder(R, Rc, r_cav, h_bed, rng)
    v = np.zeros_like(x)
    w = np.zeros_like(x)
    h = (2 * Rc / nf[0], 2 * Rc / nf[1], H / nf[2])
    grid = FluidGrid(tuple(nf), (-Rc, -Rc, 0.0), h)
    mat = material or dict(rho=2650.0, E=1e8, nu=0.3, e=0.5, mu=0.5, gamma=0.5)
    dom = dict(kind=1, L=(2 * Rc, 2 * Rc, H), Rc=Rc, H=H, r_out=r_out)
    return Sample(name, x, v, w, R, dict(mat), dom, grid,
                  radial_inflow_field(grid, U_in, Rc, r_out, h_bed), extra=dict(h_bed=h_bed))


def cached(fn, *args, **kw) -> Sample:
    """Call a workload constructor, memoising its result on disk.

    The cache lives in $CGDEM_CACHE (default ~/.cache/cgdem) and is keyed by
    the constructor name and its arguments; delete it to regenerate.
    """
    import hashlib
    import os
    import pickle

    root = os.environ.get("CGDEM_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cgdem"))
    key = hashlib.sha1(repr((fn.__name__, args, sorted(kw.items()), 5)).encode()).hexdigest()[:16]
    path = os.path.join(root, f"{fn.__name__}-{key}.pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    s = fn(*args, **kw)
    try:
        os.makedirs(root, exist_ok=True)
        tmp = path + ".tmp.%d" % os.getpid()
        with open(tmp, "wb") as f:
            pickle.dump(s, f)
        os.replace(tmp, path)
    except OSError:
        pass
    return s


def _tile_block(n_block: int, seed: int, phi: float = 0.55, d_map=None):
    """A periodic block of n_block fine-PSD spheres packed at solid fraction
    phi: diameters, positions in [0, L)^3 and L.  Copies of a periodic packing
    placed side by side form a packing of the larger region with no seams
    (every contact across a block face is a contact across the period).
    d_map, if given, maps the fine diameters to the ones packed (a
    coarse-graining rule)."""
    rng = np.random.default_rng(seed + 3000)
    d = fine_diameters(n_block, seed)
    if d_map is not None:
        d = np.asarray(d_map(d), np.float64)
    R = 0.5 * d
    L = (float((4.0 / 3.0 * math.pi * R ** 3).sum()) / phi) ** (1.0 / 3.0)
    x = pack_periodic(R, L, rng)
    return R, x, L


def tiled_cylinder(n_target: int = 2_000_000, scale: float = 2.15, seed: int = 4,
                   n_block: int = 65_536, d50: float = 0.25e-3, U_in: float = 1e-4,
                   nf=(86, 86, 43), d_map=None, h_bed: float = 0.0, name: str = "cylinder-tiled") -> Sample:
    """The sand-production cylinder scaled by `scale` in radius and height
    (radius 40 d50 scale, height 30 d50 scale, outlet 3 d50, fluid cells of
    the 200k-sphere cylinder's size), holding about n_target spheres of the
    same PSD at solid fraction 0.55: copies of one packed periodic block of
    n_block spheres tile the region, and the spheres whose centres lie in
    the bed annulus (r_out + R <= r <= Rc - R, R <= z <= h_bed) are kept.
    Packing n_target spheres directly takes the host packer tens of minutes;
    the tiled bed repeats the block's arrangement every block edge.
    A coarse-grained counterpart packs its block with the diameters d_map
    gives and fills the bed height h_bed of the fine sample (n_target is
    then unused)."""
    Rb, xb, Lb = _tile_block(n_block, seed, d_map=d_map)
    Vmean = float((4.0 / 3.0 * math.pi * Rb ** 3).mean())
    Rc = 40.0 * d50 * scale
    H = 30.0 * d50 * scale
    r_out = 3.0 * d50
    if not h_bed > 0.0:
        h_bed = n_target * Vmean / (0.55 * math.pi * (Rc ** 2 - r_out ** 2))
    if not h_bed <= H:
        raise ValueError("the scaled cylinder cannot hold n_target spheres at solid fraction 0.55")
    nxy = int(math.ceil(2 * Rc / Lb))
    nz = int(math.ceil(h_bed / Lb))
    xs, Rs = [], []
    for a in range(nxy):
        for b in range(nxy):
            for c in range(nz):
                q = xb + np.array([a * Lb - Rc, b * Lb - Rc, c * Lb])
                r = np.sqrt(q[:, 0] ** 2 + q[:, 1] ** 2)
                keep = ((r >= r_out + Rb) & (r <= Rc - Rb) & (q[:, 2] >= Rb) & (q[:, 2] <= h_bed))
                xs.append(q[keep])
                Rs.append(Rb[keep])
    x = np.concatenate(xs)
    R = np.concatenate(Rs)
    h = (2 * Rc / nf[0], 2 * Rc / nf[1], H / nf[2])
    grid = FluidGrid(tuple(nf), (-Rc, -Rc, 0.0), h)
    mat = dict(rho=2650.0, E=1e8, nu=0.3, e=0.5, mu=0.5, gamma=0.5)
    dom = dict(kind=1, L=(2 * Rc, 2 * Rc, H), Rc=Rc, H=H, r_out=r_out)
    return Sample(f"{name}-{len(R)}", x, np.zeros_like(x), np.zeros_like(x), R, mat, dom,
                  grid, radial_inflow_field(grid, U_in, Rc, r_out, h_bed),
                  extra=dict(h_bed=h_bed, block_spheres=len(Rb), block_edge=Lb))


def tiled_bed_height(n_target: int = 2_000_000, scale: float = 2.15, seed: int = 4, n_block: int = 65_536,
                     d50: float = 0.25e-3) -> float:
    """The bed height tiled_cylinder fills with n_target fine spheres (the
    block's mean sphere volume at solid fraction 0.55 over the annulus)."""
    Rb = 0.5 * fine_diameters(n_block, seed)
    Vmean = float((4.0 / 3.0 * math.pi * Rb ** 3).mean())
    Rc = 40.0 * d50 * scale
    r_out = 3.0 * d50
    return n_target * Vmean / (0.55 * math.pi * (Rc ** 2 - r_out ** 2))


def tiled_periodic(n_block: int = 12_500, reps: int = 2, seed: int = 8, nf: int = 16,
                   U=(0.0, 0.0, 0.01)) -> Sample:
    """A periodic cube of reps^3 copies of one packed periodic block of
    n_block fine-PSD spheres (solid fraction 0.55): a large periodic packing
    at the cost of packing the block."""
    Rb, xb, Lb = _tile_block(n_block, seed)
    xs = [xb + Lb * np.array([a, b, c]) for a in range(reps) for b in range(reps) for c in range(reps)]
    x = np.concatenate(xs)
    R = np.tile(Rb, reps ** 3)
    L = reps * Lb
    h = L / nf
    grid = FluidGrid((nf, nf, nf), (0.0, 0.0, 0.0), (h, h, h))
    mat = dict(rho=2650.0, E=1e8, nu=0.3, e=0.5, mu=0.5, gamma=0.5)
    dom = dict(kind=0, L=(L, L, L), Rc=0.0, H=0.0, r_out=0.0)
    return Sample(f"periodic-tiled-{len(R)}", np.mod(x, L), np.zeros_like(x), np.zeros_like(x), R, mat,
                  dom, grid, uniform_field(grid, U))


def small_periodic(n: int = 2000, seed: int = 0) -> Sample:
    """2,000 log-normal spheres (mass-median 0.25 mm, sigma_ln 0.4, 0.1-0.6 mm)
    at solid fraction 0.55 in a periodic cube, 8^3 fluid grid, uniform
    superficial velocity 0.01 m/s."""
    return periodic_sample(fine_diameters(n, seed), 0.55, seed, name="periodic-2k")


def whole_cylinder(n: int = 200_000, seed: int = 1) -> Sample:
    """The 200k-sphere cylinder's bed packed whole, without the perforation
    (the preparation stages make it), and no prescribed flow."""
    return cylinder_sample(fine_diameters(n, seed), seed, U_in=0.0, name="cylinder-whole", cavity=False)


def fine_cylinder(n: int = 200_000, seed: int = 1, U_in: float = 1e-4) -> Sample:
    """200,000 spheres, same PSD, in the 40x40x20-cell sand-production cylinder,
    with the paper's injection velocity of 1e-4 m/s (Sec. 3.1)."""
    return cylinder_sample(fine_diameters(n, seed), seed, U_in=U_in, name="cylinder-200k")


# ---------------------------------------------------------------------------
# batched ensemble (a calibration sweep): many independent samples
# ---------------------------------------------------------------------------

@dataclass
class SampleSpec:
    """Description of one ensemble member before coarse-graining."""
    index: int
    n_grains: int
    d50: float
    gamma: float         # fine-scale surface energy [J/m^2]
    k: int               # coarse-graining ratio
    kind: int            # 0 periodic cube, 1 cylinder
    seed: int
    d_fine: np.ndarray   # n_grains * k^3 fine diameters (a PSD realisation)


def ensemble_specs(n_samples: int = 64, seed: int = 3, n_lo: int = 5000, n_hi: int = 50000,
                   d50_lo: float = 0.15e-3, d50_hi: float = 0.35e-3, g_lo: float = 0.1,
                   g_hi: float = 2.0, ks=(1, 2, 3)):
    """Seeded draws of the ensemble: grain count uniform in [n_lo, n_hi], d50
    uniform, surface energy uniform, ratio k from ks, half periodic and half
    cylindrical.  Each member carries n_grains * k^3 fine diameters, from
    which the coarse-graining rule makes n_grains grains."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_samples):
        n = int(rng.integers(n_lo, n_hi + 1))
        d50 = float(rng.uniform(d50_lo, d50_hi))
        g = float(rng.uniform(g_lo, g_hi))
        k = int(ks[int(rng.integers(0, len(ks)))])
        kind = i % 2
        r2 = np.random.default_rng(seed * 1000 + i)
        d = lognormal_diameters(n * k ** 3, d50, 0.4, 0.4 * d50, 2.4 * d50, r2)
        out.append(SampleSpec(i, n, d50, g, k, kind, seed * 1000 + i, d))
    return out


def pack_member(spec: SampleSpec, d_grain: np.ndarray, U: float = 0.01) -> Sample:
    """Pack one ensemble member with the given grain diameters.  Periodic
    members: cube at solid fraction 0.55, 8 fluid cells per side.  Cylinder
    members: a cylinder of height 0.75 Rc whose bed (0.7 of the height,
    around the central cavity) holds the grains at solid fraction 0.55,
    outlet 3 grain d50, fluid cells of two grain d50 (the grain d50 is k
    times the fine d50)."""
    mat = dict(rho=2650.0, E=1e8, nu=0.3, e=0.5, mu=0.5, gamma=spec.gamma)
    if spec.kind == 0:
        return periodic_sample(d_grain, 0.55, spec.seed, nf=8, U=(0.0, 0.0, U), material=mat,
                               name=f"ens{spec.index}-periodic")
    R = 0.5 * np.asarray(d_grain)
    Vs = float((4.0 / 3.0 * math.pi * R ** 3).sum())
    d50 = spec.d50 * spec.k
    r_out = 3.0 * d50
    # cylinder of aspect H = 0.75 Rc whose bed (0.7 H, outside the central
    # cavity of radius r_out) holds Vs at solid fraction 0.55:
    # Vs = 0.55 pi (Rc^2 - r_out^2) 0.525 Rc, solved by bisection
    a, b = r_out, r_out + (Vs / (0.55 * math.pi * 0.525)) ** (1.0 / 3.0) + r_out
    for _ in range(200):
        m = 0.5 * (a + b)
        if 0.55 * math.pi * (m * m - r_out * r_out) * 0.525 * m < Vs:
            a = m
        else:
            b = m
    Rc = 0.5 * (a + b)
    scale = Rc / (40.0 * d50)
    nf = (max(4, int(round(40 * scale))), max(4, int(round(40 * scale))), max(2, int(round(20 * scale))))
    return cylinder_sample(d_grain, spec.seed, d50=d50, scale=scale, nf=nf, U_in=U, material=mat,
                           name=f"ens{spec.index}-cylinder")


def _pack_job(args):
    spec, d_grain, U = args
    return pack_member(spec, d_grain, U)


def pack_ensemble(specs, grain_diameters, U: float = 0.01, workers: int = 0):
    """Pack every member (in parallel worker processes started with spawn)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    jobs = [(s, d, U) for s, d in zip(specs, grain_diameters)]
    w = workers or min(len(jobs), os.cpu_count() or 1)
    if w <= 1:
        return [_pack_job(j) for j in jobs]
    with cf.ProcessPoolExecutor(max_workers=w, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_pack_job, jobs))

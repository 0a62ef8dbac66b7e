"""Workloads of the library: the seeded inputs of ``inputs.py`` turned into
grain-level samples with the library's own coarse-graining rule
(``cgdem_cg_scale_diameters``, Sec. 2.4) and packed.

* ``fine_cylinder``: 200k-sphere sand-production cylinder (k = 1).
* ``coarse_cylinder``: the same sand at ratio k under SSW or SSP
  (N_g = N_p / k^3, gamma_g = k gamma), same domain and fluid grid.
* ``coarse_tiled_cylinder``: the 2M-sphere tiled cylinder's coarse
  counterpart at ratio k (about 74k SSW parcels at k = 3), same domain,
  bed height and fluid grid.
* ``ensemble``: a calibration sweep of many independent samples of uneven
  size, PSD, cohesion, coarse-graining ratio and domain kind.
"""
from __future__ import annotations

import numpy as np

from . import cgdem
from . import inputs as I

SCHEME = {"none": cgdem.CG_NONE, "ssw": cgdem.CG_SSW, "ssp": cgdem.CG_SSP}


def _ensemble(n_samples, seed):
    specs = I.ensemble_specs(n_samples, seed)
    grains = [cgdem.cgdem_cg_scale_diameters(s.d_fine, s.k, cgdem.CG_SSW) for s in specs]
    return specs, I.pack_ensemble(specs, grains)


def ensemble(n_samples: int = 64, seed: int = 3):
    """(specs, samples) of the batched ensemble, memoised on disk."""
    return I.cached(_ensemble, n_samples, seed)


def ensemble_params(specs, samples, skin_frac=0.02, dt_frac=0.2):
    """Per-member library parameters: fine-scale material, ratio k, SSW,
    dt = dt_frac x Rayleigh step of the grains' volume-mean radius."""
    params = []
    for sp, s in zip(specs, samples):
        m = s.material
        Rbar = float(np.mean(s.R ** 3)) ** (1 / 3)
        dt = dt_frac * cgdem.cgdem_rayleigh_dt(Rbar, m["rho"], m["E"], m["nu"])
        skin = skin_frac * 2 * float(s.R.max())
        params.append(cgdem.sample_params(s, dt, skin, k=sp.k, scheme=cgdem.CG_SSW if sp.k > 1 else cgdem.CG_NONE))
    return params


def _coarse_cylinder(n_fine, seed, k, scheme, U_in):
    d_fine = I.fine_diameters(n_fine, seed)
    d_g = cgdem.cgdem_cg_scale_diameters(d_fine, k, SCHEME[scheme])
    return I.cylinder_sample(d_g, seed, U_in=U_in, name=f"cylinder-{scheme}-k{k}")


def coarse_cylinder(n_fine: int = 200_000, seed: int = 1, k: int = 2, scheme: str = "ssw",
                    U_in: float = 1e-4):
    """The sand-production cylinder coarse-grained at ratio k (SSW or SSP)."""
    return I.cached(_coarse_cylinder, n_fine, seed, k, scheme, U_in)


def _coarse_tiled_cylinder(n_fine, scale, seed, k, scheme):
    h_bed = I.tiled_bed_height(n_fine, scale, seed)
    return I.tiled_cylinder(n_fine, scale, seed, d_map=lambda d: cgdem.cgdem_cg_scale_diameters(d, k, SCHEME[scheme]),
                            h_bed=h_bed, name=f"cylinder-tiled-{scheme}-k{k}")


def coarse_tiled_cylinder(n_fine: int = 2_000_000, scale: float = 2.15, seed: int = 4, k: int = 3,
                          scheme: str = "ssw"):
    """The tiled cylinder of n_fine spheres (``inputs.tiled_cylinder``) coarse-
    grained at ratio k: its periodic block's grains mapped by the rule (N/k^3
    parcels under SSW), tiled over the same bed height."""
    return I.cached(_coarse_tiled_cylinder, n_fine, scale, seed, k, scheme)

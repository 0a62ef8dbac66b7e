"""What the trained closure gains over plain coarse-graining.

A fine sand-production cylinder (16,000 grains) and its SSW coarse model at
k = 2 (2,000 parcels) run on the GPU over the same physical time with the
same domain, fluid grid and radial inflow.  The closure network is trained
(tensor-core kernels) on the coarse parcels' recorded inputs against the
per-cell drag and bond-capacity ratios of the two runs, then the coarse run
is repeated with the closure fused into its force kernel.  The gain: the
per-cell drag of the coarse model, measured against the fine model, is at
least twice as close with the closure as without it (mean |ln D_coarse /
D_fine| over cells and times).  Plain SSW keeps drag per grain of k times the
diameter, so its per-cell drag misses the fine one by a factor the closure
learns from the inputs.
"""
import numpy as np
import pytest

from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import closure as CL
from paper_2211_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu

K = 2
SCALE, NF, U_IN, SEED = 0.45, (18, 18, 9), 0.05, 31


def samples():
    d = I.fine_diameters(16000, SEED)
    fine = I.cylinder_sample(d, SEED, scale=SCALE, nf=NF, U_in=U_IN, name="gain-fine")
    dg = cgdem.cgdem_cg_scale_diameters(d, K, cgdem.CG_SSW)
    coarse = I.cylinder_sample(dg, SEED, scale=SCALE, nf=NF, U_in=U_IN, name="gain-coarse")
    return fine, coarse


def dt_of(s):
    m = s.material
    Rbar = float(np.mean(s.R ** 3)) ** (1 / 3)
    return 0.2 * cgdem.cgdem_rayleigh_dt(Rbar, m["rho"], m["E"], m["nu"])


def test_closure_halves_the_cell_drag_error():
    fine, coarse = samples()
    assert abs(fine.domain["Rc"] - coarse.domain["Rc"]) < 1e-15
    dtf, dtc = dt_of(fine), dt_of(coarse)
    times = [dtc * 40 * (w + 1) for w in range(8)]
    skin_f = 0.06 * 2 * float(fine.R.max())
    skin_c = 0.06 * 2 * float(coarse.R.max())
    fr = CL.record_run(CL.make_context(fine, dtf, skin_f, 1), fine, dtf, times)
    cr = CL.record_run(CL.make_context(coarse, dtc, skin_c, K), coarse, dtc, times)
    X, Y, M = CL.targets(fr, cr)
    assert len(X) > 8000 and M[:, 0].mean() > 0.5
    theta, hist = CL.fit(X, Y, M, steps=1000, lr=3e-3)
    assert hist[-1] < hist[0]
    lo, hi = CL.input_range(X)
    cc = CL.record_run(CL.make_context(coarse, dtc, skin_c, K), coarse, dtc, times,
                       closure=(theta, lo, hi, 3.0, np.log(4.0)))
    e_plain = CL.cell_drag_error(fr, cr)
    e_closure = CL.cell_drag_error(fr, cc)
    print(f"cell drag error: plain SSW {e_plain:.4f}, closure {e_closure:.4f}; "
          f"bond capacity: plain {CL.cell_bond_error(fr, cr):.4f}, closure {CL.cell_bond_error(fr, cc):.4f}")
    assert e_plain > 0.05
    assert e_closure < 0.5 * e_plain

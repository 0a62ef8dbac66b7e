"""What the trained closure gains over plain coarse-graining.

A fine sand-production cylinder (16,000 grains) and its SSW coarse model at
k = 2 (2,000 parcels) run on the GPU over the same physical time with the
same domain, fluid grid and radial inflow.  The closure network is trained
(tensor-core kernels) on the coarse parcels' recorded inputs against the
drag and bond-capacity ratios of the two runs over blocks of 2 x 2 x 2 fluid
cells, then the coarse run is repeated with the closure fused into its force
kernel.  The gain, measured against the fine model at the recorded times:
the drag the whole bed exerts on the fluid (sum over cells of the drag
magnitude) is at least twice as close with the closure as without it, and
the per-block drag and bond-capacity errors shrink.  Plain SSW keeps the
drag of a grain k times the diameter at the coarse porosity, so the bed's
drag misses the fine one by a factor the closure learns from the inputs.
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
    X, Y, M = CL.targets(fr, cr, merge=2)
    assert len(X) > 8000 and M[:, 0].mean() > 0.5
    theta, hist = CL.fit(X, Y, M, steps=1000, lr=3e-3)
    assert hist[-1] < hist[0]
    lo, hi = CL.input_range(X)
    cc = CL.record_run(CL.make_context(coarse, dtc, skin_c, K), coarse, dtc, times,
                       closure=(theta, lo, hi, 3.0, np.log(4.0)))
    t_plain, t_closure = CL.total_drag_error(fr, cr), CL.total_drag_error(fr, cc)
    d_plain, d_closure = CL.cell_drag_error(fr, cr, merge=2), CL.cell_drag_error(fr, cc, merge=2)
    b_plain, b_closure = CL.cell_bond_error(fr, cr, merge=2), CL.cell_bond_error(fr, cc, merge=2)
    print(f"|ln bed drag ratio|: plain SSW {t_plain:.3f}, closure {t_closure:.3f}; "
          f"per block drag: {d_plain:.3f} -> {d_closure:.3f}; bond capacity: {b_plain:.3f} -> {b_closure:.3f}")
    assert t_plain > 0.1
    assert t_closure < 0.5 * t_plain
    assert d_closure < d_plain and b_closure < b_plain

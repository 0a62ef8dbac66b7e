"""Host-side logic around the library (no GPU): the produced-sand error of
Eq. 41, the closure's per-block targets and errors, the autotuner's
parameter handling."""
import math

import numpy as np
import pytest

from paper_2211_06142_gb300 import autotune as A
from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import closure as CL
from paper_2211_06142_gb300 import sand as SD


def prod(mass):
    m = np.asarray(mass, float)
    return SD.Production(np.arange(1, len(m) + 1) * 1e-3, m, 10)


def test_rmsre_reads_eq41_as_root_mean_square():
    ref, mod = prod([0.0, 1.0, 2.0, 4.0]), prod([0.5, 1.0, 1.0, 4.0])
    # times where the reference produced: relative errors 0, 0.5, 0
    assert SD.rmsre(ref, mod) == pytest.approx(100 * math.sqrt(0.25 / 3), rel=1e-12)
    assert SD.final_error(ref, mod) == 0.0
    assert SD.rmsre(prod([0, 0]), mod) is None
    # late: only the times where the reference reached 30 % of its final mass (2.0, 4.0)
    assert SD.rmsre_late(ref, mod, 0.3) == pytest.approx(100 * math.sqrt(0.25 / 2), rel=1e-12)
    assert SD.rmsre_late(ref, mod, 0.9) == 0.0


def rows(cells, drag, cap):
    """Recorded closure rows: active particles with k = 1 in the given cells."""
    n = len(cells)
    r = np.zeros((n, cgdem.CL_COLS), np.float32)
    r[:, 2] = 1.0
    r[:, CL.COL_CELL] = cells
    r[:, 5:8] = drag
    r[:, CL.COL_CAP] = cap
    return r


def test_block_sums_and_targets():
    nf = (4, 4, 2)
    # fine: two particles per cell 0 and 5, coarse: one parcel with half the drag
    fr = rows([0, 0, 5, 5], [[1, 0, 0]] * 4, [1.0] * 4)
    cr = rows([0, 5, 5, 17], [[1, 0, 0], [0.5, 0, 0], [0.5, 0, 0], [3, 0, 0]], [1.0, 0.5, 0.5, 0.0])
    fine = CL.Run([fr], [0.0], [0.0], nf)
    coarse = CL.Run([cr], [0.0], [0.0], nf)
    D, B, n = CL.cell_sums(fr, nf, merge=1)
    assert D[0] == 2.0 and D[5] == 2.0 and n[0] == 2 and B[5] == 2.0
    # blocks of 2x2x2 cells: cells 0 and 5 share block 0; cell 17 (x1 y0 z1) too
    D2, B2, n2 = CL.cell_sums(cr, nf, merge=2)
    assert n2[0] == 4 and D2[0] == pytest.approx(5.0) and len(D2) == 4
    X, Y, M = CL.targets(fine, coarse, min_parcels=1, merge=1)
    assert X.shape == (4, 5) and Y.shape == (4, 2)
    # cell 0: D 2 vs 1, B 2 vs 1; cell 5: D 2 vs 1, B 2 vs 1; cell 17: no fine drag
    assert Y[0] == pytest.approx([math.log(2), math.log(2)])
    assert Y[1] == pytest.approx([math.log(2), math.log(2)]) and Y[2] == pytest.approx(Y[1])
    assert M[3].tolist() == [0.0, 0.0] and M[:3].all()
    assert CL.cell_drag_error(fine, coarse, min_parcels=1) == pytest.approx(math.log(2))
    assert CL.total_drag_error(fine, coarse) == pytest.approx(abs(math.log(5.0 / 4.0)))


def test_standardisation_and_range():
    X = np.array([[0.2, 1.0, 2.0], [0.4, 3.0, 2.0]])
    mu, isg = CL.standardisation(X)
    assert mu == pytest.approx([0.3, 2.0, 2.0]) and isg == pytest.approx([10.0, 1.0, 1.0])
    lo, hi = CL.input_range(X, margin=0.5)
    assert lo[0] == pytest.approx(0.1) and hi[1] == pytest.approx(4.0)
    th = CL.init_theta(np.zeros(5), np.ones(5), 0, out_bias=(0.5, -0.25))
    assert th.shape == (cgdem.MLP_NPARAMS,) and th[-2] == 0.5 and th[-1] == -0.25


def test_autotune_skin_copy_keeps_the_rest():
    p = cgdem.SampleParams()
    p.r_max = 2e-4
    p.skin = 1e-6
    p.L[0] = 3e-3
    p.nf[1] = 7
    q = A._with_skin([p], 0.05)[0]
    assert q.skin == pytest.approx(0.05 * 2 * 2e-4)
    assert q.L[0] == 3e-3 and q.nf[1] == 7 and p.skin == 1e-6
    assert A.signature([p], [10], 1) == A.signature([q], [10], 1)
    assert A.signature([p], [10], 1) != A.signature([p], [11], 1)


def test_autotune_search_and_confirmation(monkeypatch, tmp_path):
    """Coordinate search over the knobs with a fake timing: the best setting
    wins, a noisy short trial is corrected by the longer confirmation runs,
    and the result is cached by workload signature."""
    monkeypatch.setenv("CGDEM_CACHE", str(tmp_path))
    calls = []

    def fake_trial(params, counts, state, Us, precision, cs, block, steps=600, device=None, ppw=32, **kw):
        calls.append((cs, block, round(params[0].skin / (2 * params[0].r_max), 6), ppw, steps))
        ms = 1.0 + abs(cs - 0.5) + 0.1 * abs(block - 128) / 128 + abs(params[0].skin / (2 * params[0].r_max) - 0.04)
        ms += 0.01 * (ppw == 16)
        if steps == 600 and (cs, block, ppw) == (0.75, 128, 32) and abs(params[0].skin - 0.02 * 2e-4) < 1e-12:
            ms -= 0.3  # one short trial that happened to run fast
        return ms

    monkeypatch.setattr(A, "trial", fake_trial)
    p = cgdem.SampleParams()
    p.r_max = 1e-4
    res = A.autotune([p], [100], None, None, cgdem.MIXED)
    # the noisy trial misleads the cell sweep (0.75 kept, so the skin sweep
    # runs there); the confirmation runs put the runner-up (0.5) back
    assert (res["cell_scale"], res["block"], res["skin_frac"], res["ppw"]) == (0.5, 128, 0.02, 32)
    assert not res["cached"] and any(c[4] == 1200 for c in calls)
    n = len(calls)
    again = A.autotune([p], [100], None, None, cgdem.MIXED)
    assert again["cached"] and len(calls) == n and again["cell_scale"] == 0.5


def test_skin_factors_follow_drift_rates():
    """Members drifting faster than the ensemble's upper quartile get a skin
    scaled by their rate over it, capped; the rest keep theirs."""
    rates = [1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 2.0, 3.0, 10.0]
    f = A.skin_factors(rates, quantile=0.75, max_factor=2.5)
    ref = float(np.quantile(rates, 0.75))
    assert f[:7].tolist() == [1.0] * 7
    assert f[7] == pytest.approx(max(1.0, 2.0 / ref)) and f[8] == pytest.approx(min(2.5, 3.0 / ref))
    assert f[9] == 2.5
    assert A.skin_factors([0.0, 0.0]).tolist() == [1.0, 1.0]
    assert len(A.skin_factors([])) == 0


def test_normalised_sand_curves_and_windows():
    """Eq. 39-41 on made-up production records: M_d ends at 1, a curve has
    no error against itself and against a scaled copy (normalisation), and
    the per-window class masses add up to the final cumulative ones."""
    from paper_2211_06142_gb300 import sand as SD
    t = np.linspace(0.1, 4.0, 40) * 1e-3
    m = 1e-6 * (1 - np.exp(-t / 1e-3))
    psd = np.outer(m, np.linspace(1, 2, 8)) / 12.0
    a = SD.Production(t, m, 100, psd=psd)
    b = SD.Production(t, 2 * m, 100, psd=2 * psd)
    td, md = SD.normalized_curve(a)
    assert td[-1] == 1.0 and md[-1] == 1.0 and np.all(np.diff(md) > 0)
    assert SD.rmsre_normalized(a, a) == 0.0
    assert SD.rmsre_normalized(a, b) == pytest.approx(0.0, abs=1e-12)
    c = SD.Production(t, m * (1 + 0.1 * (t < 1e-3)), 100, psd=psd)
    assert SD.rmsre_normalized(a, c) > 0
    w = SD.psd_windows(a)
    assert w.shape == (3, 8)
    np.testing.assert_allclose(w.sum(0), psd[-1], rtol=1e-14)
    e = SD.table2_edges()
    assert len(e) == 9 and np.all(np.diff(e) > 0)

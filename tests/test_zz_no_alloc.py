"""The allocation-free pair search.

cgdem_touching_pairs_noalloc serves callers that cannot allocate device
memory (a fixed memory pool owned by the host application, or a loop that
must not stall on an allocation).  Its scratch is a fixed array inside the
library, reused by every call.  Checked here against the library's own
contact list and against the oracle's O(N^2) brute-force search (the same
IEEE operations, so the pair sets must be identical), with and without a
skin, across the one-block scan's 1024-cell chunks, with a periodic axis two
cells wide, with a box an exact multiple of the cell edge, and with more
pairs than the output holds.  This file runs last so that, if it fails, a
run stopping at the first failure has already run every other test; it also
passes when run on its own in a fresh process.
"""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import default_dt, default_skin, small_cylinder

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_limit(name):
    """A #define of include/cgdem.h (the limits the library was built with)."""
    with open(os.path.join(ROOT, "include", "cgdem.h")) as f:
        m = re.search(r"#define\s+%s\s+(\d+)" % name, f.read())
    return int(m.group(1))


def reference_pairs(s):
    """Touching pairs from the context API: unbonded, so the active contacts
    after one force evaluation are exactly the pairs with d^2 < (Ri+Rj)^2."""
    p = cgdem.sample_params(s, default_dt(s), default_skin(s))
    ctx = cgdem.Context([p], [len(s.R)], precision=cgdem.FP64, max_neighbors=64)
    ctx.set_fluid_velocity(s.Us)
    ctx.init_particles(s.x, s.v, s.w, s.R, bond_touching=False)
    ctx.compute_forces()
    i, j, b = ctx.get_contacts()
    ctx.close()
    assert not b.any()
    return set(zip(i.tolist(), j.tolist()))


def oracle_pairs(x, R, skin, periodic, L=None):
    p = O.make_params(kind=0 if periodic else 1, L=tuple(L) if periodic else (0.0, 0.0, 0.0))
    pi, pj = O.pairs_bruteforce(p, x, R, skin)
    return set(zip(pi.tolist(), pj.tolist()))


def noalloc_call(x, R, lo, hi, periodic, r_max, skin, cap, guard=0):
    """One call on device copies of x, R; returns (pairs found, count, the
    guard entries after pairs[cap])."""
    import torch

    dev = torch.device("cuda:0")
    xd = torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev).contiguous()
    Rd = torch.tensor(np.ascontiguousarray(R), dtype=torch.float64, device=dev).contiguous()
    out = torch.full((cap + guard, 2), -1, dtype=torch.int32, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    cgdem.cgdem_touching_pairs_noalloc(xd.data_ptr(), Rd.data_ptr(), len(R), lo, hi, periodic,
                                       float(r_max), float(skin), out.data_ptr(), cap,
                                       count.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    n = int(count.item())
    pr = out[:min(n, cap)].cpu().numpy()
    assert (pr[:, 0] < pr[:, 1]).all()
    got = set(map(tuple, pr.tolist()))
    assert len(got) == len(pr)  # no pair written twice
    return got, n, out[cap:].cpu().numpy()


def sample_box(s, periodic):
    if periodic:
        return np.zeros(3), np.array(s.domain["L"], dtype=np.float64)
    return s.x.min(0) - 1e-9, s.x.max(0) + 1e-9


@pytest.mark.parametrize("kind", ["periodic", "cylinder"])
def test_noalloc_pairs_match_contact_list_twice(kind):
    s = I.cached(I.small_periodic, 2000, 0) if kind == "periodic" else small_cylinder()
    ref = reference_pairs(s)
    assert len(ref) > len(s.R) // 2
    lo, hi = sample_box(s, kind == "periodic")
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        got, n, _ = noalloc_call(s.x, s.R, lo, hi, kind == "periodic", s.R.max(), 0.0, 20 * len(s.R))
        assert n == len(ref)
        assert got == ref


def test_noalloc_with_skin_across_scan_chunks_against_bruteforce():
    """6000 spheres scattered in a box of more than 1024 search cells (the
    scan carries its sum from one 1024-cell chunk to the next), a skin of
    half the mean diameter: identical to the oracle's brute force."""
    rng = np.random.default_rng(11)
    R = 0.5 * I.fine_diameters(6000, 5)
    skin = 0.5 * float(R.mean()) * 2
    h = 2 * R.max() + skin
    hi = np.array([14.3, 11.7, 9.2]) * h
    x = rng.uniform(0, 1, size=(len(R), 3)) * hi
    ref = oracle_pairs(x, R, skin, False)
    lo, top = np.zeros(3), hi
    assert np.prod(np.floor(hi / h)) > 1024
    for _ in range(2):
        got, n, _ = noalloc_call(x, R, lo, top, 0, R.max(), skin, 40 * len(R))
        assert n == len(ref) and got == ref


def test_noalloc_periodic_axis_two_cells_wide_against_bruteforce():
    """A periodic box 2.5 cells wide in x (every cell of that axis is in the
    stencil, once) and 7 cells in y, z, with a skin."""
    R = 0.5 * I.fine_diameters(3000, 6)
    skin = 0.3 * float(R.max())
    h = 2 * R.max() + skin
    L = np.array([2.5, 7.2, 7.6]) * h
    x = np.random.default_rng(12).uniform(0, 1, size=(len(R), 3)) * L
    ref = oracle_pairs(x, R, skin, True, L)
    got, n, _ = noalloc_call(x, R, np.zeros(3), L, 1, R.max(), skin, 60 * len(R))
    assert n == len(ref) and got == ref
    assert any(abs(x[i, 0] - x[j, 0]) > 0.5 * L[0] for i, j in ref)  # pairs across the wrap


def test_noalloc_box_exact_multiple_of_the_cell_edge():
    """Equal spheres (so the cell edge is 2 R + skin) whose box is exactly 12
    cell edges, with chains of spheres spaced just inside the reach along each
    axis, across every cell face: every such pair is found."""
    r = 1e-4
    skin = 2e-5
    h = 2 * r + skin
    L = 12 * h
    rng = np.random.default_rng(13)
    xs = []
    for axis in range(3):
        for c in range(4):
            p = rng.uniform(0.1, 0.9, 3) * L
            t = np.arange(11) * (h * (1 - 1e-13))
            q = np.tile(p, (11, 1))
            q[:, axis] = 1e-7 + t
            xs.append(q)
    x = np.concatenate(xs + [rng.uniform(0, L, size=(400, 3))])
    R = np.full(len(x), r)
    ref = oracle_pairs(x, R, skin, False)
    assert len(ref) >= 12 * 10
    got, n, _ = noalloc_call(x, R, np.zeros(3), np.full(3, L), 0, r, skin, 40 * len(x))
    assert n == len(ref) and got == ref


def test_noalloc_counts_pairs_beyond_cap_without_writing_them():
    s = I.cached(I.small_periodic, 2000, 0)
    ref = oracle_pairs(s.x, s.R, 0.0, True, s.domain["L"])
    cap = len(ref) // 3
    lo, hi = sample_box(s, True)
    got, n, tail = noalloc_call(s.x, s.R, lo, hi, 1, s.R.max(), 0.0, cap, guard=64)
    assert n == len(ref) and n > cap
    assert len(got) == cap and got <= ref
    assert (tail == -1).all()


def test_noalloc_rejects_sizes_beyond_the_limit():
    limit = header_limit("CGDEM_NOALLOC_MAX_SPHERES")
    with pytest.raises(cgdem.CgdemError) as e:
        cgdem.cgdem_touching_pairs_noalloc(1, 1, limit + 1, np.zeros(3), np.ones(3), 0, 0.1,
                                           0.0, 1, 1, 1, None)
    assert e.value.code == cgdem.CGDEM_E_CAPACITY
    cells = header_limit("CGDEM_NOALLOC_MAX_CELLS")
    # a grid of more cells than the scratch holds
    side = float(np.ceil(cells ** (1 / 3)) + 2)
    with pytest.raises(cgdem.CgdemError) as e:
        cgdem.cgdem_touching_pairs_noalloc(1, 1, 10, np.zeros(3), np.full(3, side), 0, 0.5,
                                           0.0, 1, 1, 1, None)
    assert e.value.code == cgdem.CGDEM_E_CAPACITY

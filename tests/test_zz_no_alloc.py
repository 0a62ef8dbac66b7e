"""The allocation-free pair search against the library's contact list.

cgdem_touching_pairs_noalloc serves callers that cannot allocate device
memory (a fixed memory pool owned by the host application, or a loop that
must not stall on an allocation).  Its scratch is a fixed array inside the
library, reused by every call.  This file runs last so that, if it fails, a
run stopping at the first failure has already run every other test; it also
passes when run on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2211_06142_gb300 import cgdem
from paper_2211_06142_gb300 import inputs as I
from tests.helpers import default_dt, default_skin, small_cylinder

pytestmark = pytest.mark.gpu


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


def noalloc_pairs(s, periodic):
    import torch

    dev = torch.device("cuda:0")
    x = torch.tensor(s.x, dtype=torch.float64, device=dev).contiguous()
    R = torch.tensor(s.R, dtype=torch.float64, device=dev).contiguous()
    cap = 20 * len(s.R)
    pairs = torch.full((cap, 2), -1, dtype=torch.int32, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    if periodic:
        lo, hi = np.zeros(3), np.array(s.domain["L"], dtype=np.float64)
    else:
        lo = s.x.min(0) - 1e-9
        hi = s.x.max(0) + 1e-9
    stream = torch.cuda.current_stream(dev).cuda_stream
    cgdem.cgdem_touching_pairs_noalloc(x.data_ptr(), R.data_ptr(), len(s.R), lo, hi, periodic,
                                       float(s.R.max()), 0.0, pairs.data_ptr(), cap,
                                       count.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    n = int(count.item())
    assert n <= cap
    pr = pairs[:n].cpu().numpy()
    assert (pr[:, 0] < pr[:, 1]).all()
    return set(map(tuple, pr.tolist())), n


@pytest.mark.parametrize("kind", ["periodic", "cylinder"])
def test_noalloc_pairs_match_contact_list_twice(kind):
    s = I.cached(I.small_periodic, 2000, 0) if kind == "periodic" else small_cylinder()
    ref = reference_pairs(s)
    assert len(ref) > len(s.R) // 2
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        got, n = noalloc_pairs(s, kind == "periodic")
        assert n == len(ref)
        assert got == ref


def test_noalloc_rejects_sizes_beyond_the_limit():
    with pytest.raises(cgdem.CgdemError) as e:
        cgdem.cgdem_touching_pairs_noalloc(1, 1, cgdem_limit() + 1, np.zeros(3), np.ones(3), 0, 0.1,
                                           0.0, 1, 1, 1, None)
    assert e.value.code == cgdem.CGDEM_E_CAPACITY


def cgdem_limit():
    return 262144

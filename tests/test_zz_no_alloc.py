"""The allocation-free critical-step entry point against pd_stable_dt.

It serves callers that cannot allocate device memory when they need the step
(a frozen memory pool, a runtime that owns all device memory, a host callback).
Kept in a file that pytest collects last; it must pass alone in a fresh process
as well as after the other tests."""
import numpy as np
import pytest

import oracle
from paper_2506_05362_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


def test_noalloc_stable_dt_matches_context_twice():
    import torch
    from paper_2506_05362_gb300 import pd
    assert torch.cuda.is_available()
    sc = S.sphere()
    ctx = pd.Context.from_scenario(sc, contact=False)
    ref = ctx.stable_dt()
    rp, col = ctx.bonds()
    K, c, s0, Kn = oracle.constants(sc.material.E, sc.material.G0, sc.horizon, sc.material.contact_factor)
    dev = torch.device("cuda", 0)
    x = torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev)
    vol = torch.from_numpy(np.ascontiguousarray(sc.vol)).to(dev)
    rowptr = torch.from_numpy(rp).to(dev)
    colt = torch.from_numpy(col).to(dev)
    out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    for call in range(2):  # two calls in a row share the scratch array
        st = pd.pd_stable_dt_noalloc(sc.n, x.data_ptr(), vol.data_ptr(), rowptr.data_ptr(), colt.data_ptr(),
                                     c, sc.material.rho, stream.cuda_stream, out[call:].data_ptr())
        assert st == pd.PD_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    # same terms, summed in caller instead of internal column order
    assert got[0] == pytest.approx(ref, rel=1e-12)
    assert got[1] == got[0]
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    from paper_2506_05362_gb300 import pd
    dev = torch.device("cuda", 0)
    dummy = torch.zeros(4, dtype=torch.float64, device=dev)
    st = pd.pd_stable_dt_noalloc(16_777_217, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                 dummy.data_ptr(), 1.0, 1.0, 0, dummy.data_ptr())
    assert st == pd.PD_EINVAL

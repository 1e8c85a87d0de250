"""The allocation-free critical-step entry point against pd_stable_dt and the oracle.

It serves callers that cannot allocate device memory when they need the step
(a frozen memory pool, a runtime that owns all device memory, a host callback).
Kept in a file that pytest collects last; it must pass alone in a fresh process
as well as after the other tests."""
import numpy as np
import pytest

import oracle
from paper_2506_05362_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


def _device_inputs(sc, rp, col):
    import torch
    dev = torch.device("cuda", 0)
    return (torch.from_numpy(np.ascontiguousarray(sc.x)).to(dev),
            torch.from_numpy(np.ascontiguousarray(sc.vol)).to(dev),
            torch.from_numpy(np.ascontiguousarray(rp, np.int64)).to(dev),
            torch.from_numpy(np.ascontiguousarray(col, np.int32)).to(dev))


def _two_calls(pd, n, x, vol, rowptr, col, c, rho):
    """Two calls in a row on the current stream, into two device doubles."""
    import torch
    dev = torch.device("cuda", 0)
    out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    for call in range(2):  # the calls share the scratch array
        st = pd.pd_stable_dt_noalloc(n, x.data_ptr(), vol.data_ptr(), rowptr.data_ptr(), col.data_ptr(),
                                     c, rho, stream.cuda_stream, out[call:].data_ptr())
        assert st == pd.PD_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name", ["sphere", "kalthoff"])
def test_noalloc_stable_dt_matches_context_and_oracle_twice(name):
    """The sphere (4,139 nodes, 17 partial blocks) and the full notched plate
    (178,200 nodes, 697 partial blocks, so the final reduction strides over more
    partials than it has threads): the step from the oracle's bond lists against
    the context's pd_stable_dt and the oracle's own bound, on two calls in a row."""
    import torch
    from paper_2506_05362_gb300 import pd
    assert torch.cuda.is_available()
    sc = S.BY_NAME[name]()
    kinds, params = S.filters_array(sc.filters)
    rp, col = oracle.bonds(sc.x, sc.grain, sc.horizon, kinds, params)
    model = oracle.Model(sc.x, sc.vol, sc.grain, rp, col, sc.material, sc.horizon)
    want = model.stable_dt()
    ctx = pd.Context.from_scenario(sc, contact=False)
    ctx_dt = ctx.stable_dt()
    ctx.close()
    x, vol, rowptr, colt = _device_inputs(sc, rp, col)
    got = _two_calls(pd, sc.n, x, vol, rowptr, colt, model.c, sc.material.rho)
    # same terms, summed in caller order on both sides but with other roundings
    assert got[0] == pytest.approx(want, rel=1e-12)
    assert got[0] == pytest.approx(ctx_dt, rel=1e-12)
    assert got[1] == got[0]


def test_noalloc_without_bonds_gives_infinity():
    """Rows without bonds do not bound the step: all-zero row pointers give inf."""
    import torch
    from paper_2506_05362_gb300 import pd
    sc = S.small_block()
    rp = np.zeros(sc.n + 1, np.int64)
    col = np.zeros(1, np.int32)
    x, vol, rowptr, colt = _device_inputs(sc, rp, col)
    got = _two_calls(pd, sc.n, x, vol, rowptr, colt, 1.0, sc.material.rho)
    assert np.all(np.isinf(got)) and np.all(got > 0)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    from paper_2506_05362_gb300 import pd
    dev = torch.device("cuda", 0)
    dummy = torch.zeros(4, dtype=torch.float64, device=dev)
    st = pd.pd_stable_dt_noalloc(16_777_217, dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(),
                                 dummy.data_ptr(), 1.0, 1.0, 0, dummy.data_ptr())
    assert st == pd.PD_EINVAL

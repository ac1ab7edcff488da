"""The allocation-free encode entry point (vsaogm_encode_bundle_noalloc).

Some callers cannot call cudaMalloc: a real-time control loop, where an
allocation can synchronise the device and stall it, or a process whose device
memory belongs to another allocator.  For them the library offers an encode
call whose scratch is a static device array.  This test calls it through the C
ABI twice in a row on the same map and checks the memories after each call
against the regular (allocating) entry point, within the memory tolerance the
other parity tests use.  It is kept in a file of its own, collected last.
"""
import numpy as np
import pytest

from helpers import config_for, normwise
from paper_2408_09066_gb300 import synth
from paper_2408_09066_gb300 import vsaogm as V

pytestmark = pytest.mark.gpu

TOL_OMEGA = 3e-5  # as in test_gpu_parity.py


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


@pytest.mark.parametrize("D", [1024, 8192])
def test_noalloc_matches_regular_entry_point_on_two_calls(D):
    import torch
    wl = synth.small_scan(seed=4242, D=D)
    more = synth.small_scan(seed=4243, D=D)
    cfg = config_for(wl, tiles_x=2, tiles_y=2)
    dev = torch.device("cuda")
    batches = [(torch.from_numpy(w.xy).to(dev), torch.from_numpy(w.labels).to(dev))
               for w in (wl, more)]
    with V.Map(cfg) as ref, V.Map(cfg) as na:
        for xy, lab in batches:
            ref.encode_bundle(xy, lab)
            V._check(V.lib().vsaogm_encode_bundle_noalloc(
                na.handle, V._V(xy.data_ptr()), V._V(lab.data_ptr()), lab.shape[0],
                V._V(torch.cuda.current_stream().cuda_stream)))
            a, b = ref.get_memory(), na.get_memory()
            torch.cuda.synchronize()
            assert normwise(b.cpu().numpy(), a.cpu().numpy()) <= TOL_OMEGA
        assert ref.rejected() == na.rejected() == 0


def test_noalloc_rejects_more_points_than_its_scratch_holds():
    import torch
    wl = synth.small_scan(seed=1)
    cfg = config_for(wl)
    n = (1 << 18) + 1
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    lab = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with V.Map(cfg) as m:
        with pytest.raises(V.VsaogmError) as ei:
            m.encode_bundle_noalloc(xy, lab)
        assert ei.value.code == V.E_INVAL and "maximum" in str(ei.value)
        m.encode_bundle_noalloc(xy[:0], lab[:0])  # n = 0 is a no-op
        assert torch.count_nonzero(m.get_memory()).item() == 0

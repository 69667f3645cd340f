"""pxst_make_object_map_noalloc, the entry point for callers that cannot allocate device
memory (a plug-in inside a host framework that owns the GPU's memory, a real-time loop
that cannot take cudaMalloc's synchronisation): called through the C ABI, its output must
match pxst_make_object_map's (which uses a caller-allocated workspace) within the
reference-image tolerance of the other tests, on two calls in a row, so that the second
call cannot see what the first left in the shared fixed scratch. This file is collected
last on purpose."""
import numpy as np
import pytest

import gen
import parity

pytestmark = pytest.mark.gpu


def _both(s):
    import torch
    import paper_2003_12726_gb300 as px
    from gpu_util import dev, dims_of
    d = dims_of(s.frames, s.ref_shape)
    args = (dev(s.frames, torch.float32), dev(s.W, torch.float32), dev(s.M, torch.uint8),
            dev(s.u_init, torch.float64), dev(s.delta, torch.float64))
    Ia = torch.empty(s.ref_shape, dtype=torch.float32, device="cuda")
    wa = torch.empty_like(Ia)
    ws = px.workspace(d)
    px.make_object_map(d, *args, Ia, wa, ws)
    Ib = torch.full(s.ref_shape, -1.0, dtype=torch.float32, device="cuda")
    wb = torch.full_like(Ib, -1.0)
    px.make_object_map_noalloc(d, *args, Ib, wb)
    torch.cuda.synchronize()
    return Ia.cpu().numpy(), wa.cpu().numpy(), Ib.cpu().numpy(), wb.cpu().numpy()


def test_noalloc_matches_the_workspace_entry_point_on_consecutive_calls():
    scans = [gen.config_small(),
             gen.tiny2d(n_side=3, det=40, ref=120, offset=25.0, window=3, seed=gen.BASE_SEED + 77)]
    for s in scans + scans[:1]:
        Ia, wa, Ib, wb = _both(s)
        parity.check_omap(Ib, wb, Ia.astype(np.float64), wa.astype(np.float64))
        assert np.array_equal(wb > 0, wa > 0)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    import torch
    import paper_2003_12726_gb300 as px
    d = px.Dims(2, 4, 4, 1100, 1000)           # 1.1e6 reference pixels > 1048576
    t = lambda *shape, dt=torch.float32: torch.zeros(shape, dtype=dt, device="cuda")
    with pytest.raises(px.PxstError) as e:
        px.make_object_map_noalloc(d, t(2, 4, 4), t(4, 4), t(4, 4, dt=torch.uint8), t(2, 4, 4, dt=torch.float64),
                                   t(2, 2, dt=torch.float64), t(1100, 1000), t(1100, 1000))
    assert e.value.code == -5


def test_noalloc_calls_take_no_device_memory():
    """After one warm-up call (which loads the library's device code and with it the fixed
    scratch), further calls leave the device's free memory exactly as it was: nothing is
    allocated per call. The inputs and outputs are set up before the measured window."""
    import torch
    import paper_2003_12726_gb300 as px
    from gpu_util import dev, dims_of
    s = gen.tiny2d(n_side=3, det=40, ref=120, offset=25.0, window=3, seed=gen.BASE_SEED + 78)
    d = dims_of(s.frames, s.ref_shape)
    args = (dev(s.frames, torch.float32), dev(s.W, torch.float32), dev(s.M, torch.uint8),
            dev(s.u_init, torch.float64), dev(s.delta, torch.float64))
    I = torch.empty(s.ref_shape, dtype=torch.float32, device="cuda")
    w = torch.empty_like(I)
    px.make_object_map_noalloc(d, *args, I, w)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        px.make_object_map_noalloc(d, *args, I, w)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)

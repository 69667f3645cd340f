"""The served form: continuous batching with admission by device memory. Every request
finishes; a scan's result is the same alone and in the mix (within the reference image's
FP64-atomic rounding); one GPU-rendered scan served in the mix matches the oracle."""
import numpy as np
import pytest

import parity

pytestmark = pytest.mark.gpu


def _specs():
    return [dict(kind="2d", n_side=4, det=64, window=4, seed=901),
            dict(kind="2d", n_side=6, det=96, window=6, seed=902),
            dict(kind="1d", n_frames=20, ny=24, nx=200, seed=903),
            dict(kind="2d", n_side=5, det=80, window=8, seed=904),
            dict(kind="1d", n_frames=40, ny=32, nx=256, seed=905),
            dict(kind="2d", n_side=3, det=48, window=3, seed=906)]


def _requests(specs, forms, arrivals, n_iter=3, quadratic=None):
    import gen.gpu as gg
    from paper_2003_12726_gb300.serve import Request, estimate_bytes
    out = []
    quadratic = quadratic or [True] * len(specs)
    for k, (sp, f, t, q) in enumerate(zip(specs, forms, arrivals, quadratic)):
        sc = gg.render(sp)                     # once, to size the request
        est = estimate_bytes(sc.dims, sc.window, f)
        out.append(Request(rid=k, arrival=float(t), make=(lambda sp=sp: gg.render(sp)), est_bytes=est,
                           n_iter=n_iter, form=f, quadratic=q, keep_result=True))
    return out


def test_serve_mix_equals_alone():
    from paper_2003_12726_gb300.serve import Server
    specs = _specs()
    forms = [0, 1, 0, 1, 2, 0]
    # alone: each request through its own server
    alone = []
    for k in range(len(specs)):
        r = _requests([specs[k]], [forms[k]], [0.0])[0]
        Server(mem_budget=1 << 34).run([r], realtime=False)
        alone.append(r.result)
    # the mix: staggered arrivals and a budget that holds about two scans at a time
    reqs = _requests(specs, forms, [0.0, 0.002, 0.004, 0.006, 0.008, 0.010])
    budget = 2 * max(r.est_bytes for r in reqs)
    stats = Server(mem_budget=budget, n_streams=4).run(reqs, realtime=True)
    print(stats)
    assert stats["scans"] == len(reqs) and stats["p99_s"] >= stats["p50_s"] > 0
    for k, r in enumerate(reqs):
        assert r.done is not None and r.done >= r.arrival
        ua, ub = alone[k]["u"].cpu().numpy(), r.result["u"].cpu().numpy()
        agree = np.all(np.abs(ua - ub) <= parity.U_TOL, axis=0).mean()
        Ia, Ib = alone[k]["I_ref"].cpu().numpy().astype(np.float64), r.result["I_ref"].cpu().numpy().astype(np.float64)
        rl2 = parity.rel_l2(Ib, Ia)
        print(k, "u agreement", agree, "I_ref rel L2", rl2)
        assert agree >= 0.999 and rl2 < 1e-6


def test_served_scan_against_oracle():
    """GPU-rendered scans served among others, each also served without the fit: one
    iteration of the FP32, BF16 and TF32 ones against the oracle with the full criterion
    (reference image against the oracle's; the map update against the oracle's update on
    the GPU's own reference image)."""
    from types import SimpleNamespace
    import gen.gpu as gg
    from paper_2003_12726_gb300.serve import Server
    specs = _specs()
    forms = [0, 1, 0, 1, 2, 0]
    # every scan twice: with the fit and without it, in one mix
    reqs = _requests(specs + specs, forms + forms, [0.0] * 12, n_iter=1, quadratic=[True] * 6 + [False] * 6)
    Server(mem_budget=1 << 34, n_streams=3).run(reqs, realtime=False)
    for k in (0, 1, 4):
        sc = gg.render(specs[k])
        s = SimpleNamespace(frames=sc.frames.cpu().numpy(), W=sc.W.cpu().numpy(), M=sc.M.cpu().numpy(),
                            delta=sc.delta.cpu().numpy(), ref_shape=sc.ref_shape, window=sc.window)
        u0 = sc.u_init.cpu().numpy()
        host = lambda r: (r.result["u"].cpu().numpy(), r.result["err"].cpu().numpy().astype(np.float64),
                          r.result["I_ref"].cpu().numpy(), r.result["w"].cpu().numpy())
        rep = parity.check_iteration(s, u0, host(reqs[k + 6]), host(reqs[k]))
        print(specs[k], "form", forms[k], rep["update"])

"""The served form: continuous batching with admission by device memory. Every request
finishes; a scan's result is the same alone and in the mix (within the reference image's
FP64-atomic rounding); one GPU-rendered scan served in the mix matches the oracle."""
import numpy as np
import pytest

import oracle
import parity

pytestmark = pytest.mark.gpu


def _specs():
    return [dict(kind="2d", n_side=4, det=64, window=4, seed=901),
            dict(kind="2d", n_side=6, det=96, window=6, seed=902),
            dict(kind="1d", n_frames=20, ny=24, nx=200, seed=903),
            dict(kind="2d", n_side=5, det=80, window=8, seed=904),
            dict(kind="1d", n_frames=40, ny=32, nx=256, seed=905),
            dict(kind="2d", n_side=3, det=48, window=3, seed=906)]


def _requests(specs, forms, arrivals, n_iter=3):
    import gen.gpu as gg
    from paper_2003_12726_gb300.serve import Request, estimate_bytes
    out = []
    for k, (sp, f, t) in enumerate(zip(specs, forms, arrivals)):
        sc = gg.render(sp)                     # once, to size the request
        est = estimate_bytes(sc.dims, sc.window, f)
        out.append(Request(rid=k, arrival=float(t), make=(lambda sp=sp: gg.render(sp)), est_bytes=est,
                           n_iter=n_iter, form=f, keep_result=True))
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
    """A GPU-rendered scan served among others: one iteration against the oracle's."""
    import gen.gpu as gg
    from paper_2003_12726_gb300.serve import Server
    specs = _specs()
    reqs = _requests(specs, [0, 1, 0, 1, 2, 0], [0.0] * 6, n_iter=1)
    Server(mem_budget=1 << 34, n_streams=3).run(reqs, realtime=False)
    for k in (0, 1):
        sc = gg.render(specs[k])
        fr, W, M = sc.frames.cpu().numpy(), sc.W.cpu().numpy(), sc.M.cpu().numpy()
        delta, u0 = sc.delta.cpu().numpy(), sc.u_init.cpu().numpy()
        uo, Io, wo, eo = oracle.iterate(fr, W, M, delta, u0, sc.ref_shape, sc.window, 1)
        ug = reqs[k].result["u"].cpu().numpy()
        same = np.all(np.abs(ug - uo) <= parity.U_TOL, axis=0)[M > 0]
        assert same.mean() >= parity.ARGMIN_AGREE - 0.004, (k, same.mean())
        Ig = reqs[k].result["I_ref"].cpu().numpy().astype(np.float64)
        good = wo > 1e-4 * wo.max()
        assert parity.rel_l2(Ig[good], Io[good]) <= 1e-5

"""Failure handling, with every failure made on the host (no GPU fault, trap or hang):

  * a non-finite frame value at a good pixel: make_object_map reads it as 0, its pixel
    keeps its map with error +inf, the status reports PXST_ERR_INPUT, and every other pixel
    matches the oracle;
  * a whitefield value that is not finite and positive at a good pixel: the pixel is treated
    as masked (the same result as the oracle with M = 0 there), PXST_ERR_INPUT;
  * one scan with bad input in a batch leaves the other scans' results and status as they
    are alone;
  * a stream-ordered wait on a producer that never posts gives up after its limit with
    PXST_ERR_TIMEOUT, and the same workspace then serves a normal iteration; a producer that
    posts (a host thread writing pinned memory) releases the queued work;
  * the served form rejects a request larger than the memory budget without holding up the
    others, and a request cancelled mid-flight leaves the others' results unchanged.
"""
import threading
import time

import numpy as np
import pytest

import gen
import oracle
import parity

pytestmark = pytest.mark.gpu
ERR_INPUT, ERR_TIMEOUT = -7, -6


def _good_pixels(s, k, seed):
    rng = np.random.default_rng(seed)
    good = np.flatnonzero(s.M.ravel())
    return [divmod(int(p), s.M.shape[1]) for p in rng.choice(good, size=k, replace=False)]


def _iterate(s, frames, W, M, form, q):
    import torch
    import paper_2003_12726_gb300 as px
    from gpu_util import dev, dims_of
    d = dims_of(frames, s.ref_shape)
    o = px.Options(s.window[0], s.window[1], q, form)
    u = dev(s.u_init, torch.float64)
    I = torch.empty(s.ref_shape, dtype=torch.float32, device="cuda")
    w = torch.empty_like(I)
    err = torch.empty(s.M.shape, dtype=torch.float32, device="cuda")
    ws = px.workspace(d, o)
    px.iterate(d, o, 1, dev(frames, torch.float32), dev(W, torch.float32), dev(M, torch.uint8),
               dev(s.delta, torch.float64), u, I, w, err, ws)
    code, bits = px.get_status(ws)
    return code, (u.cpu().numpy(), err.cpu().numpy().astype(np.float64), I.cpu().numpy(), w.cpu().numpy())


@pytest.mark.parametrize("form", [0, 1], ids=["fp32", "bf16"])
def test_nonfinite_frame_values(form):
    s = gen.config_small()
    bad = _good_pixels(s, 2, 7)
    frames = s.frames.copy()
    frames[3, bad[0][0], bad[0][1]] = np.nan
    frames[9, bad[1][0], bad[1][1]] = np.inf
    code_i, g_int = _iterate(s, frames, s.W, s.M, form, False)
    code_q, g_q = _iterate(s, frames, s.W, s.M, form, True)
    assert code_i == ERR_INPUT and code_q == ERR_INPUT
    for (y, x) in bad:
        assert np.array_equal(g_q[0][:, y, x], s.u_init[:, y, x]) and g_q[1][y, x] == np.inf
    # the reference image: the oracle's, with the bad values read as 0
    zeroed = frames.copy()
    zeroed[~np.isfinite(zeroed)] = 0.0
    Io, wo = oracle.make_object_map(zeroed, s.W, s.M, s.u_init, s.delta, s.ref_shape)
    parity.check_omap(g_q[2], g_q[3], Io, wo)
    # every other good pixel: the full criterion against the oracle on the GPU's reference
    keep = s.M.copy()
    for (y, x) in bad:
        keep[y, x] = 0
    pix = np.flatnonzero(keep.ravel())
    inp = dict(frames=zeroed, W=s.W, M=s.M, Iref=g_q[2].astype(np.float64), w=g_q[3].astype(np.float64),
               delta=s.delta, u=s.u_init, window=s.window)
    print(parity.check_update(inp, pix, g_int[0].reshape(2, -1)[:, pix], g_int[1].ravel()[pix],
                              g_q[0].reshape(2, -1)[:, pix], g_q[1].ravel()[pix]))


@pytest.mark.parametrize("form", [0, 1], ids=["fp32", "bf16"])
def test_unusable_whitefield_values(form):
    s = gen.config_small()
    bad = _good_pixels(s, 3, 8)
    W = s.W.copy()
    W[bad[0]] = 0.0
    W[bad[1]] = -5.0
    W[bad[2]] = np.nan
    code_i, g_int = _iterate(s, s.frames, W, s.M, form, False)
    code_q, g_q = _iterate(s, s.frames, W, s.M, form, True)
    assert code_i == ERR_INPUT and code_q == ERR_INPUT
    # the same as masking those pixels
    M = s.M.copy()
    for p in bad:
        M[p] = 0
        assert np.array_equal(g_q[0][:, p[0], p[1]], s.u_init[:, p[0], p[1]]) and np.isnan(g_q[1][p])
    Io, wo = oracle.make_object_map(s.frames, s.W, M, s.u_init, s.delta, s.ref_shape)
    parity.check_omap(g_q[2], g_q[3], Io, wo)
    pix = np.flatnonzero(M.ravel())
    inp = dict(frames=s.frames, W=s.W, M=M, Iref=g_q[2].astype(np.float64), w=g_q[3].astype(np.float64),
               delta=s.delta, u=s.u_init, window=s.window)
    print(parity.check_update(inp, pix, g_int[0].reshape(2, -1)[:, pix], g_int[1].ravel()[pix],
                              g_q[0].reshape(2, -1)[:, pix], g_q[1].ravel()[pix]))


def test_bad_input_leaves_the_other_scans_of_a_batch_alone():
    import torch
    import paper_2003_12726_gb300 as px
    B = gen.BASE_SEED
    scans = [gen.tiny2d(n_side=4, det=48, step=6, ref=130, window=4, seed=B + 81),
             gen.tiny2d(n_side=5, det=64, step=4, ref=150, window=6, sigma=1.5, mag=1.2, seed=B + 82),
             gen.tiny2d(n_side=3, det=40, step=5, ref=110, window=3, seed=B + 83)]
    forms = [0, 1, 0]
    frames1 = scans[1].frames.copy()
    frames1[2, 30, 30] = np.nan
    mk = lambda s, f, fr: px.Reconstruction(fr, s.W, s.M, s.delta, s.u_init, s.ref_shape, s.window, form=f)
    alone = []
    for s, f in zip(scans, forms):
        r = mk(s, f, s.frames)
        r.run(1)
        alone.append(r)
    recs = [mk(scans[0], 0, scans[0].frames), mk(scans[1], 1, frames1), mk(scans[2], 0, scans[2].frames)]
    b = px.Batch(recs, n_iter=1, n_branches=3)
    b.run()
    torch.cuda.synchronize()
    b.close()
    assert px.get_status(recs[1].ws)[0] == ERR_INPUT
    for k in (0, 2):
        assert px.get_status(recs[k].ws)[0] == 0
        assert np.array_equal(recs[k].u.cpu().numpy(), alone[k].u.cpu().numpy()) or \
            np.all(np.abs(recs[k].u.cpu().numpy() - alone[k].u.cpu().numpy()) <= parity.U_TOL, axis=0).mean() >= 0.999
        assert parity.rel_l2(recs[k].I_ref.cpu().numpy().astype(np.float64),
                             alone[k].I_ref.cpu().numpy().astype(np.float64)) < 1e-6


def _small_state():
    import torch
    import paper_2003_12726_gb300 as px
    s = gen.config_small()
    r = px.Reconstruction(s.frames, s.W, s.M, s.delta, s.u_init, s.ref_shape, s.window)
    return s, r, torch


def test_wait_on_a_producer_that_never_posts_times_out():
    import paper_2003_12726_gb300 as px
    s, r, torch = _small_state()
    ref = px.Reconstruction(s.frames, s.W, s.M, s.delta, s.u_init, s.ref_shape, s.window)
    ref.run(1)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")          # nothing ever raises it
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    px.wait_flag(flag, 1, 50_000_000, r.ws)                           # 50 ms
    e1.record(st)
    r.run(1)
    code, bits = px.get_status(r.ws)
    assert code == ERR_TIMEOUT and bits & 0x4
    assert e0.elapsed_time(e1) >= 45.0
    # the GPU and the workspace serve the next call as usual
    r.u.copy_(torch.as_tensor(s.u_init).cuda())
    r.run(1)
    assert px.get_status(r.ws)[0] == 0
    assert np.array_equal(r.u.cpu().numpy(), ref.u.cpu().numpy()) or \
        np.all(np.abs(r.u.cpu().numpy() - ref.u.cpu().numpy()) <= parity.U_TOL, axis=0).mean() >= 0.999


def test_wait_released_by_a_host_producer():
    import paper_2003_12726_gb300 as px
    s, r, torch = _small_state()
    flag = torch.zeros(1, dtype=torch.int32).pin_memory()               # read by the GPU in place
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    px.wait_flag(flag, 16, 10_000_000_000, r.ws)                       # 10 s limit
    r.run(1)
    e1.record(st)
    view = flag.numpy()

    def produce():
        time.sleep(0.2)
        view[0] = 16                                                   # "16 frames written"
    t = threading.Thread(target=produce)
    t.start()
    torch.cuda.synchronize()
    t.join()
    assert px.get_status(r.ws)[0] == 0
    assert e0.elapsed_time(e1) >= 150.0
    uo, Io, wo, eo = oracle.iterate(s.frames, s.W, s.M, s.delta, s.u_init, s.ref_shape, s.window, 1)
    parity.check_omap(r.I_ref.cpu().numpy(), r.w.cpu().numpy(), Io, wo)


def test_timeout_option_is_checked():
    import paper_2003_12726_gb300 as px
    s, r, torch = _small_state()
    r.opts.timeout_ns = -1
    with pytest.raises(px.PxstError) as e:
        r.run(1)
    assert e.value.code == -1
    r.opts.timeout_ns = 2_000_000_000
    r.opts.form = 1
    r2 = px.Reconstruction(s.frames, s.W, s.M, s.delta, s.u_init, s.ref_shape, s.window, form=1)
    r2.opts.timeout_ns = 2_000_000_000
    r2.run(1)
    assert px.get_status(r2.ws)[0] == 0


def _serve_requests(specs, n_iter=3):
    import gen.gpu as gg
    from paper_2003_12726_gb300.serve import Request, estimate_bytes
    out = []
    for k, sp in enumerate(specs):
        sc = gg.render(sp)
        out.append(Request(rid=k, arrival=0.0, make=(lambda sp=sp: gg.render(sp)),
                           est_bytes=estimate_bytes(sc.dims, sc.window, 0), n_iter=n_iter, keep_result=True))
    return out


def _same_result(a, b):
    ua, ub = a["u"].cpu().numpy(), b["u"].cpu().numpy()
    agree = np.all(np.abs(ua - ub) <= parity.U_TOL, axis=0).mean()
    return agree, parity.rel_l2(b["I_ref"].cpu().numpy().astype(np.float64), a["I_ref"].cpu().numpy().astype(np.float64))


def test_serve_rejects_a_request_over_the_budget():
    from paper_2003_12726_gb300.serve import Server
    specs = [dict(kind="2d", n_side=4, det=64, window=4, seed=911), dict(kind="2d", n_side=6, det=160, window=6, seed=912),
             dict(kind="2d", n_side=3, det=48, window=3, seed=913)]
    reqs = _serve_requests(specs)
    budget = max(reqs[0].est_bytes, reqs[2].est_bytes) * 2 + 1
    assert reqs[1].est_bytes > budget
    st = Server(mem_budget=budget, n_streams=2).run(reqs, realtime=False)
    assert reqs[1].rejected and reqs[1].done is None and st["rejected"] == 1
    assert reqs[0].done is not None and reqs[2].done is not None and st["peak_bytes"] <= budget
    for k in (0, 2):
        alone = _serve_requests([specs[k]])[0]
        Server(mem_budget=1 << 34).run([alone], realtime=False)
        agree, rl2 = _same_result(alone.result, reqs[k].result)
        assert agree >= 0.999 and rl2 < 1e-6


def test_serve_cancel_mid_flight_leaves_the_others_unchanged():
    from paper_2003_12726_gb300.serve import Server
    specs = [dict(kind="2d", n_side=4, det=64, window=4, seed=921), dict(kind="2d", n_side=5, det=96, window=6, seed=922),
             dict(kind="1d", n_frames=24, ny=24, nx=200, seed=923)]
    reqs = _serve_requests(specs)
    reqs[1].n_iter = 400                                                 # still running when cancelled
    server = Server(mem_budget=1 << 34, n_streams=3)
    timer = threading.Timer(0.05, reqs[1].cancel)
    timer.start()
    st = server.run(reqs, realtime=False)
    timer.join()
    assert reqs[1].cancelled and reqs[1].done is None and 0 < reqs[1].iterations_done < 400
    assert st["cancelled"] == 1 and st["scans"] == 2
    for k in (0, 2):
        alone = _serve_requests([specs[k]])[0]
        Server(mem_budget=1 << 34).run([alone], realtime=False)
        agree, rl2 = _same_result(alone.result, reqs[k].result)
        assert agree >= 0.999 and rl2 < 1e-6

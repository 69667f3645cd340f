"""The batched form (pxst_batch_plan / pxst_batch_run): scans of uneven frame count,
detector size, window and form iterated by one graph launch give the same result as each
scan iterated alone, and match the oracle; the autotuner returns a legal tile shape,
restores the map, and the tuned shape keeps parity."""
import numpy as np
import pytest

import gen
import oracle
import parity

pytestmark = pytest.mark.gpu


def _scans():
    B = gen.BASE_SEED
    return [
        (gen.tiny2d(n_side=4, det=48, step=6, ref=130, window=4, seed=B + 71), 0),
        (gen.tiny2d(n_side=5, det=64, step=4, ref=150, window=6, sigma=1.5, mag=1.2, seed=B + 72), 1),
        (gen.tiny2d(n_side=3, det=40, step=5, ref=110, window=3, seed=B + 73), 0),
        (gen.config_lens1d(n_frames=24, ny=16, nx=256), 0),
        (gen.tiny2d(n_side=6, det=56, step=3, ref=140, window=5, sigma=1.5, mag=1.1, seed=B + 74), 2),
        (gen.tiny2d(n_side=4, det=72, step=6, ref=180, window=8, sigma=1.5, mag=1.3, seed=B + 75), 1),
    ]


def _rec(s, form, quadratic=True):
    import paper_2003_12726_gb300 as px
    return px.Reconstruction(s.frames, s.W, s.M, s.delta, s.u_init, s.ref_shape, s.window, quadratic=quadratic,
                             form=form)


def _host(r):
    """(u, err, I_ref, w) of a Reconstruction on the host, for parity.check_iteration."""
    return (r.u.cpu().numpy(), r.err.cpu().numpy().astype(np.float64), r.I_ref.cpu().numpy(), r.w.cpu().numpy())


def _same(ra, rb, M):
    ua, ub = ra.u.cpu().numpy(), rb.u.cpu().numpy()
    good = M > 0
    agree = np.all(np.abs(ua - ub) <= parity.U_TOL, axis=0)[good].mean()
    Ia, Ib = ra.I_ref.cpu().numpy().astype(np.float64), rb.I_ref.cpu().numpy().astype(np.float64)
    return agree, parity.rel_l2(Ib, Ia)


def test_batch_matches_each_scan_alone():
    import torch
    import paper_2003_12726_gb300 as px
    scans = _scans()
    alone = []
    for s, f in scans:
        r = _rec(s, f)
        r.run(2)
        alone.append(r)
    recs = [_rec(s, f) for s, f in scans]
    b = px.Batch(recs, n_iter=2, n_branches=3)
    assert sorted({b.branch(i) for i in range(len(recs))}) == [0, 1, 2]
    b.run()
    torch.cuda.synchronize()
    for (s, f), ra, rb in zip(scans, alone, recs):
        agree, rl2 = _same(ra, rb, s.M)
        print(s.name, "form", f, "u agreement", agree, "I_ref rel L2", rl2)
        # the reference image sums FP64 atomics: equal to rounding, so a near-tie may flip
        assert agree >= 0.999 and rl2 < 1e-6
    # the graph replays: two more iterations of every scan
    b.run()
    torch.cuda.synchronize()
    for (s, f), ra in zip(scans, alone):
        ra.run(2)
    torch.cuda.synchronize()
    for (s, f), ra, rb in zip(scans, alone, recs):
        agree, rl2 = _same(ra, rb, s.M)
        assert agree >= 0.995 and rl2 < 1e-5, (s.name, agree, rl2)
    b.close()


def test_batch_against_oracle():
    """One iteration of every scan in one batch, without and with the fit (two batches);
    2-D scans in FP32, BF16 and TF32 and the 1-D lens scan (FP32, fractional shifts) against
    the oracle with the full criterion."""
    import torch
    import paper_2003_12726_gb300 as px
    scans = _scans()
    recs = {q: [_rec(s, f, q) for s, f in scans] for q in (False, True)}
    for q in (False, True):
        b = px.Batch(recs[q], n_iter=1, n_branches=4)
        b.run()
        torch.cuda.synchronize()
        b.close()
    for k in (0, 1, 3, 4):
        s = scans[k][0]
        rep = parity.check_iteration(s, s.u_init, _host(recs[False][k]), _host(recs[True][k]))
        print(s.name, "form", scans[k][1], rep["update"])


@pytest.mark.parametrize("form", [0, 1], ids=["fp32", "bf16"])
def test_autotune(form):
    import torch
    import paper_2003_12726_gb300 as px
    s = gen.tiny2d(n_side=5, det=64, step=4, ref=150, window=6, sigma=1.5, mag=1.2, seed=gen.BASE_SEED + 76)
    r = _rec(s, form)
    r.run(1)                                  # a reference image to search against
    u0 = r.u.clone()
    tile, ms = px.autotune(r, trials=2)
    if form == 0:     # tile height (bits 0-3) and strip length (bits 4-5)
        assert (tile & 15) in (0, 1, 2, 4, 8) and 0 <= tile >> 4 <= 3 and ms > 0
    else:
        assert tile in (0, 1, 2) and ms > 0
    assert torch.equal(r.u, u0)               # the map is restored
    # the tuned shape keeps parity: one iteration from the restored state, without and with
    # the fit, against the oracle with the full criterion
    u_start = u0.cpu().numpy()
    res = {}
    for q in (False, True):
        r.u.copy_(u0)
        r.opts.quadratic = q
        r.run(1)
        res[q] = _host(r)
    rep = parity.check_iteration(s, u_start, res[False], res[True])
    print("form", form, "tuned tile", tile, "ms", ms, rep["update"])


def test_host_stream_matches_plain_steps():
    """HostStream (inputs from pinned host memory every step, copies overlapped with the
    previous step's compute on two device buffers) gives every step the result of one plain
    iteration from the host map."""
    import torch
    import paper_2003_12726_gb300 as px
    s = gen.tiny2d(n_side=5, det=64, step=4, ref=150, window=6, sigma=1.5, mag=1.2, seed=gen.BASE_SEED + 77)
    ref = _rec(s, 0)
    ref.run(1)
    want_u, want_e = ref.u.cpu().numpy(), ref.err.cpu().numpy()
    rec = _rec(s, 0)
    pinned = rec.pin_host_buffers(s.frames, s.W, s.M, s.delta, s.u_init)
    hs = px.HostStream(rec, pinned)
    h2d, d2h = hs.run(5)
    hs.synchronize()
    assert h2d == s.frames.nbytes + s.W.nbytes + s.M.nbytes + s.delta.nbytes + s.u_init.nbytes
    got_u, got_e = pinned["u_out"].numpy(), pinned["err_out"].numpy()
    agree = np.all(np.abs(got_u - want_u) <= parity.U_TOL, axis=0)[s.M > 0].mean()
    assert agree >= 0.999, agree
    np.testing.assert_allclose(got_e[s.M > 0], want_e[s.M > 0], rtol=1e-5)

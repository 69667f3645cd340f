"""The integrate option on the GPU (pxst_integrate_map, one cooperative launch of the whole
conjugate-gradient solve) against the FP64 oracle's (reading R17): both solve the normal
equations to a relative residual of 1e-12, so the projected maps agree to 1e-6 px at every
pixel; maps that couple the axes (a curl to remove), ragged detectors, isolated bad pixels
and a notched mask."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def _maps():
    rng = np.random.default_rng(gen.BASE_SEED + 601)
    s = gen.config_small()
    n = gen.nonsep2d(n_side=2, det=48, ref=150, seed=gen.BASE_SEED + 602)
    ny, nx = 37, 45
    i, j = np.mgrid[0:ny, 0:nx].astype(np.float64)
    M = np.ones((ny, nx), np.uint8)
    M[10:14, 30:] = 0                                                     # a notch from the edge
    M[20, 5] = M[5, 40] = M[30, 22] = 0                                   # isolated bad pixels
    swirl = np.stack([20 + 1.3 * i - 0.4 * (j - 22), 15 + 1.3 * j + 0.4 * (i - 18)]) + rng.normal(size=(2, ny, nx))
    return {
        "small-true": (s.M, s.u_true),
        "small-noisy": (s.M, s.u_true + 0.3 * rng.normal(size=s.u_true.shape)),
        "nonsep-bad-pixels": (n.M, n.u_true),
        "ragged-notched-swirl": (M, swirl),
    }


@pytest.mark.parametrize("name", sorted(_maps()))
def test_integrate_parity(name):
    import torch
    import paper_2003_12726_gb300 as px
    M, u = _maps()[name]
    ny, nx = M.shape
    d = px.Dims(1, ny, nx, 8, 8)
    ws = px.workspace(d)
    ug = torch.as_tensor(np.ascontiguousarray(u)).cuda()
    info = px.integrate_map(d, torch.as_tensor(M).cuda(), ug, ws, tol=1e-12)
    code, bits = px.get_status(ws)
    assert code == 0, (code, bits)
    steps, res = info.cpu().numpy()
    uo, it, res_o = oracle.integrate_map(M, u, tol=1e-12)
    got = ug.cpu().numpy()
    du = np.abs(got - uo)
    print(name, "GPU steps", steps, "residual %.2e" % res, "oracle steps", it, "residual %.2e" % res_o,
          "max |du| %.2e" % du.max())
    assert res <= 1e-12 and res_o <= 1e-12
    assert du.max() <= 1e-6
    # M = 0 pixels keep their map
    assert np.array_equal(got[:, M == 0], u[:, M == 0])


def test_integrate_is_deterministic_and_a_projection():
    """Two calls give bit-identical maps (the dot products are summed in block order), and
    integrating the result again changes it by no more than the solve's tolerance."""
    import torch
    import paper_2003_12726_gb300 as px
    M, u = _maps()["ragged-notched-swirl"]
    ny, nx = M.shape
    d = px.Dims(1, ny, nx, 8, 8)
    ws = px.workspace(d)
    Mg = torch.as_tensor(M).cuda()
    a = torch.as_tensor(np.ascontiguousarray(u)).cuda()
    b = a.clone()
    px.integrate_map(d, Mg, a, ws, tol=1e-12)
    px.integrate_map(d, Mg, b, ws, tol=1e-12)
    assert torch.equal(a, b)
    c = a.clone()
    px.integrate_map(d, Mg, c, ws, tol=1e-12)
    assert (c - a).abs().max().item() <= 1e-6
    assert px.get_status(ws)[0] == 0

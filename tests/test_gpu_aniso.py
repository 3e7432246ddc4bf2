"""Parity of the ellipsoid (anisotropic, EWA footprint) path through the C ABI
with the FP64 oracle of oracle/aniso.py.

Forward: FP32 within 2e-5 relative (floor 1 for colour / silhouette, 4 m
for depth) on pixels whose decisions sit farther than 1e-4 (relative) from
their thresholds.  The conic is formed in FP32 from J, M, R(q) and s (about
ten rounded products and sums per entry before the 2 x 2 inverse), so q
carries a few 1e-7 relative error where the sphere form has one or two
roundings; alpha = o exp(-q/2) turns a relative error d of q into q d / 2
<= 4.5 d of alpha, and the composite adds the transmittance's rounding:
twice the sphere bound covers it.  Gradients within 1e-4 relative per tensor
(L2) and per element, plus 1e-4 of each element's componentwise magnitude.
"""

import numpy as np
import pytest
import torch

from oracle import aniso
from paper_2506_02741_gb300 import _lib as L
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn
from tests import _gpu as G
from tests import _helpers as h

pytestmark = pytest.mark.gpu

FWD_TOL = 2e-5
TAU_INCL = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _q32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _case(name):
    if name == "tiny":
        sec, target, K = h.tiny_section()
        Kt, W, H, seed = K.astuple(), K.W, K.H, 21
    elif name == "qqvga_2views":
        K = syn.scaled_intrinsics(160, 120)
        sec, target = h.multiview_section(K, n_views=2)
        Kt, W, H, seed = K.astuple(), K.W, K.H, 22
    else:   # ragged image, three views
        K = syn.scaled_intrinsics(200, 130)
        sec, target = h.multiview_section(K, n_views=3, seed=9)
        Kt, W, H, seed = K.astuple(), 203, 131, 23
    sec = G.quantise(sec)
    scale, quat = syn.random_ellipsoids(sec.radius, seed)
    return sec, _q32(scale), _q32(quat), target, Kt, W, H


def _device(sec, scale, quat):
    return G.to_device(sec).with_ellipsoids(torch.from_numpy(scale), torch.from_numpy(quat))


CASES = ["tiny", "qqvga_2views", "ragged_3views"]


@pytest.mark.parametrize("case", CASES)
def test_ellipsoid_forward_parity(dev, case):
    sec, scale, quat, target, K, W, H = _case(case)
    R = api.Renderer()
    out = R.render([_device(sec, scale, quat)], api.pose12(target, dev), K, W, H, checked=True)
    torch.cuda.synchronize()
    ref = aniso.render(sec, scale, quat, target, K, W, H)
    mask = G.clean_mask(ref, tau_incl=TAU_INCL)
    assert mask.mean() > 0.9, mask.mean()
    assert ref["n_added"].mean() > 5
    G.assert_forward_close(out, ref, mask, tol=FWD_TOL)


@pytest.mark.parametrize("case", CASES)
def test_ellipsoid_gradients(dev, case):
    """Colour, opacity, scale, quaternion and target-pose gradients against
    the oracle's chain rule (upstream gradients on the clean pixels only)."""
    sec, scale, quat, target, K, W, H = _case(case)
    R = api.Renderer()
    dsec = _device(sec, scale, quat)
    R.render([dsec], api.pose12(target, dev), K, W, H, checked=True)
    ref = aniso.render(sec, scale, quat, target, K, W, H)
    clean = G.clean_mask(ref, tau_incl=TAU_INCL, tau_clamp=1e-4)
    rng = np.random.default_rng(31)
    gR = (rng.normal(0, 1, (3, H, W)) * clean).astype(np.float32)
    gD = (rng.normal(0, 1, (H, W)) * clean).astype(np.float32)
    gS = (rng.normal(0, 1, (H, W)) * clean).astype(np.float32)
    want = aniso.backward(sec, scale, quat, target, K, W, H, gR, gD, gS)
    n = sec.n
    z = lambda *s: torch.zeros(*s, device=dev)
    grads = [(z(n, 3), z(n), None, z(n, 3), z(n, 4))]
    t = lambda a: torch.from_numpy(a).to(dev)
    dtw, dmat = R.backward(t(gR), t(gD), t(gS), attr_grads=grads, pose_grad=True)
    torch.cuda.synchronize()
    got = dict(colour=grads[0][0], opacity=grads[0][1], scale=grads[0][3], quat=grads[0][4])
    for k, v in got.items():
        G.assert_grad_close(v.cpu().numpy(), want[k], name=k, abs_ref=want["abs_" + k])
    G.assert_grad_close(dtw.cpu().numpy(), want["twist"], name="twist", abs_ref=want["abs_twist"])
    G.assert_grad_close(dmat.cpu().numpy(), want["mat"], name="mat", abs_ref=want["abs_mat"])
    assert np.abs(want["scale"]).max() > 0 and np.abs(want["twist"]).max() > 0


def test_ellipsoid_replay_matches_lists(dev):
    """Without per-pixel lists (memory budget) the tile replay gives the same
    forward and the same gradients up to the order of float atomics."""
    sec, scale, quat, target, K, W, H = _case("qqvga_2views")
    dsec = _device(sec, scale, quat)
    res = []
    for budget in (None, 1):
        R = api.Renderer()
        if budget is not None:
            R.set_budget(budget)
        out = R.render([dsec], api.pose12(target, dev), K, W, H, checked=True)
        assert R.used_lists == (budget is None)
        rng = np.random.default_rng(3)
        gR = torch.from_numpy(rng.normal(0, 1, (3, H, W)).astype(np.float32)).to(dev)
        gD = torch.from_numpy(rng.normal(0, 1, (H, W)).astype(np.float32)).to(dev)
        n = sec.n
        gr = [(torch.zeros(n, 3, device=dev), torch.zeros(n, device=dev), None,
               torch.zeros(n, 3, device=dev), torch.zeros(n, 4, device=dev))]
        tw, mat = R.backward(gR, gD, None, attr_grads=gr, pose_grad=True)
        torch.cuda.synchronize()
        res.append((out, gr[0], tw, mat))
    (o1, g1, tw1, m1), (o2, g2, tw2, m2) = res
    for a, b in zip(o1, o2):
        assert torch.equal(a, b)
    for a, b in zip(g1, g2):
        if a is None:
            continue
        torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()))
    torch.testing.assert_close(tw1, tw2, rtol=1e-4, atol=1e-5 * float(tw2.abs().max()))


def test_ellipsoid_argument_errors(dev):
    sec, scale, quat, target, K, W, H = _case("tiny")
    ell = _device(sec, scale, quat)
    sph = G.to_device(sec)
    R = api.Renderer()
    with pytest.raises(L.VTError):
        R.render([ell, sph], api.pose12(target, dev), K, W, H)
    R.render([ell], api.pose12(target, dev), K, W, H)
    g = torch.zeros(W * H * 3, device=dev).reshape(3, H, W)
    vt = torch.zeros(1, 6, dtype=torch.float64, device=dev)
    with pytest.raises(L.VTError):
        R.backward(g, None, None, view_grads=[(vt, None)])
    with pytest.raises(ValueError):
        api.Section(ell.poses, ell.depth, ell.K, ell.src, ell.colour, ell.opacity, ell.radius,
                    scale=ell.scale).validate()

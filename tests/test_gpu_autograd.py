"""torch.autograd wrapper: gradients against the oracle, the memory-tight
recompute path, several outstanding forwards, and a finite-difference check
of the wiring on the GPU itself."""

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn
from paper_2506_02741_gb300.autograd import RendererPool, splat
from tests import _gpu as G
from tests import _helpers as h

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _three_sections(seed=12):
    K = syn.scaled_intrinsics(128, 96)
    full, target = h.multiview_section(K, n_views=3, seed=seed)
    plane = full.W * full.H
    view = full.src // plane
    parts = []
    for k in range(3):
        m = view == k
        parts.append(G.quantise(oracle.Section(full.W, full.H, full.K, full.poses[k:k + 1],
                                               full.depth[k:k + 1],
                                               (full.src[m] - k * plane).astype(np.uint32),
                                               full.colour[m], full.opacity[m], full.radius[m])))
    return K, parts, target


def _loss_and_grads(dev, parts, target, K, g, recompute, pool):
    secs = [G.to_device(p) for p in parts]
    learn = secs[1]
    for t in (learn.colour, learn.opacity, learn.radius):
        t.requires_grad_(True)
    pose = api.pose12(target, dev).requires_grad_(True)
    rgb, depth, sil = splat(secs, pose, K.astuple(), K.W, K.H, recompute=recompute, pool=pool)
    loss = (rgb * g[0]).sum() + (depth * g[1]).sum() + (sil * g[2]).sum()
    loss.backward()
    torch.cuda.synchronize()
    return [x.grad.cpu().numpy() for x in (learn.colour, learn.opacity, learn.radius)], \
        pose.grad.cpu().numpy()


def test_autograd_matches_oracle_and_recompute(dev):
    K, parts, target = _three_sections()
    Kt = K.astuple()
    # the GPU's decisions for these inputs (a render that keeps per-pixel
    # lists); the oracle differentiates along them
    ids, cnt = G.decisions([G.to_device(p) for p in parts], api.pose12(target, dev), Kt, K.W, K.H)
    G.check_decisions(oracle.render_lists(parts, target, Kt, K.W, K.H, ids, cnt), "autograd")
    rng = np.random.default_rng(3)
    gn = [rng.normal(0, 1, s).astype(np.float32) for s in ((3, K.H, K.W), (K.H, K.W), (K.H, K.W))]
    g = [torch.from_numpy(x).to(dev) for x in gn]
    want = oracle.backward_lists(parts, target, Kt, K.W, K.H, ids, cnt, g_rgb=gn[0], g_depth=gn[1],
                                 g_sil=gn[2])
    pool = RendererPool()
    attr, dpose = _loss_and_grads(dev, parts, target, K, g, False, pool)
    for k, name in enumerate(("colour", "opacity", "radius")):
        G.assert_grad_close(attr[k], want[name][1], name=name, abs_ref=want["abs_" + name][1])
    G.assert_grad_close(dpose, want["mat"], name="pose", noise=want["mat_noise"])
    attr2, dpose2 = _loss_and_grads(dev, parts, target, K, g, True, pool)
    assert np.array_equal(dpose, dpose2)          # deterministic pose reduction
    for a, b in zip(attr, attr2):                 # float atomics: order only
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())


def test_two_outstanding_forwards(dev):
    K, parts, target = _three_sections(seed=13)
    Kt = K.astuple()
    secs = [G.to_device(p) for p in parts]
    for t in (secs[0].colour, secs[0].opacity):
        t.requires_grad_(True)
    pool = RendererPool()
    P2 = h.right_perturb(target, 4, 0.01)
    outs = [splat(secs, api.pose12(P, dev), Kt, K.W, K.H, pool=pool)[0] for P in (target, P2)]
    (outs[0].sum() + 2.0 * outs[1].sum()).backward()
    both = [secs[0].colour.grad.clone(), secs[0].opacity.grad.clone()]
    singles = []
    for P, wgt in ((target, 1.0), (P2, 2.0)):
        secs[0].colour.grad = None
        secs[0].opacity.grad = None
        (wgt * splat(secs, api.pose12(P, dev), Kt, K.W, K.H, pool=pool)[0].sum()).backward()
        singles.append([secs[0].colour.grad.clone(), secs[0].opacity.grad.clone()])
    for k in range(2):
        torch.testing.assert_close(both[k], singles[0][k] + singles[1][k], rtol=1e-5, atol=1e-6)


def test_finite_difference_wiring(dev):
    """Central differences of the GPU forward itself agree with the autograd
    opacity gradient (Gaussians with o > 0.4, whose 1/255 cut lies outside the
    3-sigma disc, so a small change of o moves no inclusion decision)."""
    osec, target, K = h.tiny_section()
    sec = G.to_device(G.quantise(osec))
    Kt = K.astuple()
    sec.opacity.requires_grad_(True)
    pose = api.pose12(target, dev)
    w = torch.linspace(0.5, 1.5, 3 * K.H * K.W, device=dev).reshape(3, K.H, K.W)
    (splat(sec, pose, Kt, K.W, K.H)[0] * w).sum().backward()
    go = sec.opacity.grad.clone()
    cand = torch.nonzero(sec.opacity.detach() > 0.4).flatten()
    idx = cand[torch.argsort(go[cand].abs(), descending=True)[:6]]
    orig = sec.opacity.detach().clone()
    for i in idx.tolist():
        e = 1e-3
        with torch.no_grad():
            sec.opacity[i] = orig[i] + e
            ip = splat(sec, pose, Kt, K.W, K.H)[0].double()
            sec.opacity[i] = orig[i] - e
            im = splat(sec, pose, Kt, K.W, K.H)[0].double()
            sec.opacity.copy_(orig)
        fd = (((ip - im) * w.double()).sum() / (2 * e)).item()   # untouched pixels cancel exactly
        assert fd == pytest.approx(go[i].item(), rel=1e-2, abs=1e-4)

"""Pins of the oracle's compositing along given decisions (orc_render_lists,
orc_backward_lists): the definition's own lists reproduce its render and
gradients bit for bit, hand-built pixels whose decisions sit within a known
relative distance of their thresholds accept exactly the flips the margins
allow, and planted list errors (a dropped, swapped, repeated, foreign or
extra Gaussian, a walk stopped early) are rejected."""

import numpy as np
import pytest

import oracle
from paper_2506_02741_gb300 import synthetic as syn
from tests import _helpers as h

IDENT = syn.identity_pose()
K16 = (20.0, 20.0, 7.5, 5.5)
T_MIN = float(np.float32(1e-4))


def _own(sec, target, K, W, H):
    ref = oracle.render([sec], target, K, W, H, list_cap=512)
    return ref, ref["lists"].copy(), ref["n_added"].copy()


@pytest.mark.parametrize("case", ["tiny", "qqvga_2views"])
def test_own_lists_reproduce_render_and_gradients(case):
    if case == "tiny":
        sec, target, Kc = h.tiny_section()
    else:
        Kc = syn.scaled_intrinsics(160, 120)
        sec, target = h.multiview_section(Kc, n_views=2)
    K, W, H = Kc.astuple(), Kc.W, Kc.H
    ref, ids, cnt = _own(sec, target, K, W, H)
    assert cnt.max() < 512
    out = oracle.render_lists([sec], target, K, W, H, ids, cnt)
    for k in ("rgb", "depth", "sil", "T_final", "n_added"):
        np.testing.assert_array_equal(out[k], ref[k])
    assert not out["status"].any() and not out["flips"].any()
    rng = np.random.default_rng(3)
    g = [rng.normal(size=(3, H, W)), rng.normal(size=(H, W)), rng.normal(size=(H, W))]
    old = oracle.get_threads()
    oracle.set_threads(1)     # one summation order for both
    try:
        a = oracle.backward([sec], target, K, W, H, *g)
        b = oracle.backward_lists([sec], target, K, W, H, ids, cnt, *g)
    finally:
        oracle.set_threads(old)
    for k in ("colour", "opacity", "radius", "x", "abs_colour", "abs_opacity", "abs_radius"):
        np.testing.assert_array_equal(a[k][0], b[k][0])
    for k in ("twist", "mat", "twist_noise", "mat_noise"):
        np.testing.assert_array_equal(a[k], b[k])


def _pixel_of_interest(ref, min_added=4):
    """A pixel with several added Gaussians whose decisions all lie far from
    their thresholds."""
    ok = (ref["n_added"] >= min_added) & (ref["margin"] > 1e-3) & (ref["margin_T"] > 1e-2)
    ys, xs = np.nonzero(ok)
    assert ys.size
    return ys[0], xs[0]


def test_planted_list_errors_rejected():
    sec, target, Kc = h.tiny_section()
    K, W, H = Kc.astuple(), Kc.W, Kc.H
    ref, ids, cnt = _own(sec, target, K, W, H)
    y, x = _pixel_of_interest(ref)
    n = int(cnt[y, x])
    row = ids[y, x, :n].copy()

    def verdict(new):
        i2, c2 = ids.copy(), cnt.copy()
        i2[y, x, :] = -1
        i2[y, x, :len(new)] = new
        c2[y, x] = len(new)
        out = oracle.render_lists([sec], target, K, W, H, i2, c2)
        others = np.ones((H, W), bool)
        others[y, x] = False
        assert not out["status"][others].any()
        return int(out["status"][y, x])

    assert verdict(row) == 0
    assert verdict(np.delete(row, 1)) == 2                       # a Gaussian dropped
    assert verdict(row[[1, 0] + list(range(2, n))]) == 1         # two swapped
    assert verdict(np.insert(row, 1, row[1])) == 1               # one repeated
    assert verdict(row[:-1]) == 2                                # stopped one early
    # a Gaussian that cannot reach the pixel (the one farthest away on the image)
    far = int(np.argmax(np.abs(sec.src.astype(np.int64) % W - x)))
    bad = np.sort(np.append(row, far))
    assert verdict(bad) != 0
    # an invalid id
    assert verdict(np.append(row[:-1], sec.n + 5)) == 1


def _stack(depths, opacity, radius=None, pix=(8, 6), W=16, H=12):
    """Gaussians of several views (all at the identity pose) on one pixel, at
    the given depths (increasing = front to back)."""
    views = [(IDENT, {pix: float(d)}) for d in depths]
    return h.hand_section(views, W, H, K16, opacity=opacity, radius=radius)


def test_termination_flip_within_margin():
    """Four Gaussians on one pixel: alpha 0.9 three times, then the one whose
    inclusion would leave T = T_MIN (1 + 5e-6); a fifth (alpha 0.5) behind.
    The definition adds the first four; a walk that stopped at the fourth is
    correct within tau_T >= 5e-6 (one flip) and wrong below it.  (Alphas stay
    below the 0.99 clamp, which would otherwise set the margin.)"""
    T3 = (1.0 - 0.9) * (1.0 - 0.9) * (1.0 - 0.9)
    depths = [1.0, 1.1, 1.2, 1.3, 1.4]
    a4 = 1.0 - T_MIN * (1.0 + 5e-6) / T3
    sec = _stack(depths, [0.9, 0.9, 0.9, a4, 0.5])
    ref, ids, cnt = _own(sec, IDENT, K16, 16, 12)
    assert cnt[6, 8] == 4 and list(ids[6, 8, :4]) == [0, 1, 2, 3]
    assert 4e-6 < ref["margin_T"][6, 8] < 6e-6
    early = ids.copy()
    early[6, 8, 3] = -1
    c2 = cnt.copy()
    c2[6, 8] = 3
    out = oracle.render_lists([sec], IDENT, K16, 16, 12, early, c2, tau_T=2e-4)
    assert out["status"][6, 8] == 0 and out["flips"][6, 8] == 1
    assert 4e-6 < out["flip_margin"][6, 8] < 6e-6
    np.testing.assert_allclose(out["sil"][6, 8], 1.0 - T3, rtol=1e-14)
    out = oracle.render_lists([sec], IDENT, K16, 16, 12, early, c2, tau_T=1e-6)
    assert out["status"][6, 8] == 2
    # the other direction: T' = T_MIN (1 - 5e-6) ends the definition's walk
    # before the fourth; a walk that added it is within the same margin
    a4 = 1.0 - T_MIN * (1.0 - 5e-6) / T3
    sec = _stack(depths, [0.9, 0.9, 0.9, a4, 0.5])
    ref, ids, cnt = _own(sec, IDENT, K16, 16, 12)
    assert cnt[6, 8] == 3
    assert 4e-6 < ref["margin_T"][6, 8] < 6e-6
    late = ids.copy()
    late[6, 8, 3] = 3
    c2 = cnt.copy()
    c2[6, 8] = 4
    out = oracle.render_lists([sec], IDENT, K16, 16, 12, late, c2, tau_T=2e-4)
    assert out["status"][6, 8] == 0 and out["flips"][6, 8] == 1
    assert oracle.render_lists([sec], IDENT, K16, 16, 12, late, c2, tau_T=1e-6)["status"][6, 8] == 2


@pytest.mark.parametrize("rel", [-3e-6, 3e-6])
def test_inclusion_flip_within_margin(rel):
    """A Gaussian seen from its own view with sigma chosen so that the pixel
    three columns away sits at q = 9 (1 + rel): included for rel < 0,
    excluded for rel > 0.  Taking the other decision there is one flip of
    margin |rel|, accepted for tau_incl above |rel| and rejected below."""
    f = K16[0]
    D = 2.0
    r = D / (f * np.sqrt(1.0 + rel))        # q = (3 D / f)^2 / r^2 = 9 (1 + rel)
    sec = h.hand_section([(IDENT, {(8, 6): D})], 16, 12, K16, radius=[r])
    ref, ids, cnt = _own(sec, IDENT, K16, 16, 12)
    assert cnt[6, 11] == (1 if rel < 0 else 0)
    other = ids.copy()
    c2 = cnt.copy()
    if rel < 0:
        other[6, 11, 0] = -1
        c2[6, 11] = 0
    else:
        other[6, 11, 0] = 0
        c2[6, 11] = 1
    out = oracle.render_lists([sec], IDENT, K16, 16, 12, other, c2, tau_incl=1e-5)
    assert out["status"][6, 11] == 0 and out["flips"][6, 11] == 1
    assert 2.9e-6 < out["flip_margin"][6, 11] < 3.1e-6
    # the composite follows the given list: alpha = 0.9 exp(-q/2) or nothing
    want = 0.9 * np.exp(-4.5 * (1 + rel)) if rel > 0 else 0.0
    np.testing.assert_allclose(out["sil"][6, 11], want, rtol=1e-14)
    assert oracle.render_lists([sec], IDENT, K16, 16, 12, other, c2,
                               tau_incl=1e-6)["status"][6, 11] == 2


def test_backward_lists_follows_the_given_list():
    """With the walk stopped early at the termination flip, the gradient is
    the one of the shorter composite: the third Gaussian gets nothing, and
    the colour gradient of the first two is gC w."""
    T2 = (1.0 - 0.9) * (1.0 - 0.9)
    a3 = 1.0 - T_MIN * (1.0 + 5e-6) / T2
    col = np.array([[0.1, 0.2, 0.3], [0.4, 0.5, 0.6], [0.7, 0.8, 0.9], [0.2, 0.2, 0.2]])
    views = [(IDENT, {(8, 6): float(d)}) for d in (1.0, 1.1, 1.2, 1.3)]
    sec = h.hand_section(views, 16, 12, K16, colour=col, opacity=[0.9, 0.9, a3, 0.5])
    ref, ids, cnt = _own(sec, IDENT, K16, 16, 12)
    ids[6, 8, 2] = -1
    cnt[6, 8] = 2
    gR = np.zeros((3, 12, 16))
    gR[:, 6, 8] = [1.0, -2.0, 0.5]
    g = oracle.backward_lists([sec], IDENT, K16, 16, 12, ids, cnt, g_rgb=gR)
    w = np.array([0.9, 0.9 * (1.0 - 0.9)])
    np.testing.assert_allclose(g["colour"][0][:2], np.outer(w, [1.0, -2.0, 0.5]), rtol=1e-14)
    assert not g["colour"][0][2:].any() and not g["opacity"][0][2:].any()


def _aniso_own_lists(ref, H, W):
    P = H * W
    lists = [[] for _ in range(P)]
    for (i, pi, *_rest) in ref["recs"]:
        for p in pi:
            lists[p].append(i)
    cap = max(1, max(len(l) for l in lists))
    ids = np.full((P, cap), -1, np.int64)
    cnt = np.zeros(P, np.int64)
    for p, l in enumerate(lists):
        ids[p, :len(l)] = l
        cnt[p] = len(l)
    return ids.reshape(H, W, cap), cnt.reshape(H, W)


def test_ellipsoid_lists():
    """The ellipsoid oracle along its own lists reproduces its render and
    gradients bit for bit; a dropped or swapped Gaussian is rejected."""
    from oracle import aniso
    sec, target, Kc = h.tiny_section()
    K, W, H = Kc.astuple(), Kc.W, Kc.H
    scale, quat = syn.random_ellipsoids(sec.radius, 21)
    ref = aniso.render(sec, scale, quat, target, K, W, H, keep=True)
    ids, cnt = _aniso_own_lists(ref, H, W)
    out = aniso.render_lists(sec, scale, quat, target, K, W, H, ids, cnt, keep=True)
    for k in ("rgb", "depth", "sil", "T_final", "n_added"):
        np.testing.assert_array_equal(out[k], ref[k])
    assert not out["status"].any() and not out["flips"].any()
    gR = np.random.default_rng(1).normal(size=(3, H, W))
    a = aniso.backward(sec, scale, quat, target, K, W, H, gR, fwd=ref)
    b = aniso.backward(sec, scale, quat, target, K, W, H, gR, fwd=out)
    for k in ("colour", "opacity", "scale", "quat", "twist", "mat"):
        np.testing.assert_array_equal(a[k], b[k])
    ok = (ref["n_added"] >= 4) & (ref["margin"] > 1e-3) & (ref["margin_T"] > 1e-2)
    y, x = (v[0] for v in np.nonzero(ok))
    n = int(cnt[y, x])
    for new, want in ((np.delete(ids[y, x, :n], 1), 2),
                      (ids[y, x, [1, 0] + list(range(2, n))], 1)):
        i2, c2 = ids.copy(), cnt.copy()
        i2[y, x, :] = -1
        i2[y, x, :len(new)] = new
        c2[y, x] = len(new)
        st = aniso.render_lists(sec, scale, quat, target, K, W, H, i2, c2)["status"]
        assert st[y, x] == want
        st[y, x] = 0
        assert not st.any()

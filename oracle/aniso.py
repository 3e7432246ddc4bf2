"""Plain FP64 NumPy reference of the anisotropic variant of the render and
its gradient (test infrastructure; see the package docstring for who may
import it).

The ablation on the Gaussians' attributes (Sec. 4, "aniso + w/ VT") keeps
the view-tied centres and swaps the isotropic radius for an ellipsoid.  Each
Gaussian carries a colour c, an opacity o, a scale s (three standard
deviations in metres along its principal axes) and a rotation quaternion
q = (w, x, y, z), normalised on use.  Readings (the paper gives no formulas
for this variant):

  * the ellipsoid is expressed in the camera frame of the source view the
    Gaussian is tied to, so it moves with that view:
        Sigma_k = R(q) diag(s^2) R(q)^T,   Sigma_c = M Sigma_k M^T,
    M = R^T R_k the rotation from view k's camera to the target camera;
  * it is splatted with the local affine (EWA) approximation of the
    perspective projection at its centre x = (x, y, z) in the target camera,
        J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]],
        Sigma_2D = J Sigma_c J^T + eps I   (eps = 0.3 px^2, the low-pass),
    and pixel (u, v) of the target image sees
        q = d^T Sigma_2D^-1 d,   d = (u - u_c, v - v_c),
        u_c = fx x/z + cx,  v_c = fy y/z + cy;
  * a Gaussian whose scales are not all positive and finite, or whose
    quaternion is zero, is not rendered;
  * everything else is the isotropic render's: ahat = o exp(-q/2), included
    iff q <= 9 and ahat >= 1/255, alpha = min(0.99, ahat), order by the FP32
    depth key and then the id, stop before the Gaussian that would take the
    transmittance below 1e-4; outputs colour, depth (sum w z) and silhouette.

The centres, depth keys and validity come from the isotropic oracle's
definitions (centre = back-projected depth pixel, key = FP32 z of it).
Gradients follow the chain rule written out per pair (back-to-front per
pixel) and then per Gaussian; every gradient element also gets its
componentwise magnitude (the sum of the absolute values of the terms that
its formula adds), which bounds the error of an FP32 evaluation.
"""

from __future__ import annotations

import numpy as np

from . import Section, zkeys

EPS_LOWPASS = 0.3
Q_MAX = 9.0
A_MIN = float(np.float32(1.0) / np.float32(255.0))
A_CLAMP = float(np.float32(0.99))
T_MIN = float(np.float32(1e-4))


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrices (n, 3, 3) of quaternions (n, 4) = (w, x, y, z),
    normalised first."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _quat_rot_grad(q: np.ndarray, gR: np.ndarray) -> np.ndarray:
    """dL/dq (n, 4) of the unnormalised quaternion from dL/dR (n, 3, 3)."""
    q = np.asarray(q, np.float64)
    nrm = np.linalg.norm(q, axis=-1, keepdims=True)
    u = q / nrm
    w, x, y, z = u[:, 0], u[:, 1], u[:, 2], u[:, 3]
    g = gR
    # partial derivatives of the entries above with respect to (w, x, y, z)
    dw = 2 * (-z * g[:, 0, 1] + y * g[:, 0, 2] + z * g[:, 1, 0] - x * g[:, 1, 2]
              - y * g[:, 2, 0] + x * g[:, 2, 1])
    dx = 2 * (y * g[:, 0, 1] + z * g[:, 0, 2] + y * g[:, 1, 0] - 2 * x * g[:, 1, 1]
              - w * g[:, 1, 2] + z * g[:, 2, 0] + w * g[:, 2, 1] - 2 * x * g[:, 2, 2])
    dy = 2 * (-2 * y * g[:, 0, 0] + x * g[:, 0, 1] + w * g[:, 0, 2] + x * g[:, 1, 0]
              + z * g[:, 1, 2] - w * g[:, 2, 0] + z * g[:, 2, 1] - 2 * y * g[:, 2, 2])
    dz = 2 * (-2 * z * g[:, 0, 0] - w * g[:, 0, 1] + x * g[:, 0, 2] + w * g[:, 1, 0]
              - 2 * z * g[:, 1, 1] + y * g[:, 1, 2] + x * g[:, 2, 0] + y * g[:, 2, 1])
    du = np.stack([dw, dx, dy, dz], axis=1)
    # through the normalisation u = q / |q|
    return (du - u * np.sum(du * u, axis=1, keepdims=True)) / nrm


def _geometry(sec: Section, scale, quat, pose, K, W, H, eps):
    """Per-Gaussian quantities of the target view: validity, key, centre x
    (target camera), M (view -> target rotation), Sigma_k, Sigma_c, J,
    Sigma_2D, its inverse Q and the projected centre."""
    key, valid = zkeys(sec, pose, K, W, H)
    P = np.asarray(pose, np.float64).reshape(3, 4)
    R, t = P[:, :3], P[:, 3]
    fx, fy, cx, cy = (float(np.float32(k)) for k in K)
    sfx, sfy, scx, scy = (float(np.float32(k)) for k in sec.K)
    plane = sec.W * sec.H
    src = sec.src.astype(np.int64)
    view = src // plane
    pix = src - view * plane
    u = (pix % sec.W).astype(np.float64)
    v = (pix // sec.W).astype(np.float64)
    D = sec.depth.reshape(-1)[src].astype(np.float64)
    Xc = np.stack([D * ((u - scx) / sfx), D * ((v - scy) / sfy), D], axis=1)
    Rk = sec.poses[view][:, :, :3]
    tk = sec.poses[view][:, :, 3]
    mu = np.einsum("nab,nb->na", Rk, Xc) + tk
    x = (mu - t) @ R                                     # R^T (mu - t), rows
    M = np.einsum("ba,nbc->nac", R, Rk)                  # R^T R_k
    Rq = quat_to_rot(quat)
    s = np.asarray(scale, np.float64)
    Sk = np.einsum("nab,nb,ncb->nac", Rq, s * s, Rq)
    Sc = np.einsum("nab,nbc,ndc->nad", M, Sk, M)
    z = x[:, 2]
    n = len(z)
    J = np.zeros((n, 2, 3))
    with np.errstate(divide="ignore", invalid="ignore"):
        J[:, 0, 0] = fx / z
        J[:, 0, 2] = -fx * x[:, 0] / (z * z)
        J[:, 1, 1] = fy / z
        J[:, 1, 2] = -fy * x[:, 1] / (z * z)
        S2 = np.einsum("nab,nbc,ndc->nad", J, Sc, J) + eps * np.eye(2)
        det = S2[:, 0, 0] * S2[:, 1, 1] - S2[:, 0, 1] * S2[:, 1, 0]
        Q = np.stack([np.stack([S2[:, 1, 1], -S2[:, 0, 1]], 1),
                      np.stack([-S2[:, 1, 0], S2[:, 0, 0]], 1)], 1) / det[:, None, None]
        uc = fx * (x[:, 0] / z) + cx
        vc = fy * (x[:, 1] / z) + cy
    # an ellipsoid needs three positive finite scales and a non-zero quaternion
    qn = np.linalg.norm(np.asarray(quat, np.float64), axis=1)
    shape_ok = np.all((s > 0) & np.isfinite(s), axis=1) & (qn > 0) & np.isfinite(qn)
    valid = np.asarray(valid, bool) & shape_ok
    return dict(key=key, valid=valid, x=x, M=M, Rq=Rq, s=s, Sk=Sk, Sc=Sc, J=J, S2=S2, Q=Q,
                uc=uc, vc=vc, z=z, R=R, fx=fx, fy=fy)


def _box(geo, i, W, H, band=1.001):
    """Pixel box of the ellipse q <= 9 * band of Gaussian i (None if empty)."""
    ex = np.sqrt(Q_MAX * band * geo["S2"][i, 0, 0])
    ey = np.sqrt(Q_MAX * band * geo["S2"][i, 1, 1])
    u0 = max(int(np.ceil(geo["uc"][i] - ex)), 0)
    u1 = min(int(np.floor(geo["uc"][i] + ex)), W - 1)
    v0 = max(int(np.ceil(geo["vc"][i] - ey)), 0)
    v1 = min(int(np.floor(geo["vc"][i] + ey)), H - 1)
    if u0 > u1 or v0 > v1:
        return None
    return u0, u1, v0, v1


def render(sec: Section, scale, quat, pose, K, W, H, eps: float = EPS_LOWPASS,
           keep: bool = False):
    """Forward render of one anisotropic section.  Returns rgb (3, H, W),
    depth, sil, T_final, n_added, the relative decision margins (margin:
    inclusion tests q <= 9 and ahat >= 1/255; margin_T: termination;
    margin_clamp: the 0.99 clamp), and with keep=True the per-Gaussian
    records the backward replays."""
    geo = _geometry(sec, scale, quat, pose, K, W, H, eps)
    n = sec.n
    ids = np.arange(n)
    # Gaussians whose box (the one _box takes below) meets the image
    with np.errstate(invalid="ignore"):
        ex = np.sqrt(Q_MAX * 1.001 * geo["S2"][:, 0, 0])
        ey = np.sqrt(Q_MAX * 1.001 * geo["S2"][:, 1, 1])
        meets = ((np.ceil(geo["uc"] - ex) <= W - 1) & (np.floor(geo["uc"] + ex) >= 0) &
                 (np.ceil(geo["vc"] - ey) <= H - 1) & (np.floor(geo["vc"] + ey) >= 0))
    cand = geo["valid"] & meets
    order = [i for i in np.lexsort((ids, geo["key"])) if cand[i]]
    P = W * H
    T = np.ones(P)
    done = np.zeros(P, bool)
    rgb = np.zeros((3, P))
    dep = np.zeros(P)
    sil = np.zeros(P)
    nadd = np.zeros(P, np.int32)
    margin = np.full(P, np.inf)
    margin_T = np.full(P, np.inf)
    margin_c = np.full(P, np.inf)
    colour = np.asarray(sec.colour, np.float64).reshape(-1, 3)
    opac = np.asarray(sec.opacity, np.float64)
    recs = []
    for i in order:
        if not np.isfinite(geo["Q"][i]).all() or geo["z"][i] <= 0:
            continue
        b = _box(geo, i, W, H)
        if b is None:
            continue
        u0, u1, v0, v1 = b
        uu, vv = np.meshgrid(np.arange(u0, u1 + 1), np.arange(v0, v1 + 1))
        p = (vv * W + uu).reshape(-1)
        live = ~done[p]
        p = p[live]
        du = uu.reshape(-1)[live] - geo["uc"][i]
        dv = vv.reshape(-1)[live] - geo["vc"][i]
        Q = geo["Q"][i]
        q = Q[0, 0] * du * du + (Q[0, 1] + Q[1, 0]) * du * dv + Q[1, 1] * dv * dv
        G = np.exp(-0.5 * q)
        ah = opac[i] * G
        m_in = np.minimum(np.abs(q - Q_MAX) / Q_MAX, np.abs(ah - A_MIN) / A_MIN)
        margin[p] = np.minimum(margin[p], m_in)
        inc = (q <= Q_MAX) & (ah >= A_MIN)
        al = np.minimum(A_CLAMP, ah)
        Tn = T[p] * (1.0 - al)
        margin_T[p[inc]] = np.minimum(margin_T[p[inc]], np.abs(Tn[inc] - T_MIN) / T_MIN)
        stop = inc & (Tn < T_MIN)
        done[p[stop]] = True
        inc &= ~stop
        margin_c[p[inc]] = np.minimum(margin_c[p[inc]], np.abs(ah[inc] - A_CLAMP) / A_CLAMP)
        pi = p[inc]
        Ti = T[pi]
        w = al[inc] * Ti
        rgb[:, pi] += colour[i][:, None] * w
        dep[pi] += geo["z"][i] * w
        sil[pi] += w
        T[pi] = Tn[inc]
        nadd[pi] += 1
        if keep and len(pi):
            recs.append((i, pi, Ti, al[inc], ah[inc], q[inc], du[inc], dv[inc]))
    out = dict(rgb=rgb.reshape(3, H, W), depth=dep.reshape(H, W), sil=sil.reshape(H, W),
               T_final=T.reshape(H, W), n_added=nadd.reshape(H, W),
               margin=margin.reshape(H, W), margin_T=margin_T.reshape(H, W),
               margin_clamp=margin_c.reshape(H, W))
    if keep:
        out["recs"] = recs
        out["geo"] = geo
    return out


def render_lists(sec: Section, scale, quat, pose, K, W, H, ids, count, tau_incl=1e-4,
                 tau_T=2e-4, eps: float = EPS_LOWPASS, keep: bool = False):
    """Composite along given per-pixel lists of added Gaussians and check
    them against the definition, as the isotropic oracle's render_lists
    does: ids (H, W, cap) int (front to back, positions in the section),
    count (H, W).  Where an inclusion test or the termination test lies
    within the rounding of a lower precision of its threshold both outcomes
    are correct; a pixel's list is accepted (status 0) if it differs from
    the FP64 decisions only at decisions within tau_incl / tau_T (relative)
    of their thresholds: before its last entry every candidate is added or
    excluded, after it the walk stops at a candidate whose inclusion ends
    it, or excludes it.  status 1: no list of the definition (key order, a
    repeated id, an id that is no candidate of the pixel); 2: a decision
    differs by more than the margins.  Returns rgb, depth, sil, T_final,
    n_added along the lists, status, flips, flip_margin and, with keep, the
    records backward() replays."""
    geo = _geometry(sec, scale, quat, pose, K, W, H, eps)
    n = sec.n
    P = W * H
    ids = np.asarray(ids, np.int64).reshape(P, -1)
    count = np.asarray(count, np.int64).reshape(P)
    if ids.shape[1] == 0:
        ids = np.full((P, 1), -1, np.int64)
    cap = ids.shape[1]
    with np.errstate(invalid="ignore"):
        ex = np.sqrt(Q_MAX * 1.001 * geo["S2"][:, 0, 0])
        ey = np.sqrt(Q_MAX * 1.001 * geo["S2"][:, 1, 1])
        meets = ((np.ceil(geo["uc"] - ex) <= W - 1) & (np.floor(geo["uc"] + ex) >= 0) &
                 (np.ceil(geo["vc"] - ey) <= H - 1) & (np.floor(geo["vc"] + ey) >= 0))
    order = [i for i in np.lexsort((np.arange(n), geo["key"])) if (geo["valid"] & meets)[i]]
    status = np.where((count < 0) | (count > cap), 1, 0).astype(np.int32)
    # the lists themselves: valid ids in strictly increasing (key, id) order
    j = np.arange(cap)[None, :]
    used = j < count[:, None]
    good = (ids >= 0) & (ids < n)
    safe = np.where(good, ids, 0)
    status[np.any(used & ~(good & geo["valid"][safe]), axis=1)] = 1
    k = geo["key"][safe]
    incr = (k[:, :-1] < k[:, 1:]) | ((k[:, :-1] == k[:, 1:]) & (safe[:, :-1] < safe[:, 1:]))
    status[np.any(used[:, 1:] & ~incr, axis=1)] = 1
    flips = np.zeros(P, np.int32)
    fmax = np.zeros(P)
    ptr = np.zeros(P, np.int64)
    resolved = np.zeros(P, bool)
    T = np.ones(P)
    rgb = np.zeros((3, P))
    dep = np.zeros(P)
    sil = np.zeros(P)
    colour = np.asarray(sec.colour, np.float64).reshape(-1, 3)
    opac = np.asarray(sec.opacity, np.float64)
    recs = []

    def flip(mask, m, tau, p):
        ok = mask & (m < tau)
        flips[p[ok]] += 1
        fmax[p[ok]] = np.maximum(fmax[p[ok]], m[ok])
        status[p[mask & ~(m < tau)]] = 2

    for i in order:
        if not np.isfinite(geo["Q"][i]).all() or geo["z"][i] <= 0:
            continue
        b = _box(geo, i, W, H)
        if b is None:
            continue
        u0, u1, v0, v1 = b
        uu, vv = np.meshgrid(np.arange(u0, u1 + 1), np.arange(v0, v1 + 1))
        p = (vv * W + uu).reshape(-1)
        du = uu.reshape(-1) - geo["uc"][i]
        dv = vv.reshape(-1) - geo["vc"][i]
        Q = geo["Q"][i]
        q = Q[0, 0] * du * du + (Q[0, 1] + Q[1, 0]) * du * dv + Q[1, 1] * dv * dv
        G = np.exp(-0.5 * q)
        ah = opac[i] * G
        pq, pa = q <= Q_MAX, ah >= A_MIN
        mq, ma = np.abs(q - Q_MAX) / Q_MAX, np.abs(ah - A_MIN) / A_MIN
        inc = pq & pa
        m_in = np.where(inc, np.minimum(mq, ma),
                        np.maximum(np.where(pq, 0.0, mq), np.where(pa, 0.0, ma)))
        band = q <= Q_MAX * 1.001
        al = np.minimum(A_CLAMP, ah)
        Tn = T[p] * (1.0 - al)
        mT = np.abs(Tn - T_MIN) / T_MIN
        phase_a = ptr[p] < count[p]
        nxt = ids[p, np.minimum(ptr[p], cap - 1)]
        listed = phase_a & (nxt == i)
        active = (status[p] == 0) & ~resolved[p]
        status[p[active & listed & ~band]] = 1
        add = active & listed & band
        flip(add & ~inc, m_in, tau_incl, p)
        flip(add & (Tn < T_MIN), mT, tau_T, p)
        flip(active & phase_a & ~listed & inc, m_in, tau_incl, p)
        after = active & ~phase_a & band
        stop = after & (inc | (m_in < tau_incl)) & ((Tn < T_MIN) | (mT < tau_T))
        flip(stop & ~inc, m_in, np.inf, p)
        flip(stop & ~(Tn < T_MIN), mT, np.inf, p)
        resolved[p[stop]] = True
        flip(after & ~stop & inc, m_in, tau_incl, p)
        pi = p[add]
        Ti = T[pi]
        w = al[add] * Ti
        rgb[:, pi] += colour[i][:, None] * w
        dep[pi] += geo["z"][i] * w
        sil[pi] += w
        T[pi] = Tn[add]
        ptr[pi] += 1
        if keep and len(pi):
            recs.append((i, pi, Ti, al[add], ah[add], q[add], du[add], dv[add]))
    status[(status == 0) & (ptr < count)] = 1
    out = dict(rgb=rgb.reshape(3, H, W), depth=dep.reshape(H, W), sil=sil.reshape(H, W),
               T_final=T.reshape(H, W), n_added=count.reshape(H, W).astype(np.int32),
               status=status.reshape(H, W), flips=flips.reshape(H, W),
               flip_margin=fmax.reshape(H, W))
    if keep:
        out["recs"] = recs
        out["geo"] = geo
    return out


def backward(sec: Section, scale, quat, pose, K, W, H, g_rgb=None, g_depth=None, g_sil=None,
             eps: float = EPS_LOWPASS, fwd=None):
    """Gradients of <g_rgb, rgb> + <g_depth, depth> + <g_sil, sil> with the
    included sets and their order held fixed.  Returns colour (n, 3),
    opacity, scale (n, 3), quat (n, 4), x (n, 3) = dL/dx of the centres in
    the target camera, twist (6,) = dL/d(rho, phi) for P Exp(xi), mat (12,) =
    dL/dR row-major then dL/dt, and abs_* the componentwise magnitude of
    each (the sum of the absolute values of the terms its formula adds,
    propagated through the per-Gaussian chain with absolute Jacobians).
    fwd: the result of render(..., keep=True) for the same inputs, reused."""
    f = fwd if fwd is not None else render(sec, scale, quat, pose, K, W, H, eps, keep=True)
    geo = f["geo"]
    n = sec.n
    P = W * H
    gC = np.zeros((3, P)) if g_rgb is None else np.asarray(g_rgb, np.float64).reshape(3, P)
    gD = np.zeros(P) if g_depth is None else np.asarray(g_depth, np.float64).reshape(P)
    gS = np.zeros(P) if g_sil is None else np.asarray(g_sil, np.float64).reshape(P)
    colour = np.asarray(sec.colour, np.float64).reshape(-1, 3)
    opac = np.asarray(sec.opacity, np.float64)
    d_col = np.zeros((n, 3)); a_col = np.zeros((n, 3))
    d_op = np.zeros(n); a_op = np.zeros(n)
    d_Q = np.zeros((n, 2, 2)); a_Q = np.zeros((n, 2, 2))
    d_uv = np.zeros((n, 2)); a_uv = np.zeros((n, 2))
    d_z = np.zeros(n); a_z = np.zeros(n)
    # back to front: suffix sums of w v and of its componentwise magnitude
    suf = np.zeros(P)
    suf_a = np.zeros(P)
    for (i, pi, Ti, al, ah, q, du, dv) in reversed(f["recs"]):
        c = colour[i]
        z = geo["z"][i]
        w = al * Ti
        vv = gC[0, pi] * c[0] + gC[1, pi] * c[1] + gC[2, pi] * c[2] + gD[pi] * z + gS[pi]
        va = (np.abs(gC[0, pi] * c[0]) + np.abs(gC[1, pi] * c[1]) + np.abs(gC[2, pi] * c[2])
              + np.abs(gD[pi] * z) + np.abs(gS[pi]))
        dLda = Ti * vv - suf[pi] / (1.0 - al)
        aLda = Ti * va + suf_a[pi] / (1.0 - al)
        d_col[i] += (gC[:, pi] * w).sum(1)
        a_col[i] += np.abs(gC[:, pi] * w).sum(1)
        d_z[i] += (gD[pi] * w).sum()
        a_z[i] += np.abs(gD[pi] * w).sum()
        below = ah < A_CLAMP
        G = ah / opac[i]
        d_op[i] += (dLda * G)[below].sum()
        a_op[i] += (aLda * G)[below].sum()
        dLdq = np.where(below, -0.5 * ah * dLda, 0.0)
        aLdq = np.where(below, 0.5 * ah * aLda, 0.0)
        dd = np.stack([du, dv])
        for a in range(2):
            for b in range(2):
                d_Q[i, a, b] += (dLdq * dd[a] * dd[b]).sum()
                a_Q[i, a, b] += (aLdq * np.abs(dd[a] * dd[b])).sum()
        Q = geo["Q"][i]
        Qd = Q @ dd                                        # (2, m)
        d_uv[i] += (-2.0 * dLdq * Qd).sum(1)
        a_uv[i] += (2.0 * aLdq * (np.abs(Q) @ np.abs(dd))).sum(1)
        suf[pi] += w * vv
        suf_a[pi] += w * va
    return _chain(geo, sec, scale, quat, d_col, a_col, d_op, a_op, d_Q, a_Q, d_uv, a_uv, d_z, a_z)


def _chain(geo, sec, scale, quat, d_col, a_col, d_op, a_op, d_Q, a_Q, d_uv, a_uv, d_z, a_z):
    """Per Gaussian: from dL/dQ, dL/d(u_c, v_c), dL/dz (direct) to the scale,
    the quaternion, the centre and the target pose.  Only the Gaussians that
    received a term are evaluated (the others contribute nothing)."""
    n = sec.n
    live = np.flatnonzero((a_Q.reshape(n, -1).sum(1) + a_uv.sum(1) + a_z) > 0)
    sub = lambda a: a[live]
    d_Q, a_Q, d_uv, a_uv, d_z, a_z = map(sub, (d_Q, a_Q, d_uv, a_uv, d_z, a_z))
    geo = {k: (v[live] if isinstance(v, np.ndarray) and v.shape[:1] == (n,) else v)
           for k, v in geo.items()}
    quat = np.asarray(quat, np.float64)[live]
    out = _chain_rows(geo, quat, d_Q, a_Q, d_uv, a_uv, d_z, a_z)
    full = {}
    for k in ("scale", "quat", "x"):
        for pre in ("", "abs_"):
            v = out[pre + k]
            f = np.zeros((n,) + v.shape[1:])
            f[live] = v
            full[pre + k] = f
    full.update(colour=d_col, opacity=d_op, abs_colour=a_col, abs_opacity=a_op,
                twist=out["twist"], mat=out["mat"], abs_twist=out["abs_twist"],
                abs_mat=out["abs_mat"])
    return full


def _chain_rows(geo, quat, d_Q, a_Q, d_uv, a_uv, d_z, a_z):
    ok = geo["valid"] & np.isfinite(geo["Q"]).all(axis=(1, 2)) & (geo["z"] > 0)
    n = len(ok)
    Q, J, Sc, M, Rq, s = geo["Q"], geo["J"], geo["Sc"], geo["M"], geo["Rq"], geo["s"]
    x, z, fx, fy = geo["x"], geo["z"], geo["fx"], geo["fy"]
    A = np.abs
    G2 = -np.einsum("nab,nbc,ncd->nad", Q, d_Q, Q)       # dL/dSigma_2D
    aG2 = np.einsum("nab,nbc,ncd->nad", A(Q), a_Q, A(Q))
    Gc = np.einsum("nba,nbc,ncd->nad", J, G2, J)          # J^T G2 J
    aGc = np.einsum("nba,nbc,ncd->nad", A(J), aG2, A(J))
    GJ = 2.0 * np.einsum("nab,nbc,ncd->nad", G2, J, Sc)   # dL/dJ (G2, Sigma_c symmetric)
    aGJ = 2.0 * np.einsum("nab,nbc,ncd->nad", aG2, A(J), A(Sc))
    gx = np.zeros((n, 3)); ax = np.zeros((n, 3))
    with np.errstate(divide="ignore", invalid="ignore"):
        z2 = z * z
        z3 = z2 * z
        # projected centre
        gx[:, 0] += d_uv[:, 0] * fx / z
        gx[:, 1] += d_uv[:, 1] * fy / z
        gx[:, 2] += -d_uv[:, 0] * fx * x[:, 0] / z2 - d_uv[:, 1] * fy * x[:, 1] / z2
        ax[:, 0] += a_uv[:, 0] * fx / z
        ax[:, 1] += a_uv[:, 1] * fy / z
        ax[:, 2] += a_uv[:, 0] * A(fx * x[:, 0] / z2) + a_uv[:, 1] * A(fy * x[:, 1] / z2)
        # J = J(x)
        gx[:, 0] += GJ[:, 0, 2] * (-fx / z2)
        gx[:, 1] += GJ[:, 1, 2] * (-fy / z2)
        gx[:, 2] += (GJ[:, 0, 0] * (-fx / z2) + GJ[:, 0, 2] * (2 * fx * x[:, 0] / z3)
                     + GJ[:, 1, 1] * (-fy / z2) + GJ[:, 1, 2] * (2 * fy * x[:, 1] / z3))
        ax[:, 0] += aGJ[:, 0, 2] * fx / z2
        ax[:, 1] += aGJ[:, 1, 2] * fy / z2
        ax[:, 2] += (aGJ[:, 0, 0] * fx / z2 + aGJ[:, 0, 2] * A(2 * fx * x[:, 0] / z3)
                     + aGJ[:, 1, 1] * fy / z2 + aGJ[:, 1, 2] * A(2 * fy * x[:, 1] / z3))
    gx[:, 2] += d_z
    ax[:, 2] += a_z
    # Sigma_c = M Sigma_k M^T, Sigma_k = R_q diag(s^2) R_q^T
    Gk = np.einsum("nba,nbc,ncd->nad", M, Gc, M)          # M^T Gc M
    aGk = np.einsum("nba,nbc,ncd->nad", A(M), aGc, A(M))
    RtGR = np.einsum("nba,nbc,ncd->nad", Rq, Gk, Rq)
    aRtGR = np.einsum("nba,nbc,ncd->nad", A(Rq), aGk, A(Rq))
    d_scale = 2.0 * s * np.einsum("naa->na", RtGR)
    a_scale = 2.0 * A(s) * np.einsum("naa->na", aRtGR)
    gR = 2.0 * np.einsum("nab,nbc,nc->nac", Gk, Rq, s * s)
    agR = 2.0 * np.einsum("nab,nbc,nc->nac", aGk, A(Rq), s * s)
    d_quat = _quat_rot_grad(quat, gR)
    a_quat = _quat_rot_grad_abs(quat, agR)
    for arr in (gx, ax, d_scale, a_scale, d_quat, a_quat):
        arr[~ok] = 0.0
    # target pose: A = sum x g^T + Sigma_c (Gc + Gc^T), s = sum g
    Am = np.einsum("na,nb->ab", x[ok], gx[ok]) + np.einsum(
        "nab,nbc->ac", Sc[ok], Gc[ok] + np.transpose(Gc[ok], (0, 2, 1)))
    sg = gx[ok].sum(0)
    R = geo["R"]
    twist = np.array([-sg[0], -sg[1], -sg[2], Am[2, 1] - Am[1, 2], Am[0, 2] - Am[2, 0],
                      Am[1, 0] - Am[0, 1]])
    mat = np.concatenate([(R @ Am).reshape(-1), -(R @ sg)])
    aAm = np.einsum("na,nb->ab", A(x[ok]), ax[ok]) + np.einsum(
        "nab,nbc->ac", A(Sc[ok]), 2 * aGc[ok])
    asg = ax[ok].sum(0)
    abs_twist = np.array([asg[0], asg[1], asg[2], aAm[2, 1] + aAm[1, 2], aAm[0, 2] + aAm[2, 0],
                          aAm[1, 0] + aAm[0, 1]])
    abs_mat = np.concatenate([(A(R) @ aAm).reshape(-1), A(R) @ asg])
    return dict(scale=d_scale, quat=d_quat, x=gx, twist=twist, mat=mat, abs_scale=a_scale,
                abs_quat=a_quat, abs_x=ax, abs_twist=abs_twist, abs_mat=abs_mat)


def _quat_rot_grad_abs(q, agR):
    """Componentwise magnitude of _quat_rot_grad: the same products with
    absolute values (an upper bound of the terms it adds)."""
    q = np.asarray(q, np.float64)
    nrm = np.linalg.norm(q, axis=-1, keepdims=True)
    u = np.abs(q / nrm)
    w, x, y, z = u[:, 0], u[:, 1], u[:, 2], u[:, 3]
    g = agR
    s = lambda *t: sum(t)
    dw = 2 * s(z * g[:, 0, 1], y * g[:, 0, 2], z * g[:, 1, 0], x * g[:, 1, 2], y * g[:, 2, 0],
               x * g[:, 2, 1])
    dx = 2 * s(y * g[:, 0, 1], z * g[:, 0, 2], y * g[:, 1, 0], 2 * x * g[:, 1, 1],
               w * g[:, 1, 2], z * g[:, 2, 0], w * g[:, 2, 1], 2 * x * g[:, 2, 2])
    dy = 2 * s(2 * y * g[:, 0, 0], x * g[:, 0, 1], w * g[:, 0, 2], x * g[:, 1, 0],
               z * g[:, 1, 2], w * g[:, 2, 0], z * g[:, 2, 1], 2 * y * g[:, 2, 2])
    dz = 2 * s(2 * z * g[:, 0, 0], w * g[:, 0, 1], x * g[:, 0, 2], w * g[:, 1, 0],
               2 * z * g[:, 1, 1], y * g[:, 1, 2], x * g[:, 2, 0], y * g[:, 2, 1])
    du = np.stack([dw, dx, dy, dz], axis=1)
    return 2.0 * du / nrm

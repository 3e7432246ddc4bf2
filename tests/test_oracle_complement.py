"""Pins of the oracle's complement initialisation (Sec. 3.4): which pixels
yield Gaussians, and that the completed section covers the frame."""

import numpy as np

import oracle
from paper_2506_02741_gb300 import synthetic as syn


def _frame(i):
    K = syn.TINY
    path = syn.trajectory(12)
    fr = syn.render_frames(syn.make_room(syn.SCENE_SEED), K, [path[i]])
    return K, path[i], fr.depth[0], fr.rgb[0]


def test_covered_frame_yields_nothing_and_uncovered_frame_is_a_fresh_view():
    K, P, d, rgb = _frame(0)
    plane = K.W * K.H
    src, col, op, rad = oracle.section_complement(d, rgb, np.ones_like(d), K.astuple(), view=3)
    assert src.size == 0
    src, col, op, rad = oracle.section_complement(d, rgb, np.zeros_like(d), K.astuple(), view=3)
    ref = oracle.section_init(d[None], rgb[None], K.astuple(), P[None])
    np.testing.assert_array_equal(src, ref.src + 3 * plane)
    np.testing.assert_array_equal(col, ref.colour)
    np.testing.assert_array_equal(rad, ref.radius)
    assert np.all(op == 0.9)


def test_threshold_is_strict_and_invalid_depth_yields_nothing():
    K, P, d, rgb = _frame(0)
    d = d.copy()
    sil = np.ones_like(d)
    sil[2, 5] = np.float32(0.5)           # at the threshold: covered
    sil[2, 6] = np.float32(0.4999)        # below: uncovered
    sil[3, 7] = 0.0
    d[3, 7] = 0.0                         # uncovered but no depth
    src, *_ = oracle.section_complement(d, rgb, sil, K.astuple(), view=0, sil_max=0.5)
    np.testing.assert_array_equal(src, [2 * K.W + 6])


def test_completed_section_covers_the_frame():
    """A one-view section rendered from a later frame leaves pixels
    uncovered; after the complement each of them holds its own Gaussian at
    q = 0 (alpha 0.9), so its silhouette is at least 1 - 0.1 (1 - S_before)."""
    K, P0, d0, rgb0 = _frame(0)
    _, P1, d1, rgb1 = _frame(11)
    sec = oracle.section_init(d0[None], rgb0[None], K.astuple(), P0[None])
    before = oracle.render(sec, P1, K.astuple(), K.W, K.H)
    s0 = before["sil"]
    unc = (s0 < 0.5) & (d1 > 0)
    assert 5 < unc.sum() < 0.5 * unc.size
    src, col, op, rad = oracle.section_complement(d1, rgb1, s0.astype(np.float32), K.astuple(), view=1)
    assert src.size == unc.sum()
    both = oracle.Section(K.W, K.H, sec.K, np.stack([P0, P1]), np.stack([d0, d1]),
                          np.concatenate([sec.src, src]), np.concatenate([sec.colour, col]),
                          np.concatenate([sec.opacity, op]), np.concatenate([sec.radius, rad]))
    after = oracle.render(both, P1, K.astuple(), K.W, K.H)
    assert np.all(after["sil"][unc] >= 1 - 0.1 * (1 - s0[unc]) - 1e-12)
    assert np.all(after["sil"] >= s0 - 1e-12)

"""Host logic of the batch server that needs no GPU: the admission order
(shortest estimated request first, requests past the wait limit first and
oldest first), the batch time budget that follows the queue, and the set
of (section, bucket, kind) that warm-up prepares."""

import numpy as np
import pytest

from paper_2506_02741_gb300 import serving


def _req(rid, arrival, kind="render"):
    return serving.Request(rid, kind, 0, np.eye(3, 4), 0, arrival=arrival)


def test_admission_order_shortest_first_within_the_wait_limit():
    ms = {0: 5.0, 1: 0.5, 2: 2.0, 3: 0.5, 4: 9.0}
    q = [_req(0, 0.100), _req(1, 0.101), _req(2, 0.102), _req(3, 0.103), _req(4, 0.104)]
    # at t = 0.105 s nobody has waited 15 ms: shortest first, ties by arrival
    got = [r.rid for r in serving.admission_order(q, 0.105, lambda r: ms[r.rid], 15.0)]
    assert got == [1, 3, 2, 0, 4]
    # at t = 0.1165 s requests 0 and 1 have waited more than 15 ms: they go
    # first, oldest first, then the rest shortest first
    got = [r.rid for r in serving.admission_order(q, 0.1165, lambda r: ms[r.rid], 15.0)]
    assert got == [0, 1, 3, 2, 4]
    # everyone late: plain arrival order
    got = [r.rid for r in serving.admission_order(q, 1.0, lambda r: ms[r.rid], 15.0)]
    assert got == [0, 1, 2, 3, 4]


def test_admission_order_is_a_permutation():
    rng = np.random.default_rng(0)
    q = [_req(i, float(t)) for i, t in enumerate(np.sort(rng.uniform(0, 0.05, 200)))]
    ms = rng.uniform(0.1, 7.0, 200)
    got = serving.admission_order(q, 0.04, lambda r: ms[r.rid], 8.0)
    assert sorted(r.rid for r in got) == list(range(200))
    late = [r for r in got if r.arrival < 0.04 - 8e-3]
    assert got[:len(late)] == sorted(late, key=lambda r: r.arrival)
    rest = got[len(late):]
    assert all(ms[a.rid] <= ms[b.rid] for a, b in zip(rest, rest[1:]))


@pytest.mark.parametrize("queued,n,lo,hi,want", [
    ([1.0, 2.0], 2, None, 4.0, 4.0),     # fixed budget
    ([], 2, 1.0, 4.0, 1.0),              # empty queue: the floor
    ([1.0, 1.0, 1.0], 2, 1.0, 4.0, 1.5),  # a share of the queued time
    ([5.0] * 10, 2, 1.0, 4.0, 4.0),      # long queue: the cap
])
def test_batch_budget(queued, n, lo, hi, want):
    assert serving.batch_budget(queued, n, lo, hi) == pytest.approx(want)


def test_warm_up_covers_every_section_bucket_and_kind():
    """The requests given to warm() plus one request for every (section,
    bucket, kind) they leave out, at a pose of a given request of the same
    section, else at the first request's pose."""
    srv = serving.BatchServer.__new__(serving.BatchServer)
    srv.sections = [object(), object(), object()]
    srv.resolutions = [(320, 240), (640, 480)]
    p0, p2 = np.eye(3, 4), np.eye(3, 4) + 0.5
    given = [serving.Request(0, "track", 0, p0, 1), serving.Request(1, "render", 2, p2, 0),
             serving.Request(2, "render", 2, p2 + 1.0, 1)]
    every = srv._cover(given)
    assert every[:3] == given
    keys = [(r.section, r.bucket, r.kind) for r in every]
    assert len(keys) == len(set(keys)) == 3 * 2 * 2
    for r in every[3:]:
        assert r.rid == -1 and r.obs is None
        want = p2 if r.section == 2 else p0          # section 1 has no request
        np.testing.assert_array_equal(r.pose, want)
    # nothing to add when every combination is given
    assert srv._cover(every) == every

"""The allocation-free back-projection (vt_backproject_noalloc) against the
regular one, through the C ABI.

It exists for callers that cannot let the library allocate device memory
(graph capture without a memory pool, real-time loops, hosts with their own
allocator); its scratch is a fixed array inside the library.  This file is
named to run last, so a failure here leaves every other test already run.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from paper_2506_02741_gb300 import _lib as L
from paper_2506_02741_gb300 import api
from paper_2506_02741_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _call(fn, depth, K, pose):
    H, W = depth.shape
    cap = H * W
    cen = torch.full((cap, 3), -1.0, device=depth.device)
    pix = torch.full((cap,), -1, dtype=torch.int32, device=depth.device)
    n = torch.full((1,), -1, dtype=torch.int64, device=depth.device)
    st = fn(C.c_void_p(depth.data_ptr()), W, H, L.Intrinsics(*K), C.c_void_p(pose.data_ptr()),
            C.c_void_p(cen.data_ptr()), C.c_void_p(pix.data_ptr()), cap, C.c_void_p(n.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    L.check(st, fn.__name__)
    torch.cuda.synchronize()
    k = int(n.item())
    return k, cen[:k].cpu().numpy(), pix[:k].cpu().numpy()


def test_noalloc_matches_backproject_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    lib = L.lib()
    room = syn.make_room()
    K = syn.scaled_intrinsics(203, 131)          # ragged: the last block is partial
    path = syn.trajectory(12)
    for i, frame in enumerate((4, 11)):          # two calls in a row, different inputs
        depth, _ = syn.raycast(room, K, path[frame])
        depth[7 + i, 5:40] = 0.0                 # invalid pixels
        d = torch.from_numpy(depth).to(dev)
        pose = api.pose12(path[frame], dev)
        ref = _call(lib.vt_backproject, d, K.astuple(), pose)
        got = _call(lib.vt_backproject_noalloc, d, K.astuple(), pose)
        assert got[0] == ref[0] == int(np.sum(depth > 0))
        np.testing.assert_array_equal(got[2], ref[2])
        np.testing.assert_array_equal(got[1], ref[1])


def test_noalloc_rejects_oversize_depth_map():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = L.lib()
    dummy = torch.zeros(16, device="cuda")
    pose = api.pose12(syn.identity_pose())
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = lib.vt_backproject_noalloc(C.c_void_p(dummy.data_ptr()), 4097, 4096,
                                    L.Intrinsics(500.0, 500.0, 2048.0, 2048.0),
                                    C.c_void_p(pose.data_ptr()), C.c_void_p(dummy.data_ptr()),
                                    C.c_void_p(dummy.data_ptr()), 0, C.c_void_p(n.data_ptr()),
                                    None)
    assert st == L.VT_ERR_INVALID_ARG
    assert b"2^24" in lib.vt_last_error()
    # the per-side limit of every entry point applies here too
    for fn in (lib.vt_backproject_noalloc, lib.vt_backproject):
        st = fn(C.c_void_p(dummy.data_ptr()), 70000, 200, L.Intrinsics(500.0, 500.0, 10.0, 10.0),
                C.c_void_p(pose.data_ptr()), C.c_void_p(dummy.data_ptr()),
                C.c_void_p(dummy.data_ptr()), 0, C.c_void_p(n.data_ptr()), None)
        assert st == L.VT_ERR_INVALID_ARG

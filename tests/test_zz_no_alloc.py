"""The allocation-free entry point, integrate_depth_static, against the
ordinary one.

Callers that cannot allocate GPU memory when they integrate (their memory
belongs to another framework, or they are capturing a CUDA graph) pass their
own map storage; the library's per-call work list then comes from a fixed
device array.  This file is collected last on purpose: it runs after every
other test in a full run and must also pass on its own in a fresh process.
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2311_00626_gb300 as gt  # noqa: E402
import synth  # noqa: E402
from tests.runners import to_device  # noqa: E402

MAX_BLOCKS = 1 << 14
CAP = 1 << 15


def _buffers():
    t = {
        "keys": torch.full((CAP,), -1, dtype=torch.int64, device="cuda"),
        "vals": torch.full((CAP,), -1, dtype=torch.int32, device="cuda"),
        "mask": torch.zeros(CAP, dtype=torch.int32, device="cuda"),
        "pool": torch.empty(MAX_BLOCKS * 512 * 2, dtype=torch.float32, device="cuda"),
        "block_keys": torch.empty(MAX_BLOCKS, dtype=torch.int64, device="cuda"),
        "counters": torch.zeros(6, dtype=torch.int64, device="cuda"),
    }
    b = gt.MapBuffers(*(t[k].data_ptr() for k in ("keys", "vals", "mask", "pool", "block_keys",
                                                   "counters")), CAP, MAX_BLOCKS)
    return b, t


def _decode(t):
    """Sorted (keys, D, W) of caller-owned storage, as map_export orders them."""
    cnt = t["counters"].cpu().numpy()
    assert cnt[2] == 0, f"device status bits {cnt[2]}"
    n = int(min(cnt[0], MAX_BLOCKS))
    bk = t["block_keys"][:n].cpu().numpy().view(np.uint64)
    xyz = np.stack([((bk >> np.uint64(21 * a)) & np.uint64(0x1FFFFF)).astype(np.int64) - (1 << 20)
                    for a in range(3)], 1).astype(np.int32)
    pool = t["pool"].view(MAX_BLOCKS, 512, 2)[:n].cpu().numpy()
    order = np.lexsort((xyz[:, 2], xyz[:, 1], xyz[:, 0]))
    return xyz[order], pool[order, :, 0], pool[order, :, 1]


def test_static_entry_matches_integrate_depth_two_calls():
    w = synth.config_room(n_frames=300)
    frames = w.frames[:2]
    dev = to_device(frames)
    v = w.voxel_size
    ref = gt.TsdfMap(v, w.truncation_voxels, w.max_weight)
    buf, t = _buffers()
    tol = 1e-4 * float(np.float32(v))
    for k, (f, d) in enumerate(zip(frames, dev)):
        ref.integrate(f.sensor, f.T, d)
        gt.integrate_depth_static(buf, v, w.truncation_voxels, w.max_weight, d,
                                  gt.pinhole(f.sensor), f.T)
        torch.cuda.synchronize()
        rk, rD, rW = ref.export()
        sk, sD, sW = _decode(t)
        np.testing.assert_array_equal(sk, rk, err_msg=f"call {k}: block sets differ")
        np.testing.assert_array_equal(sW, rW, err_msg=f"call {k}: weights differ")
        obs = rW > 0
        assert np.abs(sD[obs] - rD[obs]).max() <= tol
        assert int(t["counters"][1].item()) == ref.stats()["voxel_updates"]
    ref.close()


def test_static_entry_refuses_oversized_maps():
    buf, _ = _buffers()
    buf.max_blocks = gt.STATIC_MAX_BLOCKS + 1
    buf.hash_capacity = 1 << 18
    w = synth.config_tiny()
    d = torch.from_numpy(w.frames[0].depth).cuda()
    with pytest.raises(gt.TsdfError) as e:
        gt.integrate_depth_static(buf, w.voxel_size, 4, 100.0, d, gt.pinhole(w.frames[0].sensor),
                                  w.frames[0].T)
    assert e.value.code == -3

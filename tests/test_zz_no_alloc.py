"""The allocation-free entry point, integrate_depth_static, against the
ordinary one.

Some callers cannot allocate GPU memory when they integrate: their device
allocator belongs to another framework that owns all of the GPU's memory, or
a real-time loop forbids allocation once it runs.  They pass their own map
storage; the library's per-call work list then comes from a fixed device
array inside the library.  The checks here: two calls in a row give the same
blocks, weights and distances as integrate_depth, bit for bit (the same
kernels run on the same inputs); no byte beyond the documented size of any
caller buffer is written; the calls allocate no device memory; oversized maps
are refused.

This file is collected last on purpose: it runs after every other test in a
full run and must also pass on its own in a fresh process.
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
TAIL = 64  # sentinel elements after each buffer's documented size


def _buffers():
    """Caller-owned storage at exactly the sizes the header documents, each
    followed by a sentinel tail inside the same allocation."""
    spec = {  # name: (elements, dtype, initial value of the documented part)
        "keys": (CAP, torch.int64, -1),
        "vals": (CAP, torch.int32, -1),
        "mask": (CAP, torch.int32, 0),
        "pool": (MAX_BLOCKS * 512 * 2, torch.float32, None),
        "block_keys": (MAX_BLOCKS, torch.int64, None),
        "counters": (gt.NUM_COUNTERS, torch.int64, 0),
    }
    full, head = {}, {}
    for name, (n, dt, init) in spec.items():
        raw = torch.empty(n + TAIL, dtype=dt, device="cuda")
        raw.view(torch.uint8).fill_(0x5A)
        if init is not None:
            raw[:n].fill_(init)
        full[name], head[name] = raw, raw[:n]
    b = gt.MapBuffers(*(head[k].data_ptr() for k in ("keys", "vals", "mask", "pool", "block_keys",
                                                      "counters")), CAP, MAX_BLOCKS)
    return b, head, full


def _tails_untouched(full, label):
    for name, raw in full.items():
        tail = raw[raw.numel() - TAIL:].view(torch.uint8)
        assert bool((tail == 0x5A).all()), f"{label}: bytes written past the end of {name}"


def _decode(t):
    """Sorted (keys, D, W) of caller-owned storage, as map_export orders them."""
    cnt = t["counters"].cpu().numpy()
    assert cnt[2] == 0, f"device status bits {cnt[2]}"
    n = int(min(cnt[0], MAX_BLOCKS))
    bk = t["block_keys"][:n].cpu().numpy().view(np.uint64)
    xyz = np.stack([((bk >> np.uint64(gt.KEY_BITS * a)) & np.uint64((1 << gt.KEY_BITS) - 1))
                    .astype(np.int64) - gt.KEY_BIAS for a in range(3)], 1).astype(np.int32)
    pool = t["pool"].view(MAX_BLOCKS, 512, 2)[:n].cpu().numpy()
    order = np.lexsort((xyz[:, 2], xyz[:, 1], xyz[:, 0]))
    return xyz[order], pool[order, :, 0], pool[order, :, 1]


def test_static_entry_matches_integrate_depth_two_calls():
    w = synth.config_room(n_frames=300)
    frames = w.frames[:2]
    dev = to_device(frames)
    v = w.voxel_size
    ref = gt.TsdfMap(v, w.truncation_voxels, w.max_weight)
    buf, head, full = _buffers()
    torch.cuda.synchronize()
    for k, (f, d) in enumerate(zip(frames, dev)):
        ref.integrate(f.sensor, f.T, d)
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
                  torch.cuda.mem_get_info()[0])
        gt.integrate_depth_static(buf, v, w.truncation_voxels, w.max_weight, d,
                                  gt.pinhole(f.sensor), f.T)
        torch.cuda.synchronize()
        after = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
                 torch.cuda.mem_get_info()[0])
        if k > 0:  # the first call on a device may load the library's kernels
            assert after == before, f"call {k}: device memory changed {before} -> {after}"
        _tails_untouched(full, f"call {k}")
        rk, rD, rW = ref.export()
        sk, sD, sW = _decode(head)
        np.testing.assert_array_equal(sk, rk, err_msg=f"call {k}: block sets differ")
        np.testing.assert_array_equal(sW, rW, err_msg=f"call {k}: weights differ")
        np.testing.assert_array_equal(sD, rD, err_msg=f"call {k}: distances differ")
        rs = ref.stats()
        cnt = head["counters"].cpu().numpy()
        assert int(cnt[1]) == rs["voxel_updates"]
        assert int(cnt[4]) == k + 1  # integration launches
        assert int(cnt[7]) == rs["block_frame_pairs"]
    ref.close()


def test_static_entry_refuses_oversized_maps():
    buf, _, full = _buffers()
    buf.max_blocks = gt.STATIC_MAX_BLOCKS + 1
    buf.hash_capacity = 1 << 18
    w = synth.config_tiny()
    d = torch.from_numpy(w.frames[0].depth).cuda()
    with pytest.raises(gt.TsdfError) as e:
        gt.integrate_depth_static(buf, w.voxel_size, 4, 100.0, d, gt.pinhole(w.frames[0].sensor),
                                  w.frames[0].T)
    assert e.value.code == -3
    torch.cuda.synchronize()
    _tails_untouched(full, "refused call")

"""The fused launch form (TSDF_LAUNCH_FUSED): each sub-batch of an
integrate_batch call allocates and integrates in one persistent cooperative
launch with a bounded grid-wide wait between the two phases.

It must give the same map as the split form (an allocation launch and an
integration launch per sub-batch), bit for bit in every storage, alone and
under CUDA-graph replay, and the oracle's map within the usual bounds.  The
bounded wait is tested by making it run out (a test hook asks it to wait
for CTAs that do not exist): the launch skips its integration, the map
reports TSDF_ERR_TIMEOUT, the GPU stays usable and map_reset recovers.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from tests.runners import compare, run_oracle, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2311_00626_gb300 as gt  # noqa: E402

TIMEOUT = -4


def _integrate(frames, dev, v, mode, storage=gt.STORAGE_FP32, per_call=None, layer=gt.LAYER_TSDF):
    m = gt.TsdfMap(v, storage=storage, launch_mode=mode, layer=layer)
    descs = [gt.frame_desc(0, f.sensor, f.T, d) for f, d in zip(frames, dev)]
    k = per_call or len(descs)
    for s in range(0, len(descs), k):
        gt.integrate_batch([m.handle], descs[s:s + k])
    torch.cuda.synchronize()
    assert m.sync() == 0
    out, st = m.export(), m.stats()
    m.close()
    return out, st


def _same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("storage", [gt.STORAGE_FP32, gt.STORAGE_FP16, gt.STORAGE_FIXED16])
def test_fused_equals_split_room(storage):
    """64 room frames in one call: two sub-batches of 32."""
    w = synth.config_room(n_frames=300)
    frames = w.frames[100:164]
    dev = to_device(frames)
    a, sa = _integrate(frames, dev, w.voxel_size, gt.LAUNCH_SPLIT, storage)
    b, sb = _integrate(frames, dev, w.voxel_size, gt.LAUNCH_FUSED, storage)
    _same(a, b)
    for k in ("blocks", "voxel_updates", "block_visits", "launches", "block_frame_pairs"):
        assert sa[k] == sb[k], k
    assert sb["launches"] == 2


def test_fused_against_oracle():
    w = synth.config_room(n_frames=300)
    frames = w.frames[:12]
    got, st = _integrate(frames, to_device(frames), w.voxel_size, gt.LAUNCH_FUSED)
    orc, oc = run_oracle(frames, w.voxel_size)
    compare(got, orc, 1e-4 * float(np.float32(w.voxel_size)), "fused room12")
    assert st["voxel_updates"] == oc["total_updates"]


def test_fused_rig_graph_replay_equals_split():
    """Rig steps (four cameras of three sizes and a LiDAR, FP16), one call
    per step, captured in a CUDA graph in the fused form and replayed."""
    w = synth.config_rig(n_steps=200)
    frames = w.frames[:50]
    dev = to_device(frames)
    ref, _ = _integrate(frames, dev, w.voxel_size, gt.LAUNCH_SPLIT, gt.STORAGE_FP16, per_call=5)
    m = gt.TsdfMap(w.voxel_size, storage=gt.STORAGE_FP16, launch_mode=gt.LAUNCH_FUSED)
    descs = [gt.frame_desc(0, f.sensor, f.T, d) for f, d in zip(frames, dev)]

    def run():
        m.reset()
        for s in range(0, len(descs), 5):
            gt.integrate_batch([m.handle], descs[s:s + 5])

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        run()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run()
    g.replay()
    torch.cuda.synchronize()
    assert m.sync() == 0
    _same(ref, m.export())
    m.close()


def test_fused_host_staging_equals_split():
    w = synth.config_room(n_frames=300)
    frames = w.frames[:40]
    host = torch.from_numpy(np.stack([f.depth for f in frames])).pin_memory()
    staging = torch.empty(4 * 32 * host[0].numel() * 4, dtype=torch.uint8, device="cuda")
    out = []
    for mode in (gt.LAUNCH_SPLIT, gt.LAUNCH_FUSED):
        m = gt.TsdfMap(w.voxel_size, launch_mode=mode)
        descs = [gt.frame_desc_host(0, f.sensor, f.T, host[i]) for i, f in enumerate(frames)]
        gt.integrate_batch_host([m.handle], descs, staging)
        torch.cuda.synchronize()
        assert m.sync() == 0
        out.append(m.export())
        m.close()
    _same(out[0], out[1])


def test_fused_falls_back_for_other_layers():
    """An occupancy map in fused mode runs the two kernels: same result."""
    w = synth.config_room(n_frames=300)
    frames = w.frames[:8]
    dev = to_device(frames)
    a, _ = _integrate(frames, dev, w.voxel_size, gt.LAUNCH_SPLIT, layer=gt.LAYER_OCCUPANCY)
    b, _ = _integrate(frames, dev, w.voxel_size, gt.LAUNCH_FUSED, layer=gt.LAYER_OCCUPANCY)
    _same(a, b)


def test_fused_wait_runs_out_and_map_recovers():
    """The grid-wide wait is asked for one CTA more than the launch has: it
    gives up after its limit, the map reports TSDF_ERR_TIMEOUT and refuses
    further calls; after map_reset (and the hook off) the map integrates
    normally again, equal to a fresh split-form map."""
    w = synth.config_room(n_frames=300)
    frames = w.frames[:4]
    dev = to_device(frames)
    descs = [gt.frame_desc(0, f.sensor, f.T, d) for f, d in zip(frames, dev)]
    m = gt.TsdfMap(w.voxel_size, launch_mode=gt.LAUNCH_FUSED)
    gt.map_wait_test(m.handle, 1)
    gt.integrate_batch([m.handle], descs)
    torch.cuda.synchronize()
    assert m.sync() == TIMEOUT
    with pytest.raises(gt.TsdfError) as e:
        gt.integrate_batch([m.handle], descs)
    assert e.value.code == TIMEOUT
    gt.map_wait_test(m.handle, 0)
    m.reset()
    gt.integrate_batch([m.handle], descs)
    torch.cuda.synchronize()
    assert m.sync() == 0
    ref, _ = _integrate(frames, dev, w.voxel_size, gt.LAUNCH_SPLIT)
    _same(ref, m.export())
    with pytest.raises(gt.TsdfError):
        gt.map_wait_test(m.handle, -1)
    m.close()

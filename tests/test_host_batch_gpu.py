"""integrate_batch_host: images in pinned host memory, copied into a staging
buffer on a copy stream while the previous sub-batch integrates.  The map
must equal the device-input batch bit for bit, for contiguous and scattered
host images, with and without colour images."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from synth.configs import color_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2311_00626_gb300 as gt  # noqa: E402


@pytest.fixture(scope="module")
def room():
    w = synth.config_room(n_frames=300)
    return w, w.frames[:70]


def _device_batch(w, frames, **kw):
    m = gt.TsdfMap(w.voxel_size, **kw)
    dev = [torch.from_numpy(np.ascontiguousarray(f.depth)).cuda() for f in frames]
    gt.integrate_batch([m.handle], [gt.frame_desc(0, f.sensor, f.T, d) for f, d in zip(frames, dev)])
    torch.cuda.synchronize()
    out = m.export()
    m.close()
    return out


@pytest.mark.parametrize("layout,slots", [("contiguous", 2), ("scattered", 2), ("contiguous", 3),
                                          ("scattered", 4)])
def test_host_batch_equals_device_batch(room, layout, slots):
    w, frames = room
    ref = _device_batch(w, frames)
    if layout == "contiguous":
        host = torch.from_numpy(np.stack([f.depth for f in frames])).pin_memory()
        imgs = [host[i] for i in range(len(frames))]
    else:
        imgs = [torch.from_numpy(np.ascontiguousarray(f.depth)).pin_memory() for f in frames]
    m = gt.TsdfMap(w.voxel_size)
    staging = torch.empty(slots * 32 * 640 * 480 * 4, dtype=torch.uint8, device="cuda")
    descs = [gt.frame_desc_host(0, f.sensor, f.T, d) for f, d in zip(frames, imgs)]
    gt.integrate_batch_host([m.handle], descs, staging)
    # a second call reuses the staging buffer after the first one's work
    m2 = gt.TsdfMap(w.voxel_size)
    gt.integrate_batch_host([m2.handle], descs, staging)
    torch.cuda.synchronize()
    for mm in (m, m2):
        assert mm.sync() == 0
        for a, b in zip(mm.export(), ref):
            np.testing.assert_array_equal(a, b)
        mm.close()


def test_host_batch_colour(room):
    w, frames = room
    frames = frames[:40]
    cols = [color_image(f.sensor, f.T, f.depth, 3, i) for i, f in enumerate(frames)]
    md = gt.TsdfMap(w.voxel_size, layer=gt.LAYER_COLOR)
    dd = [torch.from_numpy(np.ascontiguousarray(f.depth)).cuda() for f in frames]
    cc = [torch.from_numpy(c.view(np.int32)).cuda() for c in cols]
    gt.integrate_batch([md.handle], [gt.frame_desc(0, f.sensor, f.T, d, c) for f, d, c in zip(frames, dd, cc)])
    mh = gt.TsdfMap(w.voxel_size, layer=gt.LAYER_COLOR)
    hd = [torch.from_numpy(np.ascontiguousarray(f.depth)).pin_memory() for f in frames]
    hc = [torch.from_numpy(c.view(np.int32)).pin_memory() for c in cols]
    staging = torch.empty(2 * 2 * 32 * 640 * 480 * 4, dtype=torch.uint8, device="cuda")
    gt.integrate_batch_host([mh.handle], [gt.frame_desc_host(0, f.sensor, f.T, d, c)
                                          for f, d, c in zip(frames, hd, hc)], staging)
    torch.cuda.synchronize()
    for a, b in zip(mh.export_color(), md.export_color()):
        np.testing.assert_array_equal(a, b)
    md.close()
    mh.close()


def test_host_batch_staging_too_small(room):
    w, frames = room
    m = gt.TsdfMap(w.voxel_size)
    host = [torch.from_numpy(np.ascontiguousarray(f.depth)).pin_memory() for f in frames[:40]]
    small = torch.empty(32 * 640 * 480 * 4, dtype=torch.uint8, device="cuda")  # one sub-batch only
    with pytest.raises(gt.TsdfError):
        gt.integrate_batch_host([m.handle], [gt.frame_desc_host(0, f.sensor, f.T, d)
                                             for f, d in zip(frames, host)], small)
    torch.cuda.synchronize()
    assert m.num_blocks() == 0
    m.close()


def test_stage_frames_copies_and_refuses_bad_arguments():
    """stage_frames enqueues each host image into its device slice (sizes
    from zero to a full 1280x720 image, slices out of order), and refuses
    null pointers and negative sizes before enqueuing anything."""
    rng = np.random.default_rng(7)
    sizes = [0, 4, 1000, 640 * 480, 1280 * 720, 37]
    host = [torch.from_numpy(rng.standard_normal(max(n, 1)).astype(np.float32)).pin_memory() for n in sizes]
    offs = np.cumsum([0] + [(max(n, 1) * 4 + 255) // 256 * 256 for n in sizes])
    dev = torch.zeros(int(offs[-1]) // 4, dtype=torch.float32, device="cuda")
    order = [3, 0, 5, 1, 4, 2]
    gt.stage_frames([host[i].data_ptr() for i in order], [dev.data_ptr() + int(offs[i]) for i in order],
                    [sizes[i] * 4 for i in order])
    torch.cuda.synchronize()
    for i, n in enumerate(sizes):
        got = dev[int(offs[i]) // 4: int(offs[i]) // 4 + n].cpu().numpy()
        np.testing.assert_array_equal(got, host[i][:n].numpy())
    assert float(dev[int(offs[0]) // 4]) == 0.0  # the zero-byte entry wrote nothing
    with pytest.raises(gt.TsdfError):
        gt.stage_frames([host[1].data_ptr(), 0], [dev.data_ptr(), dev.data_ptr()], [16, 16])
    with pytest.raises(gt.TsdfError):
        gt.stage_frames([host[1].data_ptr()], [dev.data_ptr()], [-4])
    gt.stage_frames([], [], [])  # nothing to do

"""GPU parity of the colour layer (Table I: colour fusion) against the FP64
oracle, through the C ABI.

Block sets and colour weights bit-exact (integers up to the maximum weight);
r, g, b within the FP32 error of a running average.  One update
C' = C + (c - C) / W' rounds about two units in the last place of a value
below 256 (ulp = 2^-16 in [128, 256)); the average scales the error carried
from earlier frames by W / W' < 1, so after n updates the carried error stays
below 2 ulp * (min(n, w_max) + 1).
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from synth.configs import Frame, color_image, pinhole

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2311_00626_gb300 as gt  # noqa: E402

ULP_255 = 2.0 ** -16


def tol_color(n_frames, wmax=100.0):
    return 2 * ULP_255 * (min(n_frames, wmax) + 1)


def _colors(frames, seed=3):
    return [color_image(f.sensor, f.T, f.depth, seed, i) for i, f in enumerate(frames)]


def _oracle(frames, colors, v, trunc=4, wmax=100.0):
    import oracle
    m = oracle.OracleMap(v, trunc, wmax)
    for f, c in zip(frames, colors):
        m.integrate_color(f.sensor, f.T, f.depth, c)
    keys, _, W = m.export()
    rgb = m.export_color()
    total = m.counters()["total_updates"]
    m.close()
    return keys, rgb, W, total


def _gpu(frames, colors, v, trunc=4, wmax=100.0, batch=1):
    m = gt.TsdfMap(v, trunc, wmax, layer=gt.LAYER_COLOR)
    dd = [torch.from_numpy(np.ascontiguousarray(f.depth)).cuda() for f in frames]
    cc = [torch.from_numpy(c.view(np.int32)).cuda() for c in colors]
    if batch == 1:
        for f, d, c in zip(frames, dd, cc):
            m.integrate_color(f.sensor, f.T, d, c)
    else:
        for s in range(0, len(frames), batch):
            descs = [gt.frame_desc(0, f.sensor, f.T, d, c)
                     for f, d, c in zip(frames[s:s + batch], dd[s:s + batch], cc[s:s + batch])]
            gt.integrate_batch([m.handle], descs)
    torch.cuda.synchronize()
    assert m.sync() == 0
    keys, rgb, W = m.export_color()
    k2, D2, W2 = m.export()
    np.testing.assert_array_equal(k2, keys)
    np.testing.assert_array_equal(W2, W)
    assert np.all(D2 == 0)
    stats = m.stats()
    return m, (keys, rgb, W), stats


def _compare(g, o, n_frames, label):
    gk, grgb, gW = g
    ok, orgb, oW, _ = o
    np.testing.assert_array_equal(gk, ok, err_msg=f"{label}: block sets differ")
    bad = np.count_nonzero(gW.astype(np.float64) != oW)
    assert bad == 0, f"{label}: {bad} colour weights differ"
    err = np.abs(grgb.astype(np.float64) - orgb)
    tol = tol_color(n_frames)
    assert err.max() <= tol, f"{label}: max colour error {err.max():.3e} > {tol:.3e}"
    assert np.all(grgb[oW == 0] == 0)
    assert (oW > 0).sum() > 1000, "too few coloured voxels for a meaningful test"
    return float(err.max())


@pytest.fixture(scope="module")
def room():
    w = synth.config_room(n_frames=70)
    return w, _colors(w.frames)


def test_color_room_one_frame_per_call(room):
    w, colors = room
    frames, cols = w.frames[:12], colors[:12]
    o = _oracle(frames, cols, w.voxel_size)
    m, g, stats = _gpu(frames, cols, w.voxel_size)
    _compare(g, o, len(frames), "color room12")
    assert stats["voxel_updates"] == o[3]
    m.close()


def test_color_room_batched_pipelined(room):
    """70 frames in one integrate_batch call: three pipelined sub-batches."""
    w, colors = room
    o = _oracle(w.frames, colors, w.voxel_size)
    m, g, stats = _gpu(w.frames, colors, w.voxel_size, batch=70)
    _compare(g, o, len(w.frames), "color room70 batched")
    assert stats["voxel_updates"] == o[3] and stats["launches"] == 3
    m.close()


def test_color_weight_cap_and_ragged_image():
    """A 37x23 image integrated 130 times: weights stop at w_max = 100 while
    the average keeps moving with weight 1 / 101."""
    cam = pinhole(37, 23, 30.0, 18.0, 11.0)
    prims = synth.configs.tiny_scene()
    T = np.eye(4)
    d = synth.configs.render_frame(prims, cam, T, {}, 0, 0)
    frames = [Frame(cam, T, d)] * 130
    colors = [color_image(cam, T, d, 9, i) for i in range(130)]
    o = _oracle(frames, colors, 0.05)
    m, g, _ = _gpu(frames, colors, 0.05, batch=32)
    assert g[2].max() == 100.0
    _compare(g, o, 130, "color cap")
    m.close()


def test_query_color_matches_export(room):
    w, colors = room
    m, (keys, rgb, W), _ = _gpu(w.frames[:8], colors[:8], w.voxel_size)
    v = float(np.float32(w.voxel_size))
    rng = np.random.default_rng(0)
    bi = rng.integers(0, len(keys), 4096)
    li = rng.integers(0, 512, 4096)
    lx, ly, lz = li % 8, (li // 8) % 8, li // 64
    pts = np.stack([(keys[bi, 0] * 8 + lx + 0.5) * v, (keys[bi, 1] * 8 + ly + 0.5) * v,
                    (keys[bi, 2] * 8 + lz + 0.5) * v], 1).astype(np.float32)
    P = torch.from_numpy(pts).cuda()
    out_rgb = torch.empty((len(pts), 3), dtype=torch.float32, device="cuda")
    out_w = torch.empty(len(pts), dtype=torch.float32, device="cuda")
    m.query_color(P, out_rgb, out_w)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out_rgb.cpu().numpy(), rgb[bi, li])
    np.testing.assert_array_equal(out_w.cpu().numpy(), W[bi, li])
    # a point far from every block reads zeros
    far = torch.tensor([[1e4, 1e4, 1e4]], dtype=torch.float32, device="cuda")
    m.query_color(far, out_rgb[:1], out_w[:1])
    assert out_rgb[:1].abs().sum().item() == 0 and out_w[0].item() == 0
    m.close()


def test_color_argument_errors(room):
    w, colors = room
    f = w.frames[0]
    d = torch.from_numpy(np.ascontiguousarray(f.depth)).cuda()
    c = torch.from_numpy(colors[0].view(np.int32)).cuda()
    cm = gt.TsdfMap(w.voxel_size, layer=gt.LAYER_COLOR)
    tm = gt.TsdfMap(w.voxel_size)
    err = gt.TsdfError
    with pytest.raises(err):  # a depth frame without colour into a colour map
        cm.integrate(f.sensor, f.T, d)
    with pytest.raises(err):  # colour into a TSDF map
        tm.integrate_color(f.sensor, f.T, d, c)
    with pytest.raises(err):  # a TSDF frame carrying colour
        gt.integrate_batch([tm.handle], [gt.frame_desc(0, f.sensor, f.T, d, c)])
    with pytest.raises(err):  # a colour map and a TSDF map in one batch
        gt.integrate_batch([cm.handle, tm.handle], [gt.frame_desc(0, f.sensor, f.T, d, c),
                                                    gt.frame_desc(1, f.sensor, f.T, d)])
    lid = synth.configs.lidar64(64, 16)
    r = torch.ones((16, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(err):  # LiDAR frames carry no colour
        gt.integrate_batch([cm.handle], [gt.frame_desc(0, lid, np.eye(4), r, c)])
    P = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    o1 = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(err):
        cm.query(P, o1, o1)
    with pytest.raises(err):
        tm.query_color(P, torch.zeros((1, 3), dtype=torch.float32, device="cuda"), o1)
    with pytest.raises(err):
        gt.map_export_color(tm.handle)
    torch.cuda.synchronize()
    assert cm.sync() == 0 and tm.sync() == 0 and cm.num_blocks() == 0 and tm.num_blocks() == 0
    cm.close()
    tm.close()

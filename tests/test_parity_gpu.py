"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Block sets and per-voxel weights must match bit-exactly; distances must lie
within 1e-4 voxel sizes for FP32 storage (pinhole).  LiDAR values carry the
FP32 error of ranges up to tens of metres (range and bilinear sample in
FP32), so their bound adds 4 ulp of the largest range to 1e-4 voxel sizes.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import synth
from synth.configs import Frame
from tests.runners import compare, compare_occupancy, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

# error reports (JSON lines) go to TSDF_TEST_REPORTS when it names a directory
REPORT = os.environ.get("TSDF_TEST_REPORTS", "")


def _record(name, stats):
    if REPORT and os.path.isdir(REPORT):
        with open(os.path.join(REPORT, "parity_errors.jsonl"), "a") as fh:
            fh.write(json.dumps({"case": name, **stats}) + "\n")


def tol_pinhole(v):
    return 1e-4 * float(np.float32(v))


def tol_lidar(v, r_max):
    return 1e-4 * float(np.float32(v)) + 4 * float(np.spacing(np.float32(r_max)))


def _rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def _parity(name, frames, v, tol, **kw):
    orc, oc = run_oracle(frames, v, trunc=kw.get("trunc", 4), lidar_nearest=kw.get("lidar_nearest", False),
                         guard=kw.get("guard", 0.0))
    gpu, gs, status = run_gpu(frames, v, **kw)
    assert status == 0, f"device status {status}"
    st = compare(gpu, orc, tol, name)
    assert gs["voxel_updates"] == oc["total_updates"], (gs, oc)
    # the allocator emitted exactly the oracle's cells (same walks), and every
    # frame's band set reached the integration (one (block, frame) pair each)
    if kw.get("walk_stats", True):
        assert gs["cells"] == oc["total_cells"], (gs, oc)
    assert gs["block_frame_pairs"] == oc["total_band_blocks"], (gs, oc)
    _record(name, st)
    st["oracle_counters"] = oc
    return st


# ------------------------------------------------------------------ pinhole

def test_tiny_plane_sphere():
    w = synth.config_tiny()
    st = _parity("tiny", w.frames, w.voxel_size, tol_pinhole(w.voxel_size))
    assert st["blocks"] > 50


@pytest.mark.parametrize("batch", [1, 8])
def test_benchmark_kernel_variants(batch):
    """Without walk counters the allocator runs the variants the benchmark
    times (pinhole-only, refined reciprocals): the tiny scene and room
    frames against the oracle, one frame per call and batched."""
    w = synth.config_tiny()
    _parity(f"tiny_bench_kernels_b{batch}", w.frames, w.voxel_size, tol_pinhole(w.voxel_size),
            batch=batch, walk_stats=False)
    r = synth.config_room(n_frames=300)
    _parity(f"room16_bench_kernels_b{batch}", r.frames[40:56], r.voxel_size, tol_pinhole(r.voxel_size),
            batch=batch, walk_stats=False)


@pytest.mark.parametrize("walk_stats", [True, False])
def test_walk_cap_long_band(walk_stats):
    """A 160-voxel truncation at 1 cm (band 3.2 m, 40 blocks deep): walks
    stop after kMaxCells = 32 cells on both sides, the same cells."""
    w = synth.config_tiny()
    st = _parity(f"walk_cap_ws{int(walk_stats)}", w.frames, 0.01, tol_pinhole(0.01), trunc=160,
                 walk_stats=walk_stats)
    assert st["oracle_counters"]["truncated_rays"] > 1000


@pytest.mark.parametrize("seed,origin", [(1, (103.7, -52.1, 7.3)), (3, (-2001.13, 17.9, -3.31))])
def test_tilted_plane_far_pose(seed, origin):
    rng = np.random.default_rng(seed)
    R = _rot(rng)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = origin
    n = R[:, 2] + 0.4 * rng.normal(size=3)
    n /= np.linalg.norm(n)
    c = float(n @ (T[:3, 3] + 1.7 * R[:, 2]))
    cam = synth.pinhole(40, 30, 30.0)
    prims = synth.scene(synth.prim(synth.PLANE, *n, c))
    d = synth.render_pinhole(prims, T, cam["fu"], cam["fv"], cam["cu"], cam["cv"], 40, 30,
                             max_depth=6.0)
    _parity(f"tilted{seed}", [Frame(cam, T, d)], 0.05, tol_pinhole(0.05))


def test_tiny_rotation_entries_ieee_reciprocals():
    """A camera rotated by 1e-37 rad about x: the ray-direction terms fall
    below the range where the kernels' fast reciprocal is exact (2^-126), so
    the host selects the IEEE-reciprocal kernels for the frame; the result
    still equals the oracle's.  A second frame of ordinary pose in the same
    batch makes the whole batch take the IEEE kernels."""
    eps = 1e-37
    T = np.eye(4)
    T[1, 1] = T[2, 2] = np.cos(eps)
    T[1, 2], T[2, 1] = -np.sin(eps), np.sin(eps)
    T[:3, 3] = (0.31, -0.17, 0.05)
    cam = synth.pinhole(48, 36, 40.0)
    prims = synth.scene(synth.prim(synth.PLANE, 0.0, 0.0, 1.0, 2.1),
                        synth.prim(synth.SPHERE, 0.2, 0.1, 1.6, 0.3))
    frames = []
    for Tk in (T, _plain_pose()):
        d = synth.render_pinhole(prims, Tk, cam["fu"], cam["fv"], cam["cu"], cam["cv"], 48, 36,
                                 max_depth=6.0)
        frames.append(Frame(cam, Tk, d))
    _parity("tiny_rotation", frames[:1], 0.05, tol_pinhole(0.05))
    _parity("tiny_rotation_batch", frames, 0.05, tol_pinhole(0.05), batch=2)


def _plain_pose():
    T = np.eye(4)
    T[:3, 3] = (0.05, 0.02, -0.1)
    return T


def test_room_frames_640x480():
    """Twelve full-size frames of the room sequence (several thousand blocks,
    many CTAs and warps per frame, ragged last CTA of pixels)."""
    w = synth.config_room(n_frames=300)
    frames = w.frames[:12]
    st = _parity("room12", frames, w.voxel_size, tol_pinhole(w.voxel_size))
    assert st["blocks"] > 2000


@pytest.mark.parametrize("W,H", [(37, 23), (1, 1), (333, 7)])
def test_ragged_image_sizes(W, H):
    prims = synth.room_scene(3)
    Ts = synth.trajectory(3, prims, 4)
    cam = synth.pinhole(W, H, 0.8 * max(W, H))
    frames = [Frame(cam, T, synth.render_frame(prims, cam, T, synth.configs.ROOM_NOISE, 3, i))
              for i, T in enumerate(Ts)]
    _parity(f"ragged{W}x{H}", frames, 0.04, tol_pinhole(0.04))


def test_invalid_and_empty_frames():
    """Non-finite, negative and zero depths are invalid; an all-invalid frame
    allocates nothing."""
    cam = synth.pinhole(64, 48, 50.0, 32.0, 24.0)
    rng = np.random.default_rng(1)
    d = rng.uniform(0.5, 3.0, (48, 64)).astype(np.float32)
    d[rng.uniform(size=d.shape) < 0.3] = np.nan
    d[rng.uniform(size=d.shape) < 0.1] = np.inf
    d[rng.uniform(size=d.shape) < 0.1] = -1.0
    empty = np.zeros((48, 64), np.float32)
    frames = [Frame(cam, np.eye(4), empty), Frame(cam, np.eye(4), d)]
    _parity("invalid", frames, 0.05, tol_pinhole(0.05))
    gpu, gs, status = run_gpu([frames[0]], 0.05)
    assert status == 0 and len(gpu[0]) == 0 and gs["voxel_updates"] == 0


def test_weight_cap_repeated_frame():
    """150 repetitions of one frame: weights saturate at max_weight = 100."""
    w = synth.config_tiny()
    frames = w.frames * 150
    _parity("repeat150", frames, w.voxel_size, tol_pinhole(w.voxel_size))
    gpu, _, _ = run_gpu(frames, w.voxel_size)
    assert set(np.unique(gpu[2]).tolist()) <= {0.0, 100.0}


def test_batched_equals_sequential_and_oracle():
    """integrate_batch with 8 frames per launch gives the same map, bit for
    bit, as one frame per launch, and matches the oracle."""
    w = synth.config_room(n_frames=300)
    frames = w.frames[40:64]
    seq, _, _ = run_gpu(frames, w.voxel_size)
    bat, _, st = run_gpu(frames, w.voxel_size, batch=8)
    assert st == 0
    for a, b in zip(seq, bat):
        np.testing.assert_array_equal(a, b)
    orc, _ = run_oracle(frames, w.voxel_size)
    _record("batched8", compare(bat, orc, tol_pinhole(w.voxel_size), "batched8"))


def test_pipelined_batch_equals_sequential():
    """One integrate_batch call with 70 frames: three sub-batches whose
    allocations overlap the previous sub-batch's integration on a second
    stream (alternating mask / list sets); the map equals one frame per
    launch bit for bit."""
    w = synth.config_room(n_frames=300)
    frames = w.frames[100:170]
    seq, _, _ = run_gpu(frames, w.voxel_size)
    pip, stats, st = run_gpu(frames, w.voxel_size, batch=70)
    assert st == 0 and stats["launches"] == 3
    for a, b in zip(seq, pip):
        np.testing.assert_array_equal(a, b)
    orc, _ = run_oracle(frames, w.voxel_size)
    _record("pipelined70", compare(pip, orc, tol_pinhole(w.voxel_size), "pipelined70"))


def test_multi_map_batch():
    """One launch over three maps with different voxel sizes and interleaved
    frames: each map equals its own one-frame-per-launch result."""
    import paper_2311_00626_gb300 as gt
    from tests.runners import to_device
    sizes = [0.02, 0.05, 0.1]
    seqs = []
    for k in range(3):
        prims = synth.room_scene(50 + k)
        Ts = synth.trajectory(50 + k, prims, 6)
        cam = synth.configs.SERVING_SENSORS[k]
        seqs.append([Frame(cam, T, synth.render_frame(prims, cam, T, synth.configs.ROOM_NOISE,
                                                      50 + k, i)) for i, T in enumerate(Ts)])
    maps = [gt.TsdfMap(v) for v in sizes]
    order = [(k, i) for i in range(6) for k in range(3)]
    devs = {(k, i): to_device([seqs[k][i]])[0] for k, i in order}
    for s in range(0, len(order), 9):
        chunk = order[s:s + 9]
        descs = [gt.frame_desc(k, seqs[k][i].sensor, seqs[k][i].T, devs[(k, i)]) for k, i in chunk]
        gt.integrate_batch([m.handle for m in maps], descs)
    torch.cuda.synchronize()
    for k in range(3):
        assert maps[k].sync() == 0
        got = maps[k].export()
        ref, _, _ = run_gpu(seqs[k], sizes[k])
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b)
        orc, _ = run_oracle(seqs[k], sizes[k])
        compare(got, orc, tol_pinhole(sizes[k]), f"multimap{k}")
        maps[k].close()


def test_query_voxels_matches_export():
    import paper_2311_00626_gb300 as gt
    w = synth.config_tiny()
    (keys, D, W), _, _, m = run_gpu(w.frames, w.voxel_size, keep=True)
    v = float(np.float32(w.voxel_size))
    rng = np.random.default_rng(0)
    bi = rng.integers(0, len(keys), 4000)
    li = rng.integers(0, 512, 4000)
    loc = np.stack([li % 8, (li // 8) % 8, li // 64], 1)
    g = keys[bi].astype(np.int64) * 8 + loc
    pts = ((g + rng.uniform(0.2, 0.8, g.shape)) * v).astype(np.float32)
    far = np.array([[100.0, 100.0, 100.0], [-50.0, 3.0, 2.0]], np.float32)
    P = torch.from_numpy(np.concatenate([pts, far])).cuda()
    dist = torch.empty(len(P), device="cuda")
    wt = torch.empty(len(P), device="cuda")
    m.query(P, dist, wt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dist.cpu().numpy()[:4000], D[bi, li])
    np.testing.assert_array_equal(wt.cpu().numpy()[:4000], W[bi, li])
    assert np.all(wt.cpu().numpy()[4000:] == 0)
    m.close()


def test_capacity_error_is_reported():
    """A pool too small for the frame: map_sync reports TSDF_ERR_CAPACITY and
    later integrations are refused with the same status."""
    import paper_2311_00626_gb300 as gt
    w = synth.config_tiny()
    m = gt.TsdfMap(w.voxel_size, max_blocks=16)
    d = torch.from_numpy(w.frames[0].depth).cuda()
    m.integrate(w.frames[0].sensor, w.frames[0].T, d)
    assert m.sync() == -3
    with pytest.raises(gt.TsdfError):
        m.integrate(w.frames[0].sensor, w.frames[0].T, d)
    m.reset()
    torch.cuda.synchronize()
    assert m.sync() == 0
    m.close()


def test_argument_errors():
    import paper_2311_00626_gb300 as gt
    with pytest.raises(gt.TsdfError):
        gt.map_create(-1.0, 4, 100.0)
    m = gt.TsdfMap(0.05)
    cam = synth.pinhole(64, 48, 50.0)
    d = torch.zeros((48, 64), device="cuda")
    bad = np.eye(4)
    bad[0, 0] = 2.0  # not a rotation
    with pytest.raises(gt.TsdfError):
        m.integrate(cam, bad, d)
    with pytest.raises(gt.TsdfError):
        gt.integrate_depth(m.handle, 0, gt.pinhole(cam), np.eye(4))
    m.close()


def test_reset_then_reintegrate_is_identical():
    import paper_2311_00626_gb300 as gt
    w = synth.config_room(n_frames=300)
    frames = w.frames[:3]
    (a, _, _, m) = run_gpu(frames, w.voxel_size, keep=True)
    m.reset()
    from tests.runners import to_device
    for f, d in zip(frames, to_device(frames)):
        m.integrate(f.sensor, f.T, d)
    torch.cuda.synchronize()
    b = m.export()
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    m.close()


def test_graph_replay_of_overlapped_launches_equals_eager():
    """One-frame calls (and a one-sub-batch integrate_batch) launch their
    kernels as programmatic dependents of the stream's previous kernel;
    captured into a CUDA graph and replayed, they give the same map, bit for
    bit, as the same calls run eagerly."""
    import paper_2311_00626_gb300 as gt
    from tests.runners import to_device
    w = synth.config_room(n_frames=300)
    frames = w.frames[:24]
    dev = to_device(frames)

    def run(m):
        m.reset()
        for f, d in zip(frames[:12], dev[:12]):
            m.integrate(f.sensor, f.T, d)
        gt.integrate_batch([m.handle], [gt.frame_desc(0, f.sensor, f.T, d)
                                        for f, d in zip(frames[12:], dev[12:])])

    eager = gt.TsdfMap(w.voxel_size)
    run(eager)
    torch.cuda.synchronize()
    ref = eager.export()
    eager.close()
    m = gt.TsdfMap(w.voxel_size)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run(m)  # first calls outside the capture (lazy set-up)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run(m)
    g.replay()
    torch.cuda.synchronize()
    got = m.export()
    for x, y in zip(ref, got):
        np.testing.assert_array_equal(x, y)
    assert m.stats()["voxel_updates"] > 0
    m.close()


# -------------------------------------------------------------------- LiDAR

def _lidar_pose(seed):
    rng = np.random.default_rng(seed)
    T = np.eye(4)
    T[:3, :3] = _rot(rng)
    T[:3, 3] = rng.uniform(-50, 50, 3)
    return T


def test_lidar_inside_sphere():
    lid = synth.lidar64(n_az=128, n_el=16)
    img = np.full((16, 128), 10.0, np.float32)
    _parity("lidar_sphere", [Frame(lid, _lidar_pose(3), img)], 0.05, tol_lidar(0.05, 10.0))


def test_lidar_wrap_and_guard():
    lid = synth.lidar64(n_az=96, n_el=12)
    th = lid["theta_start"] + (np.arange(96) + 0.5) * 2 * math.pi / 96
    img = (8.0 + 0.06 * np.sin(th)[None, :] + 0.01 * np.arange(12)[:, None]).astype(np.float32)
    img[:, 20:40] += 3.0
    frames = [Frame(lid, _lidar_pose(4), img), Frame(lid, _lidar_pose(4), img)]
    _parity("lidar_wrap_guard", frames, 0.05, tol_lidar(0.05, 12.0))


def test_lidar_nearest_mode():
    lid = synth.lidar64(n_az=64, n_el=8)
    rng = np.random.default_rng(0)
    img = rng.uniform(5.0, 5.1, (8, 64)).astype(np.float32)
    _parity("lidar_nearest", [Frame(lid, _lidar_pose(6), img)], 0.05, tol_lidar(0.05, 5.1),
            lidar_nearest=True)


def test_lidar_outdoor_full_scan():
    """A full 1024x64 scan (0.5-30 m, noisy) of the seeded outdoor scene."""
    prims = synth.outdoor_scene(4)
    Ts = synth.trajectory(4, prims, 3, xy=(4.0, 36.0))
    lid = synth.lidar64()
    frames = []
    for i, T in enumerate(Ts):
        TL = synth.configs.rig_poses(T)[4]
        frames.append(Frame(lid, TL, synth.render_frame(prims, lid, TL, {"sigma": 0.02}, 4, i)))
    _parity("lidar_outdoor", frames, 0.05, tol_lidar(0.05, 30.0))


def test_rig_mixed_sensors_batched():
    """One step of the rig (four pinholes of three sizes plus the LiDAR) as a
    single batch equals the frames integrated one by one, and the oracle."""
    w = synth.config_rig(n_steps=2)
    seq, _, _ = run_gpu(w.frames, w.voxel_size)
    bat, _, st = run_gpu(w.frames, w.voxel_size, batch=5)
    assert st == 0
    for a, b in zip(seq, bat):
        np.testing.assert_array_equal(a, b)
    orc, _ = run_oracle(w.frames, w.voxel_size)
    _record("rig2", compare(bat, orc, tol_lidar(w.voxel_size, 30.0), "rig2"))


def test_far_segments_small_voxels():
    """Half-millimetre voxels: band segments start about 500 blocks from the
    sensor's block, beyond the allocator's short-key range, and take its
    full-key path.  At this voxel size 1e-4 voxels (5e-8 m) is finer than the
    FP32 spacing of a 2 m depth (2.4e-7 m), so the bound adds 2 ulp of the
    largest depth."""
    w = synth.config_tiny()
    tol = tol_pinhole(0.0005) + 2 * float(np.spacing(np.float32(2.0)))
    st = _parity("far_small_voxels", w.frames, 0.0005, tol)
    assert st["blocks"] > 1000


# --------------------------------------------------------------- occupancy

OCC = (float(np.float32(0.85)), float(np.float32(-0.4)))


def _occ_parity(name, frames, v, batch=1):
    orc, oc = run_oracle(frames, v, occupancy=OCC)
    gpu, gs, status = run_gpu(frames, v, occupancy=OCC, batch=batch)
    assert status == 0
    st = compare_occupancy(gpu, orc, len(frames), 0.85, name)
    assert gs["voxel_updates"] == oc["total_updates"]
    _record(name, st)
    return st


def test_occupancy_tiny_and_room():
    w = synth.config_tiny()
    _occ_parity("occ_tiny", w.frames, w.voxel_size)
    r = synth.config_room(n_frames=300)
    _occ_parity("occ_room12", r.frames[:12], r.voxel_size)


def test_occupancy_batched_pipelined():
    r = synth.config_room(n_frames=300)
    st = _occ_parity("occ_room40_piped", r.frames[60:100], r.voxel_size, batch=40)
    assert st["blocks"] > 2000


def test_occupancy_lidar():
    prims = synth.outdoor_scene(4)
    Ts = synth.trajectory(4, prims, 2, xy=(4.0, 36.0))
    lid = synth.lidar64()
    frames = []
    for i, T in enumerate(Ts):
        TL = synth.configs.rig_poses(T)[4]
        frames.append(Frame(lid, TL, synth.render_frame(prims, lid, TL, {"sigma": 0.02}, 4, i)))
    _occ_parity("occ_lidar", frames, 0.05)


def test_occupancy_decay_interleaved():
    """Occupancy decay (Sec. V-E) interleaved with integration: 10 room frames,
    2 decay steps, 10 more frames, 3 steps, against the oracle doing the
    same; the log-odds carry the FP32 error of a running sum of 25 terms."""
    import oracle
    import paper_2311_00626_gb300 as gt
    r = synth.config_room(n_frames=300)
    frames = r.frames[100:120]
    d_occ, d_free = float(np.float32(0.3)), float(np.float32(0.15))
    om = oracle.OracleMap(r.voxel_size)
    om.set_occupancy(*OCC)
    gm = gt.TsdfMap(r.voxel_size, layer=gt.LAYER_OCCUPANCY, l_occ=OCC[0], l_free=OCC[1])
    dev = [torch.from_numpy(np.ascontiguousarray(f.depth)).cuda() for f in frames]
    for part, steps in ((slice(0, 10), 2), (slice(10, 20), 3)):
        for f, d in zip(frames[part], dev[part]):
            om.integrate(f.sensor, f.T, f.depth)
            gm.integrate(f.sensor, f.T, d)
        for _ in range(steps):
            om.decay_occupancy(d_occ, d_free)
            gm.decay(d_occ, d_free)
    torch.cuda.synchronize()
    assert gm.sync() == 0
    st = compare_occupancy(gm.export(), om.export(), 25, 0.85, "occ_decay")
    assert st["blocks"] > 1000
    _record("occ_decay", st)
    ok, oL, oN = om.export()
    assert (oL > 0).any() and (oL < 0).any() and ((oL == 0) & (oN > 0)).any()
    with pytest.raises(gt.TsdfError):
        gm.decay(-0.1, 0.0)
    t = gt.TsdfMap(r.voxel_size)
    with pytest.raises(gt.TsdfError):  # not an occupancy layer
        t.decay(0.1, 0.1)
    t.close()
    gm.close()
    om.close()


# ------------------------------------------------------ weighting functions

@pytest.mark.parametrize("mode", [1, 2, 3])
def test_weighting_functions(mode):
    """Sensor-error weights f_w (inverse square depth, drop-off behind the
    surface, both).  Block sets exact.  Inverse square alone: weight sums
    within 1e-5 relative (FP32 sums of non-integer weights), distances within
    1e-4 voxel.  With the drop-off the weight depends on d_p itself, whose
    FP32 error (up to 4 ulp of the 5 m maximum depth, eps) moves each weight
    by up to eps / (tau - delta); the bounds add n eps / (tau - delta) to the
    weight sums and n eps / (tau - delta) * 2 tau / W to the distances (the
    sensitivity of a weighted mean), compared where W >= 0.05."""
    r = synth.config_room(n_frames=300)
    frames = r.frames[:24]
    n = len(frames)
    orc, oc = run_oracle(frames, r.voxel_size, weighting=mode)
    gpu, gs, status = run_gpu(frames, r.voxel_size, weighting=mode, batch=24)
    assert status == 0
    assert gs["voxel_updates"] == oc["total_updates"]
    if mode == 1:
        st = compare(gpu, orc, tol_pinhole(r.voxel_size), f"weighting{mode}", w_rtol=1e-5)
    else:
        (gk, gD, gW), (ok, oD, oW) = gpu, orc
        np.testing.assert_array_equal(gk, ok)
        v = float(np.float32(r.voxel_size))
        tau, delta = 4 * v, v
        eps = 4 * float(np.spacing(np.float32(5.0)))
        dw = n * eps / (tau - delta)
        werr = np.abs(gW.astype(np.float64) - oW)
        assert np.all(werr <= 1e-5 * oW + dw), werr.max()
        sel = oW >= 0.05
        derr = np.abs(gD.astype(np.float64) - oD)[sel]
        assert np.all(derr <= tol_pinhole(r.voxel_size) + dw * 2 * tau / oW[sel]), derr.max()
        st = {"blocks": len(gk), "max_err": float(derr.max()), "max_w_err": float(werr.max())}
    _record(f"weighting{mode}", st)

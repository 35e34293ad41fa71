"""Pins for the CPU oracle: closed forms, counting invariants, brute force.

Each test derives its expected values from the scene geometry and the
method's definition (nvblox Sec. IV-B, Eq. 1-3) with the independent FP64
helpers in refgeom.py, never from the oracle itself.  Voxels whose discrete
decisions (pixel rounding, image border, the d_p >= -tau test, LiDAR cell
choice) fall within a small margin of a tie are left out, since the oracle
takes those decisions in prescribed FP32 arithmetic.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth
from synth import PLANE, SPHERE, prim, scene
from tests import refgeom as G

F32 = lambda x: float(np.float32(x))  # noqa: E731


def _tau(v, trunc=4):
    return trunc * F32(v)


def _run(vox, frames, trunc=4, wmax=100.0):
    m = oracle.OracleMap(vox, trunc, wmax)
    for cam, T, d in frames:
        m.integrate(cam, T, d)
    return m


def _check_pinhole_single(cam, T, depth_expected, keys, D, W, v, tau, px_margin=1e-3,
                          dp_margin=1e-5, tol=1e-9):
    """Compare one-frame oracle output with the update rule evaluated in FP64
    on `depth_expected` (float32-rounded closed-form or brute-force depths)."""
    pL = G.voxel_centres(keys, v)
    pC = G.to_sensor(T, pL)
    i, j, inside, ok = G.pinhole_pixel(cam, pC, px_margin)
    ic = np.clip(i, 0, cam["width"] - 1)
    jc = np.clip(j, 0, cam["height"] - 1)
    d = depth_expected[jc, ic].astype(np.float64)
    valid = inside & (d > 0) & np.isfinite(d)
    dp = d - pC[..., 2]
    upd = valid & (dp >= -tau)
    ok &= ~valid | (np.abs(dp + tau) > dp_margin)
    W_exp = upd.astype(np.float64)
    D_exp = np.where(upd, np.minimum(dp, tau), 0.0)
    n_ok = int(ok.sum())
    assert n_ok > 0.9 * ok.size, "too many ambiguous voxels for a meaningful pin"
    np.testing.assert_array_equal(W[ok], W_exp[ok])
    np.testing.assert_allclose(D[ok], D_exp[ok], rtol=0, atol=tol)
    return int(upd[ok].sum())


def _check_blocks(keys, definite, possible):
    got = {tuple(k) for k in keys.tolist()}
    missing = definite - got
    extra = got - possible
    assert not missing, f"{len(missing)} blocks met by a band segment were not allocated"
    assert not extra, f"{len(extra)} allocated blocks are not met by any band segment"


# ---------------------------------------------------------------- pinhole


def test_plane_closed_form_identity():
    """Fronto-parallel plane z = 2 m seen from the identity pose: every pixel
    has depth 2, so D = min(2 - z_v, tau) and W = 1 wherever d_p >= -tau."""
    cam = synth.pinhole(64, 48, 50.0, 32.0, 24.0)
    prims = scene(prim(PLANE, 0, 0, 1, 2.0))
    T = np.eye(4)
    depth = synth.render_pinhole(prims, T, cam["fu"], cam["fv"], cam["cu"], cam["cv"], 64, 48)
    assert np.all(depth == np.float32(2.0))
    v = F32(0.05)
    tau = _tau(v)
    m = _run(0.05, [(cam, T, depth)])
    keys, D, W = m.export()
    # closed-form block set: blocks met by the segments z in [1.8, 2.2]
    definite, possible = G.pinhole_band_blocks(cam, T, np.full((48, 64), 2.0), tau, 8 * v)
    _check_blocks(keys, definite, possible)
    n = _check_pinhole_single(cam, T, np.full((48, 64), np.float32(2.0)), keys, D, W, v, tau)
    assert n == m.counters()["voxels_updated"]
    # every updated voxel in front of the band edge carries exactly +tau
    z = G.voxel_centres(keys, v)[..., 2]
    sel = (W == 1) & (z < 2.0 - tau - 1e-6)
    assert sel.sum() > 0 and np.all(D[sel] == tau)
    # occluded voxels (more than tau behind the surface) are never updated
    assert np.all(W[z > 2.0 + tau + 1e-6] == 0)


def _sphere_depth(cam, c, R, plane_z):
    """Closed-form z-depth per pixel: nearer of the sphere and plane hits."""
    H, W = cam["height"], cam["width"]
    jj, ii = np.mgrid[0:H, 0:W]
    r = np.stack([(ii - cam["cu"]) / cam["fu"], (jj - cam["cv"]) / cam["fv"], np.ones_like(ii, float)], -1)
    rr = (r * r).sum(-1)
    rc = (r * c).sum(-1)
    disc = rc * rc - rr * (c @ c - R * R)
    with np.errstate(invalid="ignore"):
        t = (rc - np.sqrt(disc)) / rr
    t = np.where(disc >= 0, t, np.inf)
    return np.minimum(t, plane_z).astype(np.float32)


def test_sphere_closed_form_tiny():
    """The tiny workload: plane z = 2 plus a sphere r = 0.3 at (0.2, 0.1, 1.5);
    the pixel depth is the smaller root of |t r - c|^2 = R^2 (r_z = 1)."""
    w = synth.config_tiny()
    f = w.frames[0]
    exp_depth = _sphere_depth(f.sensor, np.array([0.2, 0.1, 1.5]), 0.3, 2.0)
    np.testing.assert_allclose(f.depth, exp_depth, rtol=2e-7, atol=0)
    v = F32(w.voxel_size)
    tau = _tau(v)
    m = _run(w.voxel_size, [(f.sensor, f.T, f.depth)])
    keys, D, W = m.export()
    definite, possible = G.pinhole_band_blocks(f.sensor, f.T, exp_depth, tau, 8 * v)
    _check_blocks(keys, definite, possible)
    _check_pinhole_single(f.sensor, f.T, exp_depth, keys, D, W, v, tau)
    # the sphere produces distinct per-pixel depths, so pixel choice matters
    assert len(np.unique(exp_depth)) > 100


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


@pytest.mark.parametrize("seed,origin", [(1, (103.7, -52.1, 7.3)), (2, (-0.3, 0.2, -0.9)),
                                         (3, (-2001.13, 17.9, -3.31))])
def test_tilted_plane_general_pose(seed, origin):
    """Tilted plane seen from a general pose far from the origin (negative
    block coordinates, anchor-local arithmetic): closed-form depth
    t = (c - n.o) / (n . R r) per pixel."""
    rng = np.random.default_rng(seed)
    R = _random_rotation(rng)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = origin
    fwd = R[:, 2]
    n = fwd + 0.4 * rng.normal(size=3)
    n /= np.linalg.norm(n)
    c = float(n @ (T[:3, 3] + 1.7 * fwd))
    cam = synth.pinhole(40, 30, 30.0)
    prims = scene(prim(PLANE, *n, c))
    depth = synth.render_pinhole(prims, T, cam["fu"], cam["fv"], cam["cu"], cam["cv"], 40, 30,
                                 max_depth=6.0)
    jj, ii = np.mgrid[0:30, 0:40]
    r = np.stack([(ii - cam["cu"]) / cam["fu"], (jj - cam["cv"]) / cam["fv"], np.ones((30, 40))], -1)
    t_exp = (c - n @ T[:3, 3]) / ((r @ R.T) @ n)
    t_exp = np.where((t_exp > 0) & (t_exp <= 6.0), t_exp, 0.0).astype(np.float32)
    np.testing.assert_allclose(depth, t_exp, rtol=1e-6, atol=0)
    v = F32(0.05)
    tau = _tau(v)
    m = _run(0.05, [(cam, T, depth)])
    keys, D, W = m.export()
    definite, possible = G.pinhole_band_blocks(cam, T, t_exp, tau, 8 * v)
    _check_blocks(keys, definite, possible)
    _check_pinhole_single(cam, T, t_exp, keys, D, W, v, tau)


def test_brute_force_room_frame():
    """A small frame of the seeded room from a pose on its trajectory: the
    block set against a slab test over every pixel's band segment, and every
    voxel of every block against the update rule evaluated in FP64."""
    prims = synth.room_scene(7)
    Ts = synth.trajectory(7, prims, 5)
    cam = synth.pinhole(48, 36, 40.0)
    for T in Ts[::2]:
        depth = synth.render_frame(prims, cam, T, {"sigma_z2": 0.0012, "invalid_frac": 0.05,
                                                   "max_depth": 5.0}, 7, 0)
        v = F32(0.05)
        tau = _tau(v)
        m = _run(0.05, [(cam, T, depth)])
        keys, D, W = m.export()
        definite, possible = G.pinhole_band_blocks(cam, T, depth, tau, 8 * v)
        _check_blocks(keys, definite, possible)
        _check_pinhole_single(cam, T, depth, keys, D, W, v, tau)


def test_weight_counts_repeated_frame():
    """Integrating the same frame K = 150 times: W = min(K, 100) on every
    voxel the single frame updated, 0 elsewhere, and D unchanged."""
    w = synth.config_tiny()
    f = w.frames[0]
    m1 = _run(w.voxel_size, [(f.sensor, f.T, f.depth)])
    k1, D1, W1 = m1.export()
    mk = _run(w.voxel_size, [(f.sensor, f.T, f.depth)] * 150)
    kk, Dk, Wk = mk.export()
    np.testing.assert_array_equal(k1, kk)
    np.testing.assert_array_equal(Wk, np.where(W1 > 0, 100.0, 0.0))
    np.testing.assert_allclose(Dk, D1, rtol=0, atol=1e-12)
    assert mk.counters()["total_updates"] == 150 * m1.counters()["voxels_updated"]


def test_weighted_average_and_cap_closed_form():
    """60 frames at depth d1 then 40 at d2: D is the arithmetic mean of the
    truncated distances (W = 100); then 37 frames at d3: past the cap the
    average is an exponential one, D = s3 + (100/101)^37 (mean - s3)."""
    cam = synth.pinhole(32, 24, 25.0)
    T = np.eye(4)
    ds = [2.0, 2.03, 1.97]
    imgs = [synth.render_pinhole(scene(prim(PLANE, 0, 0, 1, d)), T, cam["fu"], cam["fv"],
                                 cam["cu"], cam["cv"], 32, 24) for d in ds]
    frames = [(cam, T, imgs[0])] * 60 + [(cam, T, imgs[1])] * 40
    m = _run(0.05, frames)
    keys, D, W = m.export()
    v = F32(0.05)
    tau = _tau(v)
    z = G.voxel_centres(keys, v)[..., 2]
    s = [np.minimum(float(np.float32(d)) - z, tau) for d in ds]
    pC = G.to_sensor(T, G.voxel_centres(keys, v))
    _, _, inside, ok = G.pinhole_pixel(cam, pC, 1e-3)
    sel = inside & ok & (z < 1.97 - tau - 0.01) | (inside & ok & (z > 1.5) & (z < 2.1))
    sel &= (float(np.float32(1.97)) - z >= -tau + 1e-5)
    assert sel.sum() > 100
    np.testing.assert_array_equal(W[sel], 100.0)
    np.testing.assert_allclose(D[sel], (60 * s[0][sel] + 40 * s[1][sel]) / 100, rtol=0, atol=1e-12)
    mean = D.copy()
    for _ in range(37):
        m.integrate(cam, T, imgs[2])
    keys2, D2, W2 = m.export()
    np.testing.assert_array_equal(keys, keys2)
    expect = s[2] + (100.0 / 101.0) ** 37 * (mean - s[2])
    np.testing.assert_array_equal(W2[sel], 100.0)
    np.testing.assert_allclose(D2[sel], expect[sel], rtol=0, atol=1e-12)


def test_dda_matches_slab_test():
    """The oracle's block traversal against a slab test on random segments."""
    rng = np.random.default_rng(11)
    B = 1.0
    n_checked = 0
    for _ in range(3000):
        o = rng.uniform(0, 1, 3).astype(np.float32)
        d = rng.normal(size=3).astype(np.float32) * rng.uniform(0.1, 3)
        if rng.uniform() < 0.2:
            d[rng.integers(3)] = 0.0  # axis-parallel segments
        s0 = np.float32(rng.uniform(0, 4))
        s1 = np.float32(s0 + rng.uniform(0, 2))
        cells = oracle.dda(o, d, float(s0), float(s1))
        got = {tuple(c) for c in cells.tolist()}
        definite, possible = G.segment_cells(o.astype(np.float64), d.astype(np.float64),
                                             float(s0), float(s1), B, 1e-4, 1e-5)
        assert definite <= got <= possible, (o, d, s0, s1)
        # cells are emitted as a face-connected walk
        steps = np.abs(np.diff(cells, axis=0)).sum(1)
        assert np.all(steps == 1)
        n_checked += 1
    assert n_checked == 3000


def _exact_walk(o, d, s0, s1):
    """Cells of o + s d, s in [s0, s1] (block units), in the order the
    segment enters them, in FP64.  None where FP32 rounding may decide
    otherwise: the start point within 1e-4 of a cell face, or two crossings
    (or a crossing and an end of the segment) closer than 1e-5 relative."""
    p = o + s0 * d
    if np.any(np.abs(p - np.round(p)) < 1e-4):
        return None
    c = np.floor(p).astype(np.int64)
    events = []
    for k in range(3):
        if d[k] == 0.0:
            continue
        step = 1 if d[k] > 0 else -1
        b = c[k] + (1 if step > 0 else 0)
        while True:
            t = (b - o[k]) / d[k]
            if t > s1 * (1 + 1e-5) + 1e-5:
                break
            events.append((t, k, step))
            b += step
    events.sort()
    ts = [s0] + [e[0] for e in events] + [s1]
    if any(b - a < 1e-5 * max(1.0, abs(b)) for a, b in zip(ts, ts[1:])):
        return None
    cells = [tuple(c)]
    for _, k, step in events:
        c[k] += step
        cells.append(tuple(c))
    return cells


def test_dda_cap_keeps_the_first_cells():
    """Segments of 20-80 blocks: the traversal stops after kMaxCells = 32
    cells, and those are the first 32 cells the segment enters (checked
    against an FP64 walk that orders every crossing exactly)."""
    rng = np.random.default_rng(12)
    checked = capped = 0
    for _ in range(1500):
        o = rng.uniform(0, 1, 3).astype(np.float32)
        d = (rng.normal(size=3) * rng.uniform(0.5, 3)).astype(np.float32)
        if rng.uniform() < 0.2:
            d[rng.integers(3)] = 0.0
        nd = float(np.linalg.norm(d.astype(np.float64)))
        s0 = np.float32(rng.uniform(0, 4))
        s1 = np.float32(s0 + rng.uniform(20, 80) / nd)
        exp = _exact_walk(o.astype(np.float64), d.astype(np.float64), float(s0), float(s1))
        if exp is None:
            continue
        got = [tuple(c) for c in oracle.dda(o, d, float(s0), float(s1)).tolist()]
        assert got == exp[:32], (o, d, s0, s1)
        checked += 1
        capped += len(exp) > 32
    assert checked >= 1000 and capped >= 900, (checked, capped)


def test_short_segments_stay_below_the_cap():
    """The allocation kernels drop the 32-cell cap for batches whose band
    segments span at most 8 blocks ((trunc / 4) |r| <= 8 on the host, r the
    widest pixel ray or a unit beam), on the bound that a segment of L blocks
    meets at most 7 + sqrt(3) (L + 0.06) cells under FP32 rounding (at most
    |dp_k| + 2 boundaries per axis).  Checked on the oracle's traversal with
    segments of exactly 8 blocks: random directions, the main diagonal (most
    crossings per length), starts a few ulp from block faces, and starts far
    from the anchor (coarse FP32 spacing)."""
    rng = np.random.default_rng(13)
    L = 8.0
    bound = 7 + np.sqrt(3.0) * (L + 0.06)
    worst = 0
    for it in range(6000):
        o = rng.uniform(0, 1, 3).astype(np.float32)
        kind = it % 3
        if kind == 0:
            d = rng.normal(size=3)
        else:  # close to a main diagonal
            d = rng.choice([-1.0, 1.0], 3) + rng.normal(scale=1e-3, size=3)
        d = (d / np.linalg.norm(d) * rng.uniform(0.2, 12.0)).astype(np.float32)
        nd = float(np.linalg.norm(d.astype(np.float64)))
        far = rng.uniform() < 0.3
        s0 = np.float32(rng.uniform(0, (200000.0 if far else 400.0) / nd))
        if kind == 2:  # start a few ulp off a block face on one axis
            k = int(rng.integers(3))
            p = np.float64(o[k]) + np.float64(s0) * np.float64(d[k])
            target = np.round(p) + rng.choice([-1, 1]) * rng.integers(0, 4) * np.spacing(np.float32(p))
            if d[k] != 0.0:
                s0 = np.float32(max(0.0, (target - np.float64(o[k])) / np.float64(d[k])))
        s1 = np.float32(np.float64(s0) + L / nd)
        n = len(oracle.dda(o, d, float(s0), float(s1)))
        worst = max(worst, n)
        assert n <= bound, (o, d, s0, s1, n)
    assert worst < 32 and worst >= 14, worst


# ------------------------------------------------------------------ LiDAR


def test_atan2_dec_error_bound():
    """The FP32 atan2 used for decisions stays within 4 ulp of atan2 and
    keeps the quadrant conventions of atan2."""
    rng = np.random.default_rng(5)
    ys = np.concatenate([rng.normal(size=20000) * 10 ** rng.uniform(-3, 3, 20000),
                         [0.0, 1.0, -1.0, 1.0, -1.0, 0.0, 3.0]]).astype(np.float32)
    xs = np.concatenate([rng.normal(size=20000) * 10 ** rng.uniform(-3, 3, 20000),
                         [1.0, 1.0, 1.0, -1.0, -1.0, -2.0, 0.0]]).astype(np.float32)
    worst = 0.0
    for y, x in zip(ys.tolist(), xs.tolist()):
        a = oracle.atan2_dec(y, x)
        e = math.atan2(y, x)
        ulp = np.spacing(np.float32(abs(e))) if e != 0 else np.float32(1e-45)
        err = abs(a - e) / float(ulp)
        worst = max(worst, err)
    assert worst <= 4.0, worst
    assert oracle.atan2_dec(0.0, -2.0) == F32(math.pi)
    assert oracle.atan2_dec(3.0, 0.0) == F32(math.pi / 2)


def _lidar_pose(seed):
    rng = np.random.default_rng(seed)
    T = np.eye(4)
    T[:3, :3] = _random_rotation(rng)
    T[:3, 3] = rng.uniform(-50, 50, 3)
    return T


def _check_lidar_single(lid, T, rng_img, keys, D, W, v, tau, guard, exp_fn=None, tol=1e-9):
    pC = G.to_sensor(T, G.voxel_centres(keys, v))
    u, vv, r = G.lidar_coords(lid, pC)
    d, valid, ok = G.lidar_bilinear(lid, rng_img, u, vv, guard)
    dp = d - r
    upd = valid & (dp >= -tau)
    ok &= ~valid | (np.abs(dp + tau) > 1e-5)
    assert ok.mean() > 0.9
    np.testing.assert_array_equal(W[ok], upd[ok].astype(float))
    D_exp = np.where(upd, np.minimum(dp, tau), 0.0)
    np.testing.assert_allclose(D[ok], D_exp[ok], rtol=0, atol=tol)
    return upd, ok


def test_lidar_inside_sphere_closed_form():
    """A LiDAR at the centre of a sphere of radius 10 m sees a constant range
    image, so bilinear sampling is exact and D = min(10 - |p|, tau)."""
    lid = synth.lidar64(n_az=128, n_el=16)
    T = _lidar_pose(3)
    img = np.full((16, 128), 10.0, np.float32)
    v = F32(0.05)
    tau = _tau(v)
    m = oracle.OracleMap(0.05)
    m.integrate(lid, T, img)
    keys, D, W = m.export()
    definite, possible = G.lidar_band_blocks(lid, T, img, tau, 8 * v)
    _check_blocks(keys, definite, possible)
    upd, ok = _check_lidar_single(lid, T, img, keys, D, W, v, tau, tau)
    r = np.linalg.norm(G.to_sensor(T, G.voxel_centres(keys, v)), axis=-1)
    sel = upd & ok
    np.testing.assert_allclose(D[sel], np.minimum(10.0 - r[sel], tau), rtol=0, atol=1e-9)
    assert sel.sum() > 1000


def test_lidar_bilinear_and_azimuth_wrap():
    """A smooth range image periodic in azimuth: the oracle's sample equals
    bilinear interpolation between the four surrounding beam centres,
    wrapping across the first/last column."""
    lid = synth.lidar64(n_az=96, n_el=12)
    T = _lidar_pose(4)
    k = np.arange(96)
    j = np.arange(12)
    th = lid["theta_start"] + (k + 0.5) * 2 * math.pi / 96
    img = (8.0 + 0.06 * np.sin(th)[None, :] + 0.02 * np.cos(th)[None, :]
           + 0.01 * j[:, None]).astype(np.float32)
    v = F32(0.05)
    tau = _tau(v)
    m = oracle.OracleMap(0.05)
    m.integrate(lid, T, img)
    keys, D, W = m.export()
    upd, ok = _check_lidar_single(lid, T, img, keys, D, W, v, tau, tau, tol=2e-6)
    pC = G.to_sensor(T, G.voxel_centres(keys, v))
    u, _, _ = G.lidar_coords(lid, pC)
    seam = (u - 0.5 < 0) | (u - 0.5 >= 95)
    assert (upd & ok & seam).sum() > 50, "no voxel sampled across the azimuth seam"


def test_lidar_guard_skips_fg_bg_edges():
    """A range step of 3 m between two halves of the image: voxels whose four
    neighbouring beams straddle the step are not updated (guard), the others
    are."""
    lid = synth.lidar64(n_az=64, n_el=8)
    T = _lidar_pose(5)
    img = np.full((8, 64), 6.0, np.float32)
    img[:, 20:40] = 9.0
    v = F32(0.05)
    tau = _tau(v)
    m = oracle.OracleMap(0.05)
    m.integrate(lid, T, img)
    keys, D, W = m.export()
    upd, ok = _check_lidar_single(lid, T, img, keys, D, W, v, tau, tau, tol=2e-6)
    pC = G.to_sensor(T, G.voxel_centres(keys, v))
    u, vv, r = G.lidar_coords(lid, pC)
    k0 = np.floor(u - 0.5).astype(int) % 64
    straddle = np.isin(k0, [19, 39]) & ok & (np.floor(vv - 0.5) >= 0) & (np.floor(vv - 0.5) <= 6)
    assert straddle.sum() > 20
    assert np.all(W[straddle] == 0)


def test_lidar_nearest_mode():
    """Nearest-cell sampling (test mode): the cell containing (u, v)."""
    lid = synth.lidar64(n_az=64, n_el=8)
    T = _lidar_pose(6)
    rng = np.random.default_rng(0)
    img = rng.uniform(5.0, 5.1, (8, 64)).astype(np.float32)
    v = F32(0.05)
    tau = _tau(v)
    m = oracle.OracleMap(0.05)
    m.set_lidar_sampling(nearest=True)
    m.integrate(lid, T, img)
    keys, D, W = m.export()
    pC = G.to_sensor(T, G.voxel_centres(keys, v))
    u, vv, r = G.lidar_coords(lid, pC)
    kk, jj = np.floor(u).astype(int), np.floor(vv).astype(int)
    fu, fv = u - kk, vv - jj
    ok = (np.minimum(fu, 1 - fu) > 1e-3) & (np.minimum(fv, 1 - fv) > 1e-3)
    inrow = (jj >= 0) & (jj < 8)
    d = img[np.clip(jj, 0, 7), kk % 64].astype(float)
    dp = d - r
    ok &= np.abs(dp + tau) > 1e-5
    upd = inrow & (dp >= -tau)
    np.testing.assert_array_equal(W[ok], upd[ok].astype(float))
    np.testing.assert_allclose(D[ok], np.where(upd, np.minimum(dp, tau), 0)[ok], atol=1e-9)


def test_lidar_brute_force_outdoor():
    """A LiDAR scan of the seeded outdoor scene: block set against the slab
    test over every beam's band segment; voxels against the guarded bilinear
    update rule in FP64."""
    prims = synth.outdoor_scene(9, n_boxes=60, n_cyl=20, size=(20.0, 20.0, 5.0))
    lid = synth.lidar64(n_az=180, n_el=16, max_range=30.0)
    T = np.eye(4)
    T[:3, 3] = [10.0, 10.0, 1.5]
    img = synth.render_frame(prims, lid, T, {"sigma": 0.0}, 9, 0)
    v = F32(0.1)
    tau = _tau(v)
    m = oracle.OracleMap(0.1)
    m.integrate(lid, T, img)
    keys, D, W = m.export()
    definite, possible = G.lidar_band_blocks(lid, T, img, tau, 8 * v)
    _check_blocks(keys, definite, possible)
    # the oracle takes the sample position (u, v) in FP32 (a decision input):
    # its error, below 1e-4 px at these image sizes, times the largest spread
    # the guard lets through (tau) bounds the difference to FP64 bilinear.
    _check_lidar_single(lid, T, img, keys, D, W, v, tau, tau, tol=1e-4 * tau)


# ------------------------------------------------------- occupancy layer

L_OCC, L_FREE = F32(0.85), F32(-0.4)


def test_occupancy_plane_closed_form():
    """Occupancy functor (Sec. IV-B): 7 frames of the plane z = 2 m then 5 at
    z = 2.12 m; a voxel in view adds l_free per frame that sees it in front
    of the surface (d_p > 0) and l_occ per frame that sees it within tau
    behind (-tau <= d_p <= 0); voxels further behind are never updated."""
    cam = synth.pinhole(64, 48, 50.0, 32.0, 24.0)
    T = np.eye(4)
    imgs = [synth.render_pinhole(scene(prim(PLANE, 0, 0, 1, z)), T, cam["fu"], cam["fv"],
                                 cam["cu"], cam["cv"], 64, 48) for z in (2.0, 2.12)]
    m = oracle.OracleMap(0.05)
    m.set_occupancy(L_OCC, L_FREE)
    for img in [imgs[0]] * 7 + [imgs[1]] * 5:
        m.integrate(cam, T, img)
    keys, L, N = m.export()
    v = F32(0.05)
    tau = _tau(v)
    pC = G.to_sensor(T, G.voxel_centres(keys, v))
    _, _, inside, ok = G.pinhole_pixel(cam, pC, 1e-3)
    z = pC[..., 2]
    exp_L = np.zeros_like(z)
    exp_N = np.zeros_like(z)
    for zs, k in ((float(np.float32(2.0)), 7), (float(np.float32(2.12)), 5)):
        dp = zs - z
        ok &= (np.abs(dp) > 1e-5) & (np.abs(dp + tau) > 1e-5)
        seen = inside & (dp >= -tau)
        exp_L += np.where(seen, k * np.where(dp > 0, L_FREE, L_OCC), 0.0)
        exp_N += np.where(seen, k, 0)
    assert ok.sum() > 0.9 * ok.size
    np.testing.assert_array_equal(N[ok], exp_N[ok])
    np.testing.assert_allclose(L[ok], exp_L[ok], rtol=0, atol=1e-12)
    # both signs and the mixed case occur
    assert (exp_L[ok] > 0).any() and (exp_L[ok] < 0).any()
    mixed = ok & (exp_N == 12) & (np.abs(exp_L - (7 * L_OCC + 5 * L_FREE)) < 1e-9)
    assert mixed.sum() > 0


def _decayed(L, k, d_occ, d_free):
    return np.where(L > 0, np.maximum(L - k * d_occ, 0.0), np.where(L < 0, np.minimum(L + k * d_free, 0.0), 0.0))


def test_occupancy_decay_closed_form():
    """Occupancy decay (Sec. V-E: dynamic content of an occupancy layer fades):
    after the two-plane sequence of the closed-form test above, k decay
    steps move occupied log-odds down by k * d_occ and free ones up by
    k * d_free, neither crossing 0; update counts are kept.  Checked after 3
    steps (no voxel reaches 0) and after 3 + 40 (every voxel at 0)."""
    cam = synth.pinhole(64, 48, 50.0, 32.0, 24.0)
    T = np.eye(4)
    imgs = [synth.render_pinhole(scene(prim(PLANE, 0, 0, 1, z)), T, cam["fu"], cam["fv"],
                                 cam["cu"], cam["cv"], 64, 48) for z in (2.0, 2.12)]
    m = oracle.OracleMap(0.05)
    m.set_occupancy(L_OCC, L_FREE)
    for img in [imgs[0]] * 7 + [imgs[1]] * 5:
        m.integrate(cam, T, img)
    _, L0, N0 = m.export()
    d_occ, d_free = F32(0.3), F32(0.15)
    for _ in range(3):
        m.decay_occupancy(d_occ, d_free)
    _, L3, N3 = m.export()
    np.testing.assert_array_equal(N3, N0)
    np.testing.assert_allclose(L3, _decayed(L0, 3, d_occ, d_free), rtol=0, atol=1e-12)
    moved = np.abs(L0) > 1.0
    assert (L0[moved] > 0).any() and (L0[moved] < 0).any()
    assert np.all(np.sign(L3[moved]) == np.sign(L0[moved]))  # nothing crossed 0 yet
    for _ in range(40):
        m.decay_occupancy(d_occ, d_free)
    _, L43, _ = m.export()
    assert np.all(L43 == 0.0)
    with pytest.raises(RuntimeError):
        m.decay_occupancy(-1.0, 0.0)
    t = oracle.OracleMap(0.05)
    with pytest.raises(RuntimeError):  # a TSDF layer has no decay
        t.decay_occupancy(0.1, 0.1)


def test_occupancy_lidar_sphere():
    """Inside a sphere of radius 10 m: voxels with |p| < 10 are free, those
    within tau outside it occupied, one observation each."""
    lid = synth.lidar64(n_az=128, n_el=16)
    T = _lidar_pose(3)
    img = np.full((16, 128), 10.0, np.float32)
    m = oracle.OracleMap(0.05)
    m.set_occupancy(L_OCC, L_FREE)
    m.integrate(lid, T, img)
    keys, L, N = m.export()
    v = F32(0.05)
    tau = _tau(v)
    pC = G.to_sensor(T, G.voxel_centres(keys, v))
    u, vv, r = G.lidar_coords(lid, pC)
    d, valid, ok = G.lidar_bilinear(lid, img, u, vv, tau)
    dp = d - r
    ok &= (np.abs(dp) > 1e-5) & (np.abs(dp + tau) > 1e-5)
    seen = valid & (dp >= -tau)
    np.testing.assert_array_equal(N[ok], seen[ok].astype(float))
    np.testing.assert_allclose(L[ok], np.where(seen, np.where(dp > 0, L_FREE, L_OCC), 0)[ok],
                               rtol=0, atol=1e-12)


# ---------------------------------------------------- weighting functions


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_weighted_average_closed_form(mode):
    """Sensor-error weights (Sec. IV-B, w = f_w(d_p)): two frames, the second
    taken 0.3 m further back and with the plane moved 6 cm, so the voxel
    depth d_v, the truncated distance s and the weight all differ between
    the frames; D must be the weighted mean (w_A s_A + w_B s_B) / (w_A + w_B)
    and W the weight sum, with w = 1 / d_v^2 (inverse square) and / or a
    linear drop-off from 1 at d_p = -delta to 0 at d_p = -tau."""
    cam = synth.pinhole(48, 36, 40.0)
    TA = np.eye(4)
    TB = np.eye(4)
    TB[2, 3] = -0.3
    imgA = synth.render_pinhole(scene(prim(PLANE, 0, 0, 1, 2.0)), TA, cam["fu"], cam["fv"],
                                cam["cu"], cam["cv"], 48, 36)
    imgB = synth.render_pinhole(scene(prim(PLANE, 0, 0, 1, 2.06)), TB, cam["fu"], cam["fv"],
                                cam["cu"], cam["cv"], 48, 36)
    v = F32(0.05)
    tau = _tau(v)
    delta = v
    m = oracle.OracleMap(0.05)
    m.set_weighting(mode)
    m.integrate(cam, TA, imgA)
    m.integrate(cam, TB, imgB)
    keys, D, W = m.export()
    pL = G.voxel_centres(keys, v)
    num = np.zeros(D.shape)
    den = np.zeros(D.shape)
    ok = np.ones(D.shape, bool)
    for T, img in ((TA, imgA), (TB, imgB)):
        pC = G.to_sensor(T, pL)
        i, j, inside, okp = G.pinhole_pixel(cam, pC, 1e-3)
        d = img[np.clip(j, 0, 35), np.clip(i, 0, 47)].astype(np.float64)
        dp = d - pC[..., 2]
        ok &= okp & (np.abs(dp + tau) > 1e-5) & (np.abs(dp + delta) > 1e-6)
        upd = inside & (dp >= -tau)
        w = np.ones(D.shape)
        if mode in (1, 3):
            w = w / pC[..., 2] ** 2
        if mode in (2, 3):
            w = np.where(dp < -delta, w * (tau + dp) / (tau - delta), w)
        num += np.where(upd, w * np.minimum(dp, tau), 0.0)
        den += np.where(upd, w, 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        D_exp = np.where(den > 0, num / den, 0.0)
    assert ok.mean() > 0.9
    np.testing.assert_allclose(W[ok], den[ok], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(D[ok], D_exp[ok], rtol=0, atol=1e-12)
    # the weights really vary: fractional weight sums occur
    assert np.any(np.abs(den[ok] - np.round(den[ok])) > 1e-3)


# ----------------------------------------------------------- colour layer


def _rgba(r, g, b):
    return (np.asarray(r, np.uint32) | (np.asarray(g, np.uint32) << 8)
            | (np.asarray(b, np.uint32) << 16) | np.uint32(255 << 24))


def test_color_closed_form():
    """Colour layer: voxels within tau of the surface (-tau <= d_p <= tau)
    take the colour of the pixel they project to, averaged over frames with
    weight 1; voxels further in front or behind are not coloured.  Two frames
    of the plane z = 2 m with colour images r = column, g = row, b = 40 and
    r = 200 - column, g = 2 row, b = 90: the colour is the per-channel mean."""
    cam = synth.pinhole(64, 48, 50.0, 32.0, 24.0)
    T = np.eye(4)
    depth = synth.render_pinhole(scene(prim(PLANE, 0, 0, 1, 2.0)), T, cam["fu"], cam["fv"],
                                 cam["cu"], cam["cv"], 64, 48)
    jj, ii = np.mgrid[0:48, 0:64]
    imgs = [_rgba(ii, jj, np.full_like(ii, 40)), _rgba(200 - ii, 2 * jj, np.full_like(ii, 90))]
    m = oracle.OracleMap(0.05)
    for img in imgs:
        m.integrate_color(cam, T, depth, img)
    keys, _, W = m.export()
    C = m.export_color()
    v = F32(0.05)
    tau = _tau(v)
    pC = G.to_sensor(T, G.voxel_centres(keys, v))
    i, j, inside, ok = G.pinhole_pixel(cam, pC, 1e-3)
    dp = float(np.float32(2.0)) - pC[..., 2]
    ok &= (np.abs(np.abs(dp) - tau) > 1e-5)
    col = inside & (np.abs(dp) <= tau)
    ic, jc = np.clip(i, 0, 63), np.clip(j, 0, 47)
    exp = np.stack([(ic + (200 - ic)) / 2.0, (jc + 2 * jc) / 2.0, np.full(ic.shape, 65.0)], -1)
    np.testing.assert_array_equal(W[ok], np.where(col, 2.0, 0.0)[ok])
    np.testing.assert_allclose(C[ok & col], exp[ok & col], rtol=0, atol=1e-12)
    assert np.all(C[ok & ~col] == 0)
    assert (ok & col).sum() > 1000 and (ok & ~col & inside).sum() > 1000

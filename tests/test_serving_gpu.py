"""Serving: continuous batching over several maps gives, for every map, the
same map as integrating its own frames alone, one frame per launch: bit for
bit with FP32 storage; with FP16 storage block sets and weights bit for bit
and distances within the FP16 bound, 2e-3 of the truncation distance (a
batch keeps a voxel in FP32 registers across its frames and rounds to FP16
once per launch, one frame per launch rounds after every frame).

Requests for four maps (three voxel sizes, FP16 storage) from pinhole
cameras of three resolutions and a LiDAR arrive as Poisson streams; the
server batches whatever has arrived, limited by frames per launch and by a
small staging budget so that admission has to wait for memory.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from synth.configs import ROOM_NOISE, SERVING_SENSORS, render_frame

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2311_00626_gb300 as gt  # noqa: E402
from paper_2311_00626_gb300.serving import Request, Server  # noqa: E402

SIZES = [0.02, 0.05, 0.1, 0.05]
N_PER_MAP = 6


def _streams(seed=11):
    rng = np.random.default_rng(seed)
    reqs = []
    for m, v in enumerate(SIZES):
        prims = synth.room_scene(100 + m)
        Ts = synth.trajectory(100 + m, prims, N_PER_MAP)
        t = 0.0
        for i in range(N_PER_MAP):
            t += rng.exponential(1 / 30.0)
            sensor = SERVING_SENSORS[(m + i) % len(SERVING_SENSORS)]
            T = Ts[i]
            if sensor["kind"] == "lidar":
                T = T.copy()
                T[:3, :3] = np.eye(3)  # LiDAR mounted level, z up
            d = render_frame(prims, sensor, T, ROOM_NOISE if sensor["kind"] == "pinhole"
                             else {"sigma": 0.02}, 100 + m, i)
            reqs.append(Request(len(reqs), m, sensor, T, torch.from_numpy(d).pin_memory(), t))
    reqs.sort(key=lambda r: r.arrival)
    return reqs


def _maps(storage):
    return [gt.TsdfMap(v, storage=storage) for v in SIZES]


def _alone(reqs, storage):
    maps = _maps(storage)
    for r in reqs:  # per-map order = arrival order
        maps[r.map_id].integrate(r.sensor, r.T, r.depth.cuda())
    torch.cuda.synchronize()
    out = [m.export() for m in maps]
    for m in maps:
        assert m.sync() == 0
        m.close()
    return out


@pytest.mark.parametrize("paced,storage", [(False, 0), (True, 0), (False, 1), (True, 1)])
def test_mix_equals_alone(paced, storage):
    reqs = _streams()
    ref = _alone(reqs, storage)
    maps = _maps(storage)
    # a staging budget of about three 1280x720 images forces admission waits
    srv = Server(maps, staging_bytes=3 * 1280 * 720 * 4 + 4096, max_frames=5)
    done = srv.run(reqs, paced=paced)
    assert len(done) == len(reqs)
    if not paced:
        assert srv.launches < len(reqs)  # all arrived at once: frames were batched
    for k, m in enumerate(maps):
        assert m.sync() == 0
        (gk, gD, gW), (rk, rD, rW) = m.export(), ref[k]
        np.testing.assert_array_equal(gk, rk)
        np.testing.assert_array_equal(gW, rW)
        if storage == gt.STORAGE_FP32:
            np.testing.assert_array_equal(gD, rD)
        else:
            tau = 4 * float(np.float32(SIZES[k]))
            assert np.abs(gD - rD).max() <= 2e-3 * tau
        m.close()
    lat = Server.latency_stats(done)
    if paced:
        assert lat["p50_ms"] >= 0 and lat["p99_ms"] >= lat["p50_ms"]

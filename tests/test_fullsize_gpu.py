"""Full-size parity: the whole 300-frame 640x480 room sequence, integrated in
the launch configuration the benchmark times (32 frames per integrate_batch
call), against the FP64 oracle over every voxel.

FP32 storage: block set and weights bit-exact, distances within 1e-4 voxel.
FP16 storage (D / tau and W as halves, FP32 arithmetic): block set and
weights bit-exact (weights are integers <= 100, exact in FP16), distance
error against the oracle reported and bounded by 2e-3 of the truncation
distance.
"""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import synth
from tests.runners import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

# error reports (JSON lines) go to TSDF_TEST_REPORTS when it names a directory
REPORT = os.environ.get("TSDF_TEST_REPORTS", "")
BATCH = 32


@pytest.fixture(scope="module")
def room():
    w = synth.config_room(n_frames=300)
    orc, counters = run_oracle(w.frames, w.voxel_size)
    return w, orc, counters


def _record(name, stats):
    if REPORT and os.path.isdir(REPORT):
        with open(os.path.join(REPORT, "precision.jsonl"), "a") as fh:
            fh.write(json.dumps({"case": name, **stats}) + "\n")


def test_room_300_frames_fp32(room):
    w, orc, oc = room
    gpu, gs, status = run_gpu(w.frames, w.voxel_size, batch=BATCH)
    assert status == 0
    st = compare(gpu, orc, 1e-4 * float(np.float32(w.voxel_size)), "room300_fp32")
    assert gs["voxel_updates"] == oc["total_updates"]
    assert gs["cells"] == oc["total_cells"]
    assert gs["block_frame_pairs"] == oc["total_band_blocks"]
    v = float(np.float32(w.voxel_size))
    _record("room300_fp32", {**st, "max_err_vox": st["max_err"] / v, "rms_err_vox": st["rms_err"] / v})


def test_room_300_frames_fp32_benchmark_kernels(room):
    """The kernel variants the benchmark times (no walk counters: the
    pinhole-only allocator with refined reciprocals) against the oracle."""
    w, orc, oc = room
    gpu, gs, status = run_gpu(w.frames, w.voxel_size, batch=BATCH, walk_stats=False)
    assert status == 0
    st = compare(gpu, orc, 1e-4 * float(np.float32(w.voxel_size)), "room300_fp32_bench_kernels")
    assert gs["voxel_updates"] == oc["total_updates"]
    assert gs["block_frame_pairs"] == oc["total_band_blocks"]
    assert gs["cells"] == 0  # the counting variant did not run
    _record("room300_fp32_bench_kernels", st)


def test_room_300_frames_one_call_pipelined(room):
    """All 300 frames in one integrate_batch call (ten pipelined sub-batches)."""
    w, orc, oc = room
    gpu, gs, status = run_gpu(w.frames, w.voxel_size, batch=300)
    assert status == 0 and gs["launches"] == 10
    st = compare(gpu, orc, 1e-4 * float(np.float32(w.voxel_size)), "room300_fp32_pipelined")
    assert gs["voxel_updates"] == oc["total_updates"]
    _record("room300_fp32_pipelined", st)


def test_room_300_frames_fp16(room):
    w, orc, oc = room
    gpu, gs, status = run_gpu(w.frames, w.voxel_size, storage=1, batch=BATCH)
    assert status == 0
    tau = 4 * float(np.float32(w.voxel_size))
    v = float(np.float32(w.voxel_size))
    st = compare(gpu, orc, 2e-3 * tau, "room300_fp16")
    assert gs["voxel_updates"] == oc["total_updates"]
    ok, oD, oW = orc
    obs = oW > 0
    near = obs & (np.abs(oD) < tau / 4)
    err = np.abs(gpu[1].astype(np.float64) - oD)
    _record("room300_fp16", {**st, "max_err_vox": st["max_err"] / v, "rms_err_vox": st["rms_err"] / v,
                             "max_err_tau": st["max_err"] / tau,
                             "near_surface_max_err_tau": float(err[near].max() / tau),
                             "near_surface_rms_err_tau": float(np.sqrt(np.mean(err[near] ** 2)) / tau)})


def test_room_300_frames_fixed16(room):
    """16-bit fixed-point storage (D / tau, FP16 weight) on the room sequence."""
    w, orc, oc = room
    gpu, gs, status = run_gpu(w.frames, w.voxel_size, storage=2, batch=BATCH)
    assert status == 0
    tau = 4 * float(np.float32(w.voxel_size))
    v = float(np.float32(w.voxel_size))
    st = compare(gpu, orc, 2e-3 * tau, "room300_fixed16")
    assert gs["voxel_updates"] == oc["total_updates"]
    ok, oD, oW = orc
    obs = oW > 0
    near = obs & (np.abs(oD) < tau / 4)
    err = np.abs(gpu[1].astype(np.float64) - oD)
    _record("room300_fixed16", {**st, "max_err_vox": st["max_err"] / v, "rms_err_vox": st["rms_err"] / v,
                                "max_err_tau": st["max_err"] / tau, "rms_err_tau": st["rms_err"] / tau,
                                "near_surface_max_err_tau": float(err[near].max() / tau),
                                "near_surface_rms_err_tau": float(np.sqrt(np.mean(err[near] ** 2)) / tau)})

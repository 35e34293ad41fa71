"""Run the same frames through the oracle and through the CUDA library."""
from __future__ import annotations

import numpy as np


def run_oracle(frames, voxel_size, trunc=4, wmax=100.0, lidar_nearest=False, guard=0.0,
               occupancy=None, weighting=0):
    import oracle
    m = oracle.OracleMap(voxel_size, trunc, wmax)
    if lidar_nearest or guard:
        m.set_lidar_sampling(lidar_nearest, guard)
    if occupancy is not None:
        m.set_occupancy(*occupancy)
    if weighting:
        m.set_weighting(weighting)
    cells = pairs = 0
    for f in frames:
        m.integrate(f.sensor, f.T, f.depth)
        c = m.counters()
        cells += c["candidates"]
        pairs += c["band_blocks"]
    out = m.export()
    counters = m.counters()
    counters["total_cells"] = cells
    counters["total_band_blocks"] = pairs
    m.close()
    return out, counters


def to_device(frames):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(f.depth)).cuda() for f in frames]


def run_gpu(frames, voxel_size, trunc=4, wmax=100.0, storage=0, batch=1, lidar_nearest=False,
            guard=0.0, max_blocks=0, keep=False, occupancy=None, weighting=0, walk_stats=True):
    """Integrate `frames` (in order) into a fresh map, `batch` frames per
    integrate_batch call (batch=1: integrate_depth / integrate_lidar).

    walk_stats: count walked cells (stats["cells"]), which selects the
    allocator variant with the counters; False runs the variants the
    benchmark times (pinhole-only batches, refined reciprocals where the
    host's range check allows) and leaves the cell count at 0."""
    import torch
    import paper_2311_00626_gb300 as gt
    occ = {} if occupancy is None else {"layer": gt.LAYER_OCCUPANCY, "l_occ": occupancy[0],
                                        "l_free": occupancy[1]}
    m = gt.TsdfMap(voxel_size, trunc, wmax, storage=storage, max_blocks=max_blocks,
                   lidar_nearest=lidar_nearest, lidar_guard=guard, weighting=weighting, **occ)
    if walk_stats:
        gt.map_walk_stats(m.handle, True)  # the tests compare walked cells with the oracle's
    dev = to_device(frames)
    if batch == 1:
        for f, d in zip(frames, dev):
            m.integrate(f.sensor, f.T, d)
    else:
        for s in range(0, len(frames), batch):
            descs = [gt.frame_desc(0, f.sensor, f.T, d)
                     for f, d in zip(frames[s:s + batch], dev[s:s + batch])]
            gt.integrate_batch([m.handle], descs)
    torch.cuda.synchronize()
    status = m.sync()
    out = m.export()
    stats = m.stats()
    if keep:
        return out, stats, status, m
    m.close()
    return out, stats, status


def compare(gpu, orc, tol_d, label="", w_rtol=0.0):
    """Block set and weights bit-exact (weights within w_rtol relative when
    they are not integers); distances within tol_d (metres) wherever the
    oracle's weight is nonzero; untouched voxels hold zeros."""
    gk, gD, gW = gpu
    ok, oD, oW = orc
    assert gk.shape == ok.shape, f"{label}: {len(gk)} blocks on the GPU, {len(ok)} in the oracle"
    np.testing.assert_array_equal(gk, ok, err_msg=f"{label}: block sets differ")
    if w_rtol:
        np.testing.assert_allclose(gW, oW, rtol=w_rtol, atol=0, err_msg=f"{label}: weights")
    else:
        bad = np.count_nonzero(gW.astype(np.float64) != oW)
        assert bad == 0, f"{label}: {bad} voxel weights differ"
    obs = oW > 0
    err = np.abs(gD[obs].astype(np.float64) - oD[obs]) if obs.any() else np.zeros(1)
    assert err.max() <= tol_d, f"{label}: max |dD| {err.max():.3e} > {tol_d:.3e}"
    assert np.all(gD[~obs] == 0)
    return {"blocks": len(gk), "observed": int(obs.sum()), "max_err": float(err.max()),
            "rms_err": float(np.sqrt(np.mean(err ** 2)))}


def compare_occupancy(gpu, orc, n_frames, l_max, label=""):
    """Block set bit-exact; log-odds within the FP32 error of a running sum
    of n_frames terms of magnitude <= l_max (n * ulp(n * l_max) / 2)."""
    gk, gL, _ = gpu
    ok, oL, oN = orc
    np.testing.assert_array_equal(gk, ok, err_msg=f"{label}: block sets differ")
    tol = n_frames * float(np.spacing(np.float32(n_frames * l_max))) / 2 + 1e-12
    err = np.abs(gL.astype(np.float64) - oL)
    assert err.max() <= tol, f"{label}: max |dL| {err.max():.3e} > {tol:.3e}"
    assert np.all(gL[oN == 0] == 0)
    return {"blocks": len(gk), "observed": int((oN > 0).sum()), "max_err": float(err.max()),
            "tol": tol}

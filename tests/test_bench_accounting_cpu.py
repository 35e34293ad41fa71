"""The benchmark's algorithmic-byte accounting for the derived layers, on CPU.

The rooflines of `bench.py --workload layers` divide these byte counts by
measured times, so the per-unit figures are pinned here: an FP32 TSDF block
is 512 voxels x {D, W} x 4 B, an ESDF state block 512 x 4 B, a block's six
faces 6 x 64 states, a triangle three FP32 vertices.
"""
from __future__ import annotations

import bench


def test_per_unit_sizes():
    assert bench.TSDF_BLOCK_B == 4096
    assert bench.ESDF_BLOCK_B == 2048
    assert bench.ESDF_FACES_B == 1536
    assert bench.TRI_POS_B == 36


def test_esdf_bytes_is_linear_in_each_count():
    # marking: TSDF read + state read + state write; sweep: state read + write;
    # exchange: the block's states + its six facing faces
    assert bench.esdf_bytes(1, 0, 0) == 4096 + 2 * 2048
    assert bench.esdf_bytes(0, 1, 0) == 2 * 2048
    assert bench.esdf_bytes(0, 0, 1) == 2048 + 1536
    m, s, p = 20369, 46749, 65445
    assert bench.esdf_bytes(m, s, p) == (m * bench.esdf_bytes(1, 0, 0) + s * bench.esdf_bytes(0, 1, 0)
                                         + p * bench.esdf_bytes(0, 0, 1))


def test_mesh_bytes():
    assert bench.mesh_bytes(1, 0) == 4096
    assert bench.mesh_bytes(0, 1) == 36
    assert bench.mesh_bytes(20369, 1168505) == 20369 * 4096 + 1168505 * 36


def test_alu_operation_counts_match_their_itemisation():
    """The ALU rooflines' algorithmic operation counts are the sums of the
    items listed beside them in bench.py."""
    segment = 6 + 3 + 3 + 3 + 6 + 3 * (2 + 1 + 1 + 2) + 7
    cell = 4 + 2 + 4 + 2
    projection = 2 + 3 + 1 + 6 + 5 + 3 + 1 + 1 + 3 + 7
    assert (bench.OPS_PER_SEGMENT, bench.OPS_PER_CELL, bench.OPS_PER_PROJECTION) == (segment, cell, projection)

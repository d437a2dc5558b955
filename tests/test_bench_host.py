"""Host-side pieces of bench.py (no GPU): the kernel-source hash that gates the
ncu figures, and the algorithmic byte counts it reports."""
from __future__ import annotations

import os
import shutil

import bench


def _copy_sources(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2111_14704_gb300", "csrc")
    dst = tmp_path / "paper_2111_14704_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("push_binned.cuh", "rsol_device.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    return dst


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    dst = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    p = dst / "push_binned.cuh"
    text = p.read_text()
    p.write_text("// a new comment line\n/* and a block\n   comment */\n" +
                 text.replace("namespace rsol {", "namespace rsol {  // trailing remark", 1) + "\n\n")
    assert bench.kernel_source_hash() == h0
    p.write_text(text.replace("namespace rsol {", "namespace rsol {\nconstexpr int unused_probe = 1;", 1))
    assert bench.kernel_source_hash() != h0


def test_algorithmic_bytes_of_the_push():
    # per packet: read cell 4 + offsets 12 + momenta 12 + weight 4, write 28;
    # per node: read six field components, write eight feedback densities
    assert bench.BYTES_PER_PACKET == 4 + 12 + 12 + 4 + 28
    assert bench.BYTES_PER_NODE == 6 * 4 + 8 * 4
    n_nodes = bench.GRID[0] * bench.GRID[1] * bench.GRID[2]
    per_packet = (bench.BYTES_PER_PACKET * bench.N_PARTICLES + bench.BYTES_PER_NODE * n_nodes) / bench.N_PARTICLES
    assert abs(per_packet - 67.0) < 1e-9  # 8 packets per cell: 60 + 56 / 8

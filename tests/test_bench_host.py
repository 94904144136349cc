"""Host-side logic of bench.py (no GPU): the kernel-source hashes that decide
whether a committed DRAM-traffic figure still belongs to the kernel being
timed, the reading of those figures from the profile summaries, and the FIFO
latency of the sequential serving arm."""
import os
import shutil

import pytest

import bench


def _copy_csrc(tmp_path):
    src = os.path.join(bench.ROOT, 'paper_1704_04551_gb300', 'csrc')
    dst = tmp_path / 'paper_1704_04551_gb300' / 'csrc'
    shutil.copytree(src, dst)
    return dst


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    dst = _copy_csrc(tmp_path)
    monkeypatch.setattr(bench, 'ROOT', str(tmp_path))
    h0 = bench.collide_source_sha()
    c0 = bench.couple_source_sha()
    p = dst / 'lbm.cu'
    text = p.read_text()
    p.write_text('// a new comment line\n' + text.replace('\n', '  // trailing note\n', 1))
    assert bench.collide_source_sha() == h0
    p.write_text(text.replace('COLLIDE_THREADS = 128', 'COLLIDE_THREADS = 256', 1))
    assert bench.collide_source_sha() != h0
    assert bench.couple_source_sha() == c0  # lbm.cu is not a source of the fused kernel


def test_committed_traffic_figures_match_the_current_sources():
    # the profiles in the repository were taken on the kernels as they are
    t32 = bench.collide_traffic('f32', 'tube256')
    t16 = bench.collide_traffic('f16', 'tube256_f16')
    tc = bench.couple_traffic(3000)
    assert t32 is not None and t16 is not None and tc is not None
    # DRAM traffic near the algorithmic bytes of a 256^3 tube launch (FP32
    # 1.93 GB, FP16 1.05 GB): no wasted re-reads
    assert 0.9 < t32 / 1.928e9 < 1.05
    assert 0.9 < t16 / 1.048e9 < 1.05
    # other workloads: no figure (their force-density share differs)
    assert bench.collide_traffic('f16', 'mix512') is None


def test_traffic_is_withheld_when_the_kernel_changed(tmp_path, monkeypatch):
    dst = _copy_csrc(tmp_path)
    shutil.copytree(os.path.join(bench.ROOT, 'profiles'), tmp_path / 'profiles')
    monkeypatch.setattr(bench, 'ROOT', str(tmp_path))
    assert bench.couple_traffic(10) is not None
    p = dst / 'couple.cu'
    p.write_text(p.read_text().replace('COUPLE_PER_THREAD = 2', 'COUPLE_PER_THREAD = 3', 1))
    assert bench.couple_traffic(10) is None


@pytest.mark.parametrize('arrivals,service,expected', [
    ([0.0, 0.0, 0.0], [1.0, 2.0, 3.0], [1.0, 3.0, 6.0]),   # burst: queueing adds up
    ([0.0, 5.0, 5.5], [1.0, 1.0, 1.0], [1.0, 1.0, 1.5]),   # idle server, then a wait
])
def test_fifo_latency(arrivals, service, expected):
    assert bench.fifo_latency(arrivals, service) == pytest.approx(expected)

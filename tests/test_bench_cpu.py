"""Host-side logic of bench.py that needs no GPU: workload names, algorithmic bytes, measured-traffic sources."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workload_names_state_the_shell_levels_and_precisions():
    for name, c in bench.CONFIGS.items():
        w = bench.workload_name(c)
        assert w.startswith('shell 6x%d^2x%d' % (c['Ns'], c['Nr']))
        assert 'FP64 residual' in w and 'FP64 outer FGMRES' in w and 'FGMRES(%d)' % c['restart'] in w
    assert '%d subdomains' % (6 * 6 * 6 * 8) in bench.workload_name(bench.CONFIGS['shell192'])
    assert 'three-level' in bench.workload_name(bench.CONFIGS['shell192'])


def test_algorithmic_bytes_of_the_bench_categories():
    """apply: read x and write y; the sweeps read more than the vector (factors) and the backward writes z."""
    c = dict(bench.CFG)
    N = 6 * c['Ns'] ** 2 * c['Nr']
    assert bench.algorithmic_bytes('apply_ppbe_fp32', c, N, 4) == 2 * 2 * N * 4
    assert bench.algorithmic_bytes('apply_vtbe', c, N, 8) == 2 * 7 * N * 8
    assert bench.algorithmic_bytes('apply_ppbe_coarse_fp32', c, N, 4) == 2 * 2 * (N // 8) * 4
    fwd = bench.algorithmic_bytes('ras_fwd_ppbe_coarse_fp32', c, N, 4)
    bwd = bench.algorithmic_bytes('ras_bwd_ppbe_coarse_fp32', c, N, 4)
    cp = c.get('coarse_p') or c['p']
    cells = bench.box_cells(c['Ns'] // 2, c['Nr'] // 2, cp, c['overlap_coarse'])
    assert cells > N // 8  # overlapping boxes hold more cells than the grid
    assert fwd == cells * (4 * (2 * 2 + 5 * 2 + 1) + 8)
    assert bwd == cells * (4 * (2 + 5 * 2 + 3) + 9) + (N // 8) * 2 * 4
    assert bench.algorithmic_bytes('net_fwd', c, N, 4) is None


def test_measured_traffic_entries_name_a_committed_capture_that_holds_the_figure():
    for cat, (nbytes, src) in bench.TRAFFIC.items():
        path = os.path.join(ROOT, src)
        assert src.startswith('profiles/') and os.path.exists(path), src
        assert str(nbytes) in open(path).read(), (cat, src)


def test_stable_dt_keeps_the_alfven_cfl_number_below_the_target():
    """dt = 0.9 / CFL_A(dt = 1) rounded down to two significant digits (paper Sec. 4.2 stability margin)."""
    assert bench.stable_dt(15671.774610187082) == 5.7e-05     # the 6 x 64^2 x 64 bench shell, seed 1
    for c in (3599.6, 7615.4, 23735.2, 31799.0, 41877.8, 1.0, 12345.678):
        dt = bench.stable_dt(c)
        assert 0.8 < c * dt <= bench.CFL_TARGET
        assert float('%.2g' % dt) == dt

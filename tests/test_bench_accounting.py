"""Host-side accounting of bench.py: the P2P pair count behind the roofline and the scaling of
the profiled DRAM traffic."""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
import workload as wl  # noqa: E402


def test_pair_count_one_ring_lattice():
    # 16^3 lattice, depth 2 (64 particles per leaf), one near ring and no correction ring:
    # every target meets the 27 leaves of its ring, 27 * 64 sources (self included)
    n = 16
    x = wl.lattice_positions(n)
    h = 2 * math.pi / n
    pairs, flops = bench.p2p_work(x, 2 * math.pi, 2, 1, h, Rc=0, rho_cut=5.0)
    assert pairs == n ** 3 * 27 * 64
    # all ring-1 octants are within 6.5 sigma of the target leaf: every pair is smoothed
    assert flops == bench.FLOPS_PER_PAIR * pairs


def test_pair_count_singular_octants_far_away():
    # the same lattice with a tiny core: every octant of the other leaves is >= 6.5 sigma
    # away (singular kernel); only the own leaf (gap 0) stays smoothed
    n = 16
    x = wl.lattice_positions(n)
    h = 2 * math.pi / n
    pairs, flops = bench.p2p_work(x, 2 * math.pi, 2, 1, 0.05 * h, Rc=0, rho_cut=5.0)
    own = n ** 3 * 64
    assert pairs == n ** 3 * 27 * 64
    assert flops == bench.FLOPS_PER_PAIR * own + bench.FLOPS_PER_PAIR_SINGULAR * (pairs - own)


def test_correction_ring_adds_only_close_octants():
    # ring 2 with rho_cut sigma below the cell-geometry gap of every ring-2 octant adds nothing
    n = 16
    x = wl.lattice_positions(n)
    h = 2 * math.pi / n
    base = bench.p2p_work(x, 2 * math.pi, 2, 1, h, Rc=0, rho_cut=5.0)
    none = bench.p2p_work(x, 2 * math.pi, 2, 1, h, Rc=2, rho_cut=4.0)   # ring-2 gaps are >= 5h
    some = bench.p2p_work(x, 2 * math.pi, 2, 1, h, Rc=2, rho_cut=5.5)
    assert none == base
    assert some[0] > base[0] and some[1] - base[1] == bench.FLOPS_PER_PAIR * (some[0] - base[0])


def test_profiled_traffic_scales_with_particles(tmp_path, monkeypatch):
    # the committed counters are valid only for the current source; they scale linearly
    t = bench.profiled_traffic("k_p2p_f32", ["p2p.cu"], 2 ** 21)
    if t is None:  # counters of another source revision: nothing to scale
        return
    t8 = bench.profiled_traffic("k_p2p_f32", ["p2p.cu"], 2 ** 24)
    assert np.isclose(t8, 8 * t)

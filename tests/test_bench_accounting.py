"""Host-side accounting of bench.py: the P2P pair count behind the roofline and the scaling of
the profiled DRAM traffic."""
import math
import os
import sys

import numpy as np
import pytest

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


def _half_cull_cases():
    n = 16
    h = 2 * math.pi / n
    lat = wl.lattice_positions(n)
    # random positions: leaves of 30 to 100 particles, so some leaves hold two 64-target chunks
    rnd = np.random.default_rng(7).uniform(0, 2 * math.pi, (n ** 3, 3))
    return [("lattice", lat, h), ("random", rnd, h)]


@pytest.mark.parametrize("case", ["lattice", "random"])
def test_correction_ring_half_cull_matches_brute_force(case):
    # ring 2 culled per (half of a 64-target chunk of a leaf, source octant): on the 16^3
    # lattice the halves are the leaf's two x-slabs, and a ring-2 octant on the +x side with
    # rho_cut = 5.5 is near only the upper slab; random positions add leaves of more than 64
    # particles (two chunks).  The count equals a direct loop over (target leaf, chunk, half,
    # ring-2 leaf, octant) with the same box gaps, and lies between the uncorrected count and
    # the count with the whole leaf's box
    name, x, h = [c for c in _half_cull_cases() if c[0] == case][0]
    L = 2 * math.pi
    base = bench.p2p_work(x, L, 2, 1, h, Rc=0, rho_cut=5.0)
    leafbox = bench.p2p_work(x, L, 2, 1, h, Rc=2, rho_cut=5.5, half_cull=False)
    half = bench.p2p_work(x, L, 2, 1, h, Rc=2, rho_cut=5.5, half_cull=True)
    assert base[0] < half[0] < leafbox[0]
    # direct count
    ns, w = 4, L / 4
    xf = np.mod(x, L).astype(np.float32).astype(np.float64)
    cell = np.clip((xf / w).astype(int), 0, ns - 1)
    octv = np.clip((xf / (w / 2)).astype(int) - 2 * cell, 0, 1)
    leaf = (cell[:, 0] * ns + cell[:, 1]) * ns + cell[:, 2]
    okey = octv[:, 0] * 4 + octv[:, 1] * 2 + octv[:, 2]
    cut2 = (5.5 * h) ** 2
    total = 0
    for lf in range(ns ** 3):
        idx = np.nonzero(leaf == lf)[0]
        idx = idx[np.lexsort((idx, okey[idx]))]         # the kernel's order within the leaf
        halves = [idx[k:k + 32] for k in range(0, len(idx), 32)]  # chunks of 64, halves of 32
        c = np.array([lf // (ns * ns), (lf // ns) % ns, lf % ns])
        for t in np.ndindex(5, 5, 5):
            o = np.array(t) - 2
            if np.abs(o).max() <= 1:
                continue
            nb = c + o
            src = (np.mod(nb[0], ns) * ns + np.mod(nb[1], ns)) * ns + np.mod(nb[2], ns)
            shift = np.floor_divide(nb, ns) * L
            sidx = np.nonzero(leaf == src)[0]
            for oc in range(8):
                so = sidx[okey[sidx] == oc]
                if len(so) == 0:
                    continue
                slo = xf[so].min(0) + shift
                shi = xf[so].max(0) + shift
                for hv in halves:
                    if len(hv) == 0:
                        continue
                    tlo, thi = xf[hv].min(0), xf[hv].max(0)
                    gap = np.maximum(0.0, np.maximum(slo - thi, tlo - shi))
                    if float((gap * gap).sum()) < cut2:
                        total += len(hv) * len(so)
    assert half[0] - base[0] == total

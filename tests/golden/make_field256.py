"""Write the oracle's values at sampled targets of the 256^3 benchmark field.

Calls only ``oracle`` and the input generator ``workload``.  Field: 256^3 lattice, k0 = 4,
seed 1, sigma = h (the benchmark workload).  Two target sets, both drawn with seeds:

* ``near``: 128 random particles (seed 3) and 32 particles within h of a face of the box
  (seed 5), with the direct FP64 sum over the central 27 boxes (K = 1);
* ``full``: the first 8 random and the first 8 face targets of ``near``, with in addition the
  far-image increment 2 <= max|n_i| <= 13 (singular kernel, exact there), so that
  near + far is the full 27^3-box sum of Section 4.1 that the benchmark's S = 2 handle computes.

Output: ``field256_k4_seed1.txt``, one row per target: particle index, face flag, u_K1 (3),
S_K1 (3), u_far (3), S_far (3) (nan where not computed).  Run time: the far increment is
16 x 16.8M x 19,656 singular pairs (hours on a few cores); the K = 1 part minutes.

    python tests/golden/make_field256.py [threads]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import workload as wl  # noqa: E402

N_SIDE, K0, SEED = 256, 4, 1
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "field256_k4_seed1.txt")


def face_targets(n, count, seed):
    """Seeded particles with a lattice index 0 or n - 1 on some axis (within h of a face)."""
    i = np.arange(n ** 3, dtype=np.int64)
    ix, iy, iz = i // (n * n), (i // n) % n, i % n
    on = ((ix == 0) | (ix == n - 1) | (iy == 0) | (iy == n - 1) | (iz == 0) | (iz == n - 1))
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(i[on], size=count, replace=False))


def targets():
    """(indices, face flags, full-set mask) in file order."""
    rnd = wl.target_subset(N_SIDE ** 3, 128, seed=3)
    fac = face_targets(N_SIDE, 32, seed=5)
    idx = np.concatenate([rnd, fac])
    face = np.concatenate([np.zeros(128, bool), np.ones(32, bool)])
    full = np.zeros(160, bool)
    full[:8] = True
    full[128:136] = True
    return idx, face, full


def load(path=OUT):
    """Read the file back: dict of index, face, u_near, S_near, u_far, S_far."""
    a = np.loadtxt(path)
    return {"index": a[:, 0].astype(np.int64), "face": a[:, 1] > 0.5, "u_near": a[:, 2:5],
            "S_near": a[:, 5:8], "u_far": a[:, 8:11], "S_far": a[:, 11:14]}


def main(threads=0):
    f = wl.make_vortex_lattice(N_SIDE, K0, SEED)
    x, g, s = f["x"], f["alpha"], f["sigma"]
    idx, face, full = targets()
    t = time.time()
    un, sn = oracle.direct(x, g, s, K=1, targets=idx, nthreads=threads)
    print("K=1 at %d targets: %.0f s" % (len(idx), time.time() - t), flush=True)
    uf = np.full((len(idx), 3), np.nan)
    sf = np.full((len(idx), 3), np.nan)
    t = time.time()
    sel = np.nonzero(full)[0]
    for k, i in enumerate(sel):
        uf[i], sf[i] = [a[0] for a in oracle.far_images(x, g, x[idx[i:i + 1]], g[idx[i:i + 1]], s, kmin=2, K=13,
                                                         nthreads=threads)]
        print("far increment %d/%d: %.0f s" % (k + 1, len(sel), time.time() - t), flush=True)
    rows = np.column_stack([idx, face.astype(float), un, sn, uf, sf])
    hdr = ("256^3 lattice, k0=4, seed 1, sigma=h, L=2pi: index face u_K1[3] S_K1[3] u_far[3] S_far[3]; "
           "far = image boxes 2<=max|n|<=13 (written by make_field256.py from oracle/ only)")
    np.savetxt(OUT, rows, fmt=["%d", "%d"] + ["%.17e"] * 12, header=hdr)
    print("wrote", OUT)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 0)

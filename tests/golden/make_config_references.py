"""Write the oracle's full-size, full-length references of the three large workloads.

For the 4096^2 HMF (unstable homogeneous waterbag, 1000 steps), the 2048^2 ring (1000 steps) and
the 4096^2 self-gravitating sheet (2000 steps) this runs the FP64 oracle (oracle/, Sec. 3 steps 1-4,
OpenMP on the host cores) from the shared seeded initial state and stores, in
tests/golden/config_<name>.npz:
  moments  [steps, 8]  (t, mass, Mx, My, kinetic, potential, energy, l2) after every step
  f200     f after 200 steps on the strided sub-grid rows[::64] x cols[::64]
  fend     the same after the last step
  stride   (64, 64)
Nothing here comes from the CUDA path.  About 45 minutes on 8 host cores.

    python tests/golden/make_config_references.py [name ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1206_3229_gb300 import inputs as I  # noqa: E402

STRIDE = 64
SNAP = 200


def grid_of(w):
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic, w.dt,
                  w.eps, w.G)


def make(w):
    g = grid_of(w)
    f = I.initial_state(w)
    t0 = time.time()
    f, m1 = O.run(g, f, SNAP)
    f200 = f[::STRIDE, ::STRIDE].copy()
    f, m2 = O.run(g, f, w.steps - SNAP)
    m2[:, 0] += SNAP * w.dt          # each oracle run counts time from its own start
    moments = np.concatenate([m1, m2])
    out = os.path.join(HERE, f"config_{w.name}.npz")
    np.savez_compressed(out, moments=moments, f200=f200, fend=f[::STRIDE, ::STRIDE].copy(),
                        stride=np.array([STRIDE, STRIDE]))
    print(f"{w.name}: {w.steps} steps in {time.time() - t0:.0f} s -> {out}", flush=True)


if __name__ == "__main__":
    O.set_threads(os.cpu_count() or 1)
    names = sys.argv[1:] or [I.RING_2048.name, I.HMF_4096_UNSTABLE.name, I.SHEET_4096.name]
    for n in names:
        make(I.WORKLOADS[n])

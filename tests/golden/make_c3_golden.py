"""Write tests/golden/c3_prefix.npz: the first NSTEPS steps of the c3
trajectory (N_b=8, 16x16 mesh, dt=0.02, U=1.5, driven, seed 2) from the FP64
CPU oracle. Calls only oracle/ and kbe_inputs/. Takes ~5 min on 8 cores.

Stored: obs [NSTEPS+1, 6]; nkb [NSTEPS+1, 256, 8]; the time-diagonal blocks
G^<(i,i), G^>(i,i) at i in DIAG; and NSAMP sampled entries (i, j, x, k, a, b)
-> value per row i in ROWS, drawn with seed 24680 uniformly over the row.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import kbe_inputs as ki  # noqa: E402
import oracle  # noqa: E402

NSTEPS = 24
DIAG = [1, 8, 16, 24]
ROWS = [4, 12, 20, 24]
NSAMP = 1024


def main(out=os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_prefix.npz"), threads=None):
    if threads:
        oracle.oracle.set_threads(int(threads))
    s = ki.config("c3")
    o = oracle.Oracle(s, nt_max=NSTEPS)
    rng = np.random.default_rng(24680)
    samples, values, diag = [], [], {}
    t0 = time.time()
    for n in range(1, NSTEPS + 1):
        o.step(1)
        if n in ROWS:
            lt, gt = o.row(n, 0), o.row(n, 1)
            for _ in range(NSAMP):
                j = int(rng.integers(0, n + 1))
                x = int(rng.integers(0, 2))
                k = int(rng.integers(0, s.nk))
                a, b = (int(v) for v in rng.integers(0, s.nb, 2))
                samples.append((n, j, x, k, a, b))
                values.append((lt if x == 0 else gt)[j, k, a, b])
        if n in DIAG:
            diag[n] = (o.block(n, n, 0), o.block(n, n, 1))
        print(f"step {n} {time.time() - t0:.0f}s", flush=True)
    obs = np.array([o.observables(n)[1] for n in range(NSTEPS + 1)])
    nkb = np.array([o.observables(n)[0] for n in range(NSTEPS + 1)])
    np.savez_compressed(out, obs=obs, nkb=nkb, samples=np.array(samples, np.int32),
                        values=np.array(values, np.complex128), diag_rows=np.array(DIAG),
                        diag_lesser=np.stack([diag[i][0] for i in DIAG]),
                        diag_greater=np.stack([diag[i][1] for i in DIAG]),
                        nsteps=NSTEPS, seconds=time.time() - t0, threads=oracle.oracle.threads())
    print("wrote", out, time.time() - t0)


if __name__ == "__main__":
    main(threads=sys.argv[1] if len(sys.argv) > 1 else None)

"""Write tests/golden/c2_full.npz: sampled G entries and all observables of
the full c2 trajectory (N_b=4, 8x8, N_t=512, dt=0.02, driven) from the FP64
CPU oracle. Calls only oracle/ and kbe_inputs/. Takes ~1-2 h on 8 cores.

Stored: obs [513, 6]; nkb [513, 64, 4]; G^<(i,i) and G^>(i,i) blocks at
i in DIAG; and 4096 sampled entries (i, j, x, k, a, b) -> value, drawn with
seed 12345 uniformly over the stored triangle of the last row set ROWS.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import kbe_inputs as ki  # noqa: E402
import oracle  # noqa: E402

DIAG = [64, 128, 256, 384, 512]
ROWS = [32, 100, 200, 300, 400, 480, 511, 512]
NSAMP = 512   # per row in ROWS


def main(out=os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_full.npz"), threads=None):
    if threads:
        oracle.oracle.set_threads(int(threads))
    s = ki.config("c2")
    o = oracle.Oracle(s)
    rng = np.random.default_rng(12345)
    samples, values, diag = [], [], {}
    t0 = time.time()
    for n in range(1, s.nt + 1):
        o.step(1)
        if n in ROWS:
            for _ in range(NSAMP):
                j = int(rng.integers(0, n + 1))
                x = int(rng.integers(0, 2))
                k = int(rng.integers(0, s.nk))
                a, b = (int(v) for v in rng.integers(0, s.nb, 2))
                samples.append((n, j, x, k, a, b))
                values.append(o.block(n, j, x)[k, a, b])
        if n in DIAG:
            diag[n] = (o.block(n, n, 0), o.block(n, n, 1))
        if n % 32 == 0:
            print(f"step {n} {time.time() - t0:.0f}s", flush=True)
    obs = np.array([o.observables(n)[1] for n in range(s.nt + 1)])
    nkb = np.array([o.observables(n)[0] for n in range(s.nt + 1)])
    np.savez_compressed(out, obs=obs, nkb=nkb, samples=np.array(samples, np.int32),
                        values=np.array(values, np.complex128), diag_rows=np.array(DIAG),
                        diag_lesser=np.stack([diag[i][0] for i in DIAG]),
                        diag_greater=np.stack([diag[i][1] for i in DIAG]),
                        seconds=time.time() - t0, threads=oracle.oracle.threads())
    print("wrote", out, time.time() - t0)


if __name__ == "__main__":
    main(threads=sys.argv[1] if len(sys.argv) > 1 else None)

"""Write oracle/c2_iterations.json: GMRES iteration counts of the FP64 oracle on the four c2
systems (128 x 128 Q1, M = 4, p = 3, ell = 0.5, field-split Gauss-Seidel + ILU(0), GMRES(restart),
relative residual 1e-10).  Used only to scale the timed CPU sample of bench.py to full solves.

    python oracle/c2_iterations.py [restart]      (default 300)

Calls nothing but the oracle.  Runs the four systems in parallel processes (about an hour of CPU).
"""

import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

SIGMAS = (0.25, 0.5, 1.0, 1.5)
RESTART = int(sys.argv[1]) if len(sys.argv) > 1 else 300


def solve(sigma):
    import oracle as O
    prob = O.build_problem(128, 4, 3, sigma=sigma, ell=0.5)
    blocks = O.fs_blocks(prob)
    N, P = prob.N, prob.P
    x, info = O.gmres(lambda v: O.sg_matvec(prob, v.reshape(N, P)).ravel(),
                      lambda v: O.fs_precond(prob, v.reshape(N, P), blocks=blocks).ravel(),
                      prob.F.ravel(), rtol=1e-10, restart=RESTART, max_iters=6000)
    return sigma, info["iters"], info["rel_resid"], info["converged"]


if __name__ == "__main__":
    import multiprocessing as mp
    with ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(solve, SIGMAS))
    out = {"restart": RESTART, "rtol": 1e-10,
           "iters": {str(s): it for s, it, _, _ in res},
           "rel_resid": {str(s): r for s, _, r, _ in res},
           "converged": {str(s): c for s, _, _, c in res}}
    with open(os.path.join(HERE, "c2_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))

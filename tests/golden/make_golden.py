"""Write oracle-only expected values for the GPU parity tests.

Every number stored here comes from the FP64 CPU oracle (``oracle``) on the
seeded synthetic designs of ``paper_2511_04025_b300.inputs``; nothing here
touches the CUDA library.  Run:  python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2511_04025_b300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    # 32^3, 8 charges +-1, VF 15 %: FP64 PCG case
    "plain32_s0": (lambda: inputs.plain_32(0), 32),
    "plain32_s1": (lambda: inputs.plain_32(1), 32),
    # 64^3, 32 charges N(0,1), VF 8 %: FP64 vs FP32 + refinement
    "gaussian64_s0": (lambda: inputs.gaussian_64(0), 64),
}


def make(name: str):
    mk, r = CASES[name]
    d = mk()
    t0 = time.time()
    res = oracle.homogenize(d, r, tol=1e-12)
    dt = time.time() - t0
    out = dict(
        name=name, r=r, t=res["t"], margin=res["margin"], n_solid=int(res["mask"].sum()),
        ambiguous=res["ambiguous"], C=res["C"].tolist(), Calt=res["Calt"].tolist(),
        iters=[int(i) for i in res["iters"]], relres=[float(x) for x in res["relres"]], status=int(res["status"]),
        oracle_seconds=dt, oracle_threads=oracle.num_threads(), tol=1e-12,
        source="oracle.homogenize (FP64 CPU), tests/golden/make_golden.py")
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, f"{dt:.1f}s", out["iters"], out["relres"], flush=True)


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(CASES)):
        make(n)

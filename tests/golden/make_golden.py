"""Write oracle-only expected values for the GPU parity tests.

Every number stored here comes from the FP64 CPU oracle (``oracle``) on the
seeded synthetic designs of ``paper_2511_04025_b300.inputs``; nothing here
touches the CUDA library.  Run:  python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np

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
    # 128^3, 48 charges on one O_h orbit, VF 5 %: FP32 + refinement at full size
    # (oracle PCG to 1e-11: each iteration streams a 4 GB block-CSR matrix)
    "cubic128_s0": (lambda: inputs.cubic_128(0), 128, 1e-11),
}


def make(name: str):
    mk, r, *rest = CASES[name]
    tol = rest[0] if rest else 1e-12
    d = mk()
    t0 = time.time()
    res = oracle.homogenize(d, r, tol=tol)
    dt = time.time() - t0
    out = dict(
        name=name, r=r, t=res["t"], margin=res["margin"], n_solid=int(res["mask"].sum()),
        ambiguous=res["ambiguous"], C=res["C"].tolist(), Calt=res["Calt"].tolist(),
        iters=[int(i) for i in res["iters"]], relres=[float(x) for x in res["relres"]], status=int(res["status"]),
        oracle_seconds=dt, oracle_threads=oracle.num_threads(), tol=tol,
        source="oracle.homogenize (FP64 CPU), tests/golden/make_golden.py")
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, f"{dt:.1f}s", out["iters"], out["relres"], flush=True)


# The active-set problem (Sec. 4.2.1: void culled, no ersatz floor) on the
# same designs.
ACTIVE_CASES = {
    "plain32_s0_active": (lambda: inputs.plain_32(0), 32, 1e-12),
    "gaussian64_s0_active": (lambda: inputs.gaussian_64(0), 64, 1e-12),
}


def make_active(name: str):
    mk, r, tol = ACTIVE_CASES[name]
    d = mk()
    t0 = time.time()
    res = oracle.homogenize_active(d, r, tol=tol)
    dt = time.time() - t0
    out = dict(
        name=name, r=r, t=res["t"], n_solid=int(res["mask"].sum()), pin=res["pin"],
        n_active_nodes=int(oracle.active_nodes(r, res["rho"]).sum()), C=res["C"].tolist(),
        iters=[int(i) for i in res["iters"]], relres=[float(x) for x in res["relres"]], status=int(res["status"]),
        oracle_seconds=dt, oracle_threads=oracle.num_threads(), tol=tol,
        source="oracle.homogenize_active (FP64 CPU), tests/golden/make_golden.py")
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, f"{dt:.1f}s", out["iters"], out["relres"], flush=True)


# Inverse-design gradient at full size: 64^3, 24 charges +-1, 10 % solid
# (t from the binary rule, then held fixed), smoothed density with
# kappa = ln(9) r, objective sum (C^H - C^T)^2 with C^T isotropic (bulk 0.05,
# shear 0.02), so dE/dC^H = 2 (C^H - C^T) at the oracle's own C^H.
GRAD_CASES = {
    "gradient64_s0": (lambda: inputs.gradient_64(0), 64, 1e-12),
}


def make_grad(name: str):
    mk, r, tol = GRAD_CASES[name]
    d = mk()
    t0 = time.time()
    t = oracle.voxelize(d, r)["t"]
    kap = oracle.default_kappa(r)
    F, gF = oracle.field_grid(d, r)
    rho = oracle.beta(oracle.distance(F, gF, d.iso), t, kap)
    u, iters, relres, st = oracle.solve(r, rho, tol=tol)
    C, _ = oracle.chom(r, rho, u)
    G = 2.0 * (C - inputs.isotropic_target())
    g = oracle.gradient_backward(d, r, G, t, kap, F, gF, rho, u)
    dt = time.time() - t0
    out = dict(
        name=name, r=r, t=t, kappa=kap, dEdC=G.tolist(), C=C.tolist(), g_pos=g["g_pos"].tolist(),
        g_q=g["g_q"].tolist(), g_alpha=g["g_alpha"].tolist(), g_iso=g["g_iso"], g_t=g["g_t"],
        objective=float(np.sum((C - inputs.isotropic_target()) ** 2)),
        iters=[int(i) for i in iters], relres=[float(x) for x in relres], status=int(st),
        oracle_seconds=dt, oracle_threads=oracle.num_threads(), tol=tol,
        source="oracle.solve/chom/gradient_backward (FP64 CPU), tests/golden/make_golden.py")
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, f"{dt:.1f}s", out["iters"], out["relres"], flush=True)


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(CASES) + list(GRAD_CASES) + list(ACTIVE_CASES)):
        if n in GRAD_CASES:
            make_grad(n)
        elif n in ACTIVE_CASES:
            make_active(n)
        else:
            make(n)

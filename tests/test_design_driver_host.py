"""Host logic of the inverse-design driver (design.py) with the library
calls replaced by a smooth model of C^H: the alternating schedule, the
evaluation count, alpha kept non-negative and moved downhill by the Adam
steps, positions wrapped into the cell, and an incumbent that the CMA-ES stage
never worsens.  The model: C^H isotropic with shear 0.02 and bulk
K = 0.05 + 0.01 c . alpha + 0.01 sum cos(2 pi x_m), V the target fraction."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_04025_b300 import design as design_mod  # noqa: E402
from paper_2511_04025_b300 import inputs, objectives, shl  # noqa: E402


def _iso(k, g):
    lam = k - 2.0 * g / 3.0
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[:3, :3] += 2.0 * g * np.eye(3)
    C[3:, 3:] = g * np.eye(3)
    return C


class FakeLibrary:
    def __init__(self, na, seed=0):
        self.c = np.random.default_rng(seed).standard_normal(na)
        self.tickets = {}
        self.calls = {"submit": 0, "grad": 0, "voxelize": 0}

    def bulk(self, d):
        return 0.05 + 0.01 * float(self.c @ d.alpha) + 0.01 * float(np.cos(2 * np.pi * d.pos[:, 0]).sum())

    def C(self, d):
        return _iso(self.bulk(d), 0.02)

    def serve_submit(self, h, d, r, opts, session=-1):
        assert d.vf is not None and d.t is None  # every candidate gets its thickness from the volume fraction
        self.calls["submit"] += 1
        t = len(self.tickets) + 1
        self.tickets[t] = self.C(d)
        return t

    def serve_wait(self, h, t):
        return {"C": self.tickets.pop(t), "stats": {"status": shl.SHL_OK}}

    def voxelize(self, h, d, r, **kw):
        self.calls["voxelize"] += 1
        return {"t": 0.02}

    def grad(self, h, d, r, opts, G, u=None, t=None, want_alpha=False, dEdV=0.0):
        self.calls["grad"] += 1
        dCdK = _iso(1.0, 0.0)  # C is linear in K
        g = float(np.sum(np.asarray(G) * dCdK)) * 0.01 * self.c if want_alpha else None
        return {"C": self.C(d), "V": d.vf, "g_alpha": g}


@pytest.fixture
def fake(monkeypatch):
    d = inputs.random_design(3, 6, 0.1)
    lib = FakeLibrary((d.K + 1) ** 3)
    monkeypatch.setattr(design_mod.shl, "shl_serve_submit", lib.serve_submit)
    monkeypatch.setattr(design_mod.shl, "shl_serve_wait", lib.serve_wait)
    monkeypatch.setattr(design_mod.shl, "shl_voxelize", lib.voxelize)
    monkeypatch.setattr(design_mod.shl, "shl_grad", lib.grad)
    return d, lib


def _driver(d, **kw):
    drv = design_mod.InverseDesign(handle=None, design=d, r=16, objective="Keff", vf=0.1, popsize=6, seed=1, **kw)
    drv._u = object()  # stands in for the device buffer of the forward displacements
    return drv


def test_schedule_and_evaluation_count(fake):
    d, lib = fake
    drv = _driver(d)
    hist = drv.run(outer=2, n_alpha=3, n_gen=2)
    assert hist.stage == ["alpha", "positions", "alpha", "positions"]
    assert hist.evaluations == 1 + 2 * (1 + 2 * 6) == lib.calls["submit"]
    assert lib.calls["grad"] == 2 * 3 * 2  # a forward and an adjoint call per Adam step
    assert np.all(np.isfinite(hist.objective))
    assert np.all(drv.design.alpha >= 0.0)
    assert np.all((drv.design.pos >= 0.0) & (drv.design.pos < 1.0))


def test_alpha_steps_go_downhill(fake):
    d, lib = fake
    drv = _driver(d, lr_alpha=0.02)
    k0 = lib.bulk(drv.design)
    drv.alpha_steps(5)
    assert lib.bulk(drv.design) > k0  # maximising K_eff / V
    # each weight moved along +c unless clamped at zero
    moved = drv.design.alpha - 1.0
    assert np.all((np.sign(moved) == np.sign(lib.c)) | (drv.design.alpha == 0.0))
    fn = objectives.objective("Keff")
    direct = float(fn(torch.tensor(lib.C(drv.design)), torch.tensor(0.1, dtype=torch.float64)))
    assert drv.value == pytest.approx(direct, rel=1e-12)


def test_position_stage_never_worsens_the_incumbent(fake):
    d, lib = fake
    drv = _driver(d, sigma0=0.05)
    before = drv.value
    drv.position_generations(4)
    assert drv.value <= before
    fn = objectives.objective("Keff")
    direct = float(fn(torch.tensor(lib.C(drv.design)), torch.tensor(0.1, dtype=torch.float64)))
    assert drv.value == pytest.approx(direct, rel=1e-12)

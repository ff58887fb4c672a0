"""GPU parity of the paper's comparison variants: the minimum-map complementarity functions
(App. B.1) and the mass-inverse complementarity preconditioner (Sec. 5.4), each against
the FP64 oracle run with the same option, and Sec. 7.5's stick-slip comparison."""
import json
import math
import os

import numpy as np
import pytest

import scenegen as sg
from oracle import Oracle, OracleOptions
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
VARIANTS = [("minmap", "delassus"), ("fb", "mass"), ("minmap", "mass")]


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_band(o, q, v, opts, n=3, eps=1e-6, seed=0):
    """The oracle's frame from (q, v) and its own spread under perturbations of q of the
    size of the FP32 global solve's error (eps relative to the position scale), max over n
    seeded draws: relative displacement, relative impulses, and per-residual absolute.
    The minimum map switches branches and the mass-preconditioned iteration cycles, so
    near a tie or on a cycle the exact answer moves by more than any FP32 path can match."""
    rng = np.random.default_rng(seed)
    base = o.frame(q, v, opts)
    dq, dl = 0.0, 0.0
    dr = np.zeros(len(base[2]["residuals"]))
    scale = np.abs(q).max()
    for _ in range(n):
        r = o.frame(q + eps * scale * rng.normal(size=q.shape), v, opts)
        if len(r[2]["contacts"]) != len(base[2]["contacts"]):
            continue
        dq = max(dq, _relerr(r[0] - q, base[0] - q))
        dl = max(dl, _relerr(r[2]["lam"], base[2]["lam"]))
        dr = np.maximum(dr, np.abs(np.array(r[2]["residuals"]) - base[2]["residuals"]))
    return base, dq, dl, dr


@pytest.mark.parametrize("ncp,precond", VARIANTS)
@pytest.mark.parametrize("model", [sg.MODEL_ARAP, sg.MODEL_SNH])
def test_variant_frame_matches_oracle(ncp, precond, model):
    sc = sg.cube_drop(m=6, model=model, height=-0.003, seed=2, mu=0.5)
    o = Oracle(sc)
    opts = OracleOptions(n_iters=5, n_cr=sc.n_cr, ncp=ncp, precond=precond)
    (q, v, info), band_q, band_l, band_r = _oracle_band(o, sc.q0, sc.v0, opts)
    sim = Simulator(sc, ncp=ncp, precond=precond)
    sim.set_state(sc.q0, sc.v0)
    sim.step(n_iters=5)
    qg, _ = sim.state()
    ct = sim.contacts()
    keys_o = [(c["vertex"], c["obstacle"]) for c in info["contacts"]]
    assert list(zip(ct["vertex"].tolist(), ct["obstacle"].tolist())) == keys_o
    assert len(keys_o) > 3
    assert _relerr(qg - sc.q0, q - sc.q0) < max(1e-4, 10 * band_q)
    assert _relerr(ct["lam"], info["lam"]) < max(1e-3, 10 * band_l)
    res = sim.stats()["residuals"]
    assert len(res) == len(info["residuals"])
    for rg, ro, br in zip(res, info["residuals"], band_r):
        assert abs(rg - ro) < 1e-4 + 0.05 * ro + 10 * br
    sim.close()


@pytest.mark.parametrize("ncp,precond", VARIANTS)
def test_variant_trajectory_resynchronised(ncp, precond):
    # 30 frames of the drop through impact, each GPU frame from the oracle's state. The
    # minimum map's branch switches and the mass-preconditioned iteration's two-cycles
    # amplify rounding within a frame (the oracle's own frames move by up to 1e-2 .. 0.8 of
    # the displacement under 1e-7 perturbations of its input), so these variants are held
    # to looser gates than the FB / Delassus path: displacement within 2e-2, penetration
    # within 1e-3 L, energy within 1e-2. The mass-preconditioned iteration does not
    # converge (it settles on a two-cycle, Sec. 5.4's point), so after 5 iterations its
    # frames differ by up to 0.1 of the displacement: there only penetration and energy
    # (5e-2) are gated and the displacement error is printed with the residual difference.
    sc = sg.cube_drop(m=5, seed=3, height=0.02, mu=0.4)
    o = Oracle(sc)
    opts = OracleOptions(n_iters=5, n_cr=sc.n_cr, ncp=ncp, precond=precond)
    sim = Simulator(sc, ncp=ncp, precond=precond)
    L = sc.bbox_diagonal
    q, v = sc.q0.copy(), sc.v0.copy()
    n_contact = 0
    worst = worst_r = 0.0
    for _ in range(30):
        sim.set_state(q, v)
        qn, vn, info = o.frame(q, v, opts)
        sim.step(n_iters=5)
        qg, vg = sim.state()
        err = _relerr(qg - q, qn - q)
        worst = max(worst, err)
        if precond != "mass":
            assert err < 2e-2
        assert abs(o.max_penetration(qg) - o.max_penetration(qn)) < 1e-3 * L
        e_o, e_g = o.energy(qn, vn), o.energy(qg, vg)
        assert abs(e_g - e_o) < (5e-2 if precond == "mass" else 1e-2) * max(abs(e_o), 1e-12)
        if info["contacts"]:
            n_contact += 1
            worst_r = max(worst_r, abs(sim.stats()["residuals"][-1] - info["residuals"][-1]))
        q, v = qn, vn
    assert n_contact > 10
    print(ncp, precond, "worst relative displacement error %.2e, residual difference %.1e"
          % (worst, worst_r))
    sim.close()


def _gpu_slope_acceleration(gold, dmu, T=1.0, **kw):
    th = math.radians(gold["theta_deg"])
    down = np.array([math.cos(th), 0.0, -math.sin(th)])
    sc = sg.slope_box(mu=gold["mu_star"] + dmu, theta_deg=gold["theta_deg"],
                      rho=gold["density"], E=gold["youngs_modulus"])
    sim = Simulator(sc, n_iters=gold["paper_lg_iterations"],
                    n_cr_iters=gold["paper_cr_iterations"], **kw)
    sim.set_state(sc.q0, sc.v0)
    nf = int(round(T / sc.h))
    sim.step(n_frames=nf // 2)
    v_half = float(sim.state()[1].mean(0) @ down)
    sim.step(n_frames=nf - nf // 2)
    a = (float(sim.state()[1].mean(0) @ down) - v_half) / (T / 2)
    sim.close()
    return a, max(9.81 * (math.sin(th) - (gold["mu_star"] + dmu) * math.cos(th)), 0.0)


def test_stick_slip_comparison_of_preconditioners():
    """Sec. 7.5 on the GPU, the same brackets as the oracle's pin: the Delassus
    preconditioner slides at mu* - 0.01 with the analytic acceleration and sticks at
    mu* + 0.01; the mass-inverse one sticks at mu* - 0.03 and slides at mu* - 0.1."""
    gold = json.load(open(os.path.join(GOLDEN, "stick_slip.json")))
    a, a_exp = _gpu_slope_acceleration(gold, -0.01)
    assert abs(a - a_exp) < 0.03 * a_exp
    a, _ = _gpu_slope_acceleration(gold, +0.01)
    assert abs(a) < 1e-3
    a, a_exp = _gpu_slope_acceleration(gold, -0.03, precond="mass")
    assert a_exp > 0.25 and abs(a) < 1e-3
    a, a_exp = _gpu_slope_acceleration(gold, -gold["paper_mass_preconditioner_accuracy"],
                                       precond="mass")
    assert abs(a - a_exp) < 0.03 * a_exp

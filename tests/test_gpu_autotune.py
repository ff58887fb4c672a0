"""The autotuner of the profile products: it times every candidate launch configuration
(CTAs per SM, balance of the tile split, tiles in flight or the bulk-copy form) and keeps the
fastest; whatever it picks, the solve and the frame keep their parity with the oracle. The
bulk-copy form on its own (autotune = 2): the solve and a contact frame against the oracle
and against the register form, in FP32 and BF16."""
import numpy as np
import pytest

import scenegen as sg
from oracle import Oracle, OracleOptions
from oracle.fem import FEM
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_autotuned_products_keep_parity_and_beat_or_match_the_default():
    sc = sg.star_pull(n_side=20, layers=12)
    sim = Simulator(sc, autotune=1)
    t = sim.tuning()
    print("tuning:", t)
    assert t["tuned"] == 1 and t["candidates"] == 32
    # the fixed configuration is one of the candidates, so the choice is never slower
    assert t["pass1_us"] <= t["pass1_default_us"] and t["pass2_us"] <= t["pass2_default_us"]
    assert t["pass1_unroll"] in (0, 1, 2, 3) and t["pass2_unroll"] in (0, 1, 2, 3)
    b = np.random.default_rng(3).normal(size=(sc.n_verts, 3))
    f = FEM(sc)
    xr = np.zeros_like(b)
    xr[f.free_verts] = f.solve(b[f.free_verts].reshape(-1)).reshape(-1, 3)
    assert _relerr(sim.apply_inverse(b), xr) < 1e-5
    sim.close()


def test_autotuned_frame_with_contact_matches_oracle():
    sc = sg.cube_drop(m=9, model=sg.MODEL_COROT, height=-0.003, seed=2, mu=0.5)
    q, _, info = Oracle(sc).frame(sc.q0, sc.v0, OracleOptions(n_iters=5, n_cr=sc.n_cr))
    sim = Simulator(sc, autotune=1)
    sim.step(n_iters=5)
    qg, _ = sim.state()
    assert len(info["contacts"]) > 3
    assert _relerr(qg, q) < 1e-5
    sim.close()


def test_fixed_configuration_is_reported_without_tuning():
    sim = Simulator(sg.cube_drop(m=5))
    t = sim.tuning()
    assert t["tuned"] == 0 and t["pass1_ctas"] > 0 and t["pass2_ctas"] > 0
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_bulk_copy_products_match_the_register_form(prec):
    # several row groups and column tiles per CTA, ragged rows, a partly filled last tile
    sc = sg.star_pull(n_side=20, layers=12)
    reg = Simulator(sc, s_precision=prec, refine=0)
    blk = Simulator(sc, s_precision=prec, refine=0, autotune=2)
    assert blk.tuning()["pass1_unroll"] == 3 and blk.tuning()["pass2_unroll"] == 3
    b = np.random.default_rng(5).normal(size=(sc.n_verts, 3))
    xa, xb = reg.apply_inverse(b), blk.apply_inverse(b)
    # the same values summed in another order: FP32 rounding only
    assert _relerr(xb, xa) < 2e-6
    if prec == 0:
        f = FEM(sc)
        xr = np.zeros_like(b)
        xr[f.free_verts] = f.solve(b[f.free_verts].reshape(-1)).reshape(-1, 3)
        assert _relerr(xb, xr) < 1e-5
    reg.close()
    blk.close()


def test_bulk_copy_frame_with_contact_matches_oracle():
    sc = sg.cube_drop(m=9, model=sg.MODEL_COROT, height=-0.003, seed=2, mu=0.5)
    q, _, info = Oracle(sc).frame(sc.q0, sc.v0, OracleOptions(n_iters=5, n_cr=sc.n_cr))
    sim = Simulator(sc, autotune=2)
    sim.step(n_iters=5)
    qg, _ = sim.state()
    assert len(info["contacts"]) > 3
    assert _relerr(qg, q) < 1e-5
    assert sim.stats()["n_contacts"] == len(info["contacts"])
    sim.close()

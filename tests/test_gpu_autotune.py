"""The autotuner of the profile products: it times every candidate launch configuration
(CTAs per SM, balance of the tile split, tiles in flight) and keeps the fastest; whatever it
picks, the solve and the frame keep their parity with the oracle."""
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
    assert t["tuned"] == 1 and t["candidates"] == 24
    # the fixed configuration is one of the candidates, so the choice is never slower
    assert t["pass1_us"] <= t["pass1_default_us"] and t["pass2_us"] <= t["pass2_default_us"]
    assert t["pass1_unroll"] in (0, 1, 2) and t["pass2_unroll"] in (0, 1, 2)
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

"""GPU parity at the benchmarked size: the 59.8k-DoF star (43 x 43 x 27 lattice, 19,926
vertices, 101,400 tetrahedra, stable Neo-Hookean E = 1e6) placed 9.4 cm into the first row
of cylinders, 837 contacts, one 5-iteration frame with 10 CR iterations (Alg. 4), in the
launch configuration the benchmark times (autotuned products, a 16-CTA constraint-solve
cluster, contact capacity 4096). The FP64 oracle runs the same frame on the host (its W
from 2,511 direct solves, about a minute and a half).

Gates (single step from an identical state, FP32 on the device):
  * the contact sets are equal (vertex, obstacle), in order;
  * ||q - q_ref|| / ||q_ref|| <= 1e-5; the displacement-relative error is reported;
  * ||lambda - lambda_ref|| / ||lambda_ref|| <= 1e-5 over the contacts whose normal impulse
    is not rounding residue: |lambda_n| >= 1e-6 max lambda_n (at lambda_n = 0 the friction
    indicator flips, App. B.2); the excluded count is reported;
  * W~ at every pair of contact vertices within 1e-5 of its largest entry (Eq. 27), read
    from the oracle's W = H A^-1 H^T through W_jk = W~(v_j, v_k) D_j D_k^T;
  * the residual R_k of every iteration within 1e-4.
"""
import numpy as np
import pytest

import scenegen as sg
from oracle import Oracle, OracleOptions
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu

N_SIDE, PLACEMENT = 43, 0.094


@pytest.fixture(scope="module")
def star_frame():
    sc = sg.star_pull(n_side=N_SIDE, seed=0)
    q0, v0 = sg.star_placed(sc, PLACEMENT)
    sim = Simulator(sc, autotune=1, contact_capacity=4096)
    sim.set_state(q0, v0)
    sim.step(n_iters=5)
    qg, vg = sim.state()
    gpu = dict(q=qg, v=vg, contacts=sim.contacts(), stats=sim.stats(), delassus=sim.delassus(),
               tuning=sim.tuning())
    sim.close()
    # the same frame with the two-exchange constraint solve
    sim = Simulator(sc, autotune=1, contact_capacity=4096, cr_exchanges=2)
    sim.set_state(q0, v0)
    sim.step(n_iters=5)
    gpu["q2"], _ = sim.state()
    gpu["lam2"] = sim.contacts()["lam"]
    sim.close()
    o = Oracle(sc)
    q, v, info = o.frame(q0, v0, OracleOptions(n_iters=5, n_cr=10))
    return dict(scene=sc, q0=q0, gpu=gpu, ref=dict(q=q, v=v, info=info))


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_fullsize_contact_sets_equal(star_frame):
    ct = star_frame["gpu"]["contacts"]
    ref = star_frame["ref"]["info"]["contacts"]
    keys_g = list(zip(ct["vertex"].tolist(), ct["obstacle"].tolist()))
    keys_o = [(c["vertex"], c["obstacle"]) for c in ref]
    assert len(keys_o) >= 800, len(keys_o)
    assert keys_g == keys_o


def test_fullsize_positions_match(star_frame):
    qg, q, q0 = star_frame["gpu"]["q"], star_frame["ref"]["q"], star_frame["q0"]
    err = _relerr(qg, q)
    disp = _relerr(qg - q0, q - q0)
    print(f"\nfull-size star: |q - q_ref|/|q_ref| = {err:.2e}, displacement-relative {disp:.2e}")
    assert err <= 1e-5, err
    vg, v = star_frame["gpu"]["v"], star_frame["ref"]["v"]
    assert _relerr(vg, v) <= 1e-3, _relerr(vg, v)


@pytest.mark.parametrize("form", ["one_exchange", "two_exchanges"])
def test_fullsize_impulses_match(star_frame, form):
    lam_g = star_frame["gpu"]["contacts"]["lam"] if form == "one_exchange" else \
        star_frame["gpu"]["lam2"]
    lam_o = star_frame["ref"]["info"]["lam"]
    keep = np.abs(lam_o[:, 0]) >= 1e-6 * np.abs(lam_o[:, 0]).max()
    err = _relerr(lam_g[keep], lam_o[keep])
    print(f"\nfull-size star ({form}): lambda rel. error {err:.2e} over {int(keep.sum())} "
          f"contacts, {int((~keep).sum())} excluded (|lambda_n| < 1e-6 max)")
    assert keep.sum() >= 0.5 * len(keep)
    assert err <= 1e-5, err
    if form == "two_exchanges":
        assert _relerr(star_frame["gpu"]["q2"], star_frame["ref"]["q"]) <= 1e-5


def test_fullsize_delassus_matches(star_frame):
    Wt, cv = star_frame["gpu"]["delassus"]
    info = star_frame["ref"]["info"]
    contacts = info["contacts"]
    c = len(contacts)
    D = np.stack([np.stack([ct["n"], ct["f1"], ct["f2"]]) for ct in contacts])   # (c, 3, 3)
    W = info["W"].reshape(c, 3, c, 3).transpose(0, 2, 1, 3)                        # (c, c, 3, 3)
    # W_jk = W~ D_j D_k^T with orthonormal D: W~ = tr(D_j^T W_jk D_k) / 3
    Wt_ref = np.einsum("jab,jkac,kcb->jk", D, W, D) / 3.0
    vert = [ct["vertex"] for ct in contacts]
    assert len(set(vert)) == c                                   # one contact per vertex
    pos = {int(v): i for i, v in enumerate(cv)}
    idx = np.array([pos[v] for v in vert])
    Wg = Wt[np.ix_(idx, idx)]
    err = np.abs(Wg - Wt_ref).max() / np.abs(Wt_ref).max()
    print(f"\nfull-size star: W~ max error {err:.2e} of its largest entry ({c} x {c})")
    assert err <= 1e-5, err


def test_fullsize_residuals_match(star_frame):
    rg = np.array(star_frame["gpu"]["stats"]["residuals"])
    ro = np.array(star_frame["ref"]["info"]["residuals"])
    assert len(rg) == len(ro) == 6
    print("\nfull-size star residuals (device / oracle): " +
          ", ".join(f"{a:.3e}/{b:.3e}" for a, b in zip(rg, ro)))
    assert np.abs(rg - ro).max() <= 1e-4, np.abs(rg - ro).max()

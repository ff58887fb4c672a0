"""The Jacobi global step (SIM_GLOBAL_JACOBI), the incomplete solve of Sec. 8's convergence
comparison, on the GPU: its frames against the oracle's, and the comparison itself on the
twisted bar (energies evaluated by the oracle on the GPU's frames)."""
import numpy as np
import pytest

import scenegen as sg
from oracle import Oracle, OracleOptions
from oracle.local import elastic_energy
from paper_2503_15078_b300 import Simulator

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("sweeps,iters", [(1, 5), (1, 40), (4, 12)])
def test_jacobi_frames_match_oracle(sweeps, iters):
    sc = sg.twisting_bar(E=1e6)
    o = Oracle(sc)
    q, _, _ = o.frame(sc.q0, sc.v0, OracleOptions(n_iters=iters, global_solver="jacobi",
                                                   jacobi_sweeps=sweeps))
    sim = Simulator(sc, global_solver="jacobi", jacobi_sweeps=sweeps)
    sim.set_state(sc.q0, sc.v0)
    sim.step(n_iters=iters)
    assert _relerr(sim.state()[0] - sc.q0, q - sc.q0) < 1e-4
    sim.close()


def test_complete_solve_converges_faster_than_jacobi_on_the_gpu():
    sc = sg.twisting_bar(E=1e7)
    o = Oracle(sc)
    f = o.fem
    s_tilde = o.predict(sc.q0, sc.v0)
    q_star, _, _ = o.frame(sc.q0, sc.v0, OracleOptions(n_iters=1500))

    def eps(x):
        kin = 0.5 / sc.h ** 2 * float((f.mass[:, None] * (x - s_tilde) ** 2).sum())
        return kin + elastic_energy(f.deformation_gradients(x), f.model, f.V, f.emu, f.elam,
                                    f.alpha)

    e0, es = eps(sc.q0), eps(q_star)
    sims = {"sparse_inverse": Simulator(sc),
            "jacobi": Simulator(sc, global_solver="jacobi", jacobi_sweeps=1)}
    for k in (3, 10, 30):
        err = {}
        for name, sim in sims.items():
            sim.set_state(sc.q0, sc.v0)
            sim.step(n_iters=k)
            err[name] = (eps(sim.state()[0]) - es) / (e0 - es)
        assert 0 < err["sparse_inverse"] < 0.6 * err["jacobi"], (k, err)
    for sim in sims.values():
        sim.close()

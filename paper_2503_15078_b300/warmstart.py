"""Training and evaluation of the learned warm start through the C ABI (an addition to the
paper's method, whose frames start from lambda = 0).

collect    runs the plain method (cold start) over scenes and returns, per contact and
           frame, the features seen at the frame's start and the frame's final impulse and
           normal move (the targets)
train      fits the network on the GPU (sim_mlp_train: the project's own tensor-core
           forward/backward kernels and Adam)
evaluate   iterations and device milliseconds until the frame's residual reaches a
           tolerance, per frame, for a given start (cold, previous frame, learned, or a
           portfolio: the cold start and a warm start side by side, best of the two);
           evaluate_to_tolerance measures the same with frames that stop on the device
"""
from __future__ import annotations

import numpy as np

from . import SimError, Simulator, WarmStartNet

MODES = {"cold": 0, "learned": 1, "previous": 2}
# portfolio starts: two copies of the scene in one batch, copy 0 cold, copy 1 this start
PORTFOLIO = {"portfolio": 1, "portfolio_previous": 2}


def collect(scenes, frames, n_iters=20, tol=1e-4, **opts):
    """Samples of the frames whose final residual reached tol (their impulses are the
    method's answer, not an iterate still moving)."""
    Xs, Ts = [], []
    for sc in scenes:
        sim = Simulator(sc, n_iters=n_iters, **opts)
        for _ in range(frames):
            try:
                sim.step()
                X, T = sim.warmstart_samples()
                r = sim.stats()["residuals"]
            except SimError:   # a frame that left the state non-finite ends the trajectory
                break
            if len(X) and r[-1] <= tol:
                Xs.append(X)
                Ts.append(T)
        sim.close()
    if not Xs:
        return np.zeros((0, WarmStartNet.FEATURES), np.float32), np.zeros((0, 4), np.float32)
    return np.concatenate(Xs), np.concatenate(Ts)


SHRINK = (0.0, 0.25, 0.5, 0.75, 1.0)


def train(X, T, epochs=60, batch=512, lr=1e-3, seed=0, device=0, X_val=None, T_val=None):
    """Fit the network; with a validation set, then scale each output (its row of the last
    layer) by the factor in SHRINK with the lowest validation error, so that an output with
    no skill on held-out frames (better left at zero: no change from the previous frame's
    impulse) is switched off. Returns the network and the per-epoch losses."""
    net = WarmStartNet(device=device, max_batch=max(batch, 64), seed=seed)
    losses = net.train(X, T, epochs=epochs, batch=batch, lr=lr, seed=seed + 1)
    if X_val is not None and len(X_val):
        Y = net.forward(X_val)
        theta = net.params()
        H, OUT = 128, 8
        w4 = theta[-OUT - H * OUT:-OUT].reshape(H, OUT)
        b4 = theta[-OUT:]
        for c in range(Y.shape[1]):
            err = [float(np.mean((a * Y[:, c] - T_val[:, c]) ** 2)) for a in SHRINK]
            a = SHRINK[int(np.argmin(err))]
            w4[:, c] *= a
            b4[c] *= a
        net.set_params(theta)
    return net, losses


def evaluate_from_states(scenes, frames, modes, net=None, k_max=40, tol=1e-4, gains=None,
                         **opts):
    """A/B from identical states: each scene's reference trajectory is run with the cold start
    and k_max iterations per frame; every frame with contacts is then replayed once per
    start in `modes` from the reference state of the frame before it (one cold frame to set
    up the previous frame's impulses, then the frame under test). Returns, per mode, the
    iterations until the residual reaches tol (k_max + 1 if never) and the device time to
    get there, over the same frames. A portfolio mode runs the frame as a two-copy batch
    (sim_set_portfolio) and reaches tol at the first iteration where either copy does; its
    time is the batch's."""
    out = {m: {"iters": [], "ms": [], "res": []} for m in modes}
    pf_modes = [m for m in modes if m in PORTFOLIO]
    for sc in scenes:
        ref = Simulator(sc, n_iters=k_max, **opts)
        states = [ref.state()]
        contact = []
        for _ in range(frames):
            try:
                ref.step()
                contact.append(ref.stats()["n_contacts"] > 0)
                states.append(ref.state())
            except SimError:
                break
        ref.close()
        sim = Simulator(sc, n_iters=k_max, **opts)
        pf = None
        if pf_modes:
            pf = Simulator([sc, sc], n_iters=k_max, **opts)
            pf.set_portfolio(2)
        if gains is not None:
            for s_g in (sim, pf):
                if s_g is not None:
                    s_g.set_warmstart_gains(*gains)
        for f in range(1, len(contact)):
            if not contact[f]:
                continue
            for m in modes:
                s_m = pf if m in PORTFOLIO else sim
                state = states[f - 1]
                if s_m is pf:
                    state = tuple(np.concatenate([a, a]) for a in state)
                try:
                    s_m.set_state(*state)
                    s_m.set_warmstart(0)
                    s_m.step()                      # frame f - 1: the previous impulses
                    mode = PORTFOLIO[m] if s_m is pf else MODES[m] if isinstance(m, str) else int(m)
                    s_m.set_warmstart(mode, net)
                    s_m.step()                      # frame f from the reference state
                    st = s_m.stats()
                    # a portfolio reaches the tolerance when either copy does
                    r = (s_m.scene_residuals().min(axis=0) if s_m is pf
                         else np.asarray(st["residuals"]))
                except SimError:
                    out[m]["iters"].append(k_max + 1)
                    out[m]["ms"].append(np.nan)
                    out[m]["res"].append(np.full(k_max + 1, np.nan))
                    continue
                out[m]["res"].append(r[:k_max + 1])
                hit = np.nonzero(r <= tol)[0]
                k = int(hit[0]) if len(hit) else k_max + 1
                ph = s_m.phase_times()
                per_iter = sum(ph[p] for p in ("local", "assemble", "spmv1", "solve", "spmv2",
                                               "reduce")) / k_max
                start = ph["collide"] + ph["delassus"] + ph["warmstart"]
                out[m]["iters"].append(k)
                out[m]["ms"].append(start + min(k, k_max) * per_iter + ph["integrate"])
        sim.close()
        if pf is not None:
            pf.close()
    res = {}
    for m, d in out.items():
        it, ms = np.asarray(d["iters"]), np.asarray(d["ms"])
        res[m] = {"frames": int(len(it)), "mean_iters": float(it.mean()) if len(it) else 0.0,
                  "median_iters": float(np.median(it)) if len(it) else 0.0,
                  "unreached": int((it > k_max).sum()),
                  "mean_ms": float(np.nanmean(ms)) if len(ms) else 0.0,
                  "iters": it.tolist(), "residuals": np.asarray(d["res"])}
    return res


def evaluate_to_tolerance(scenes, frames, modes, net=None, k_max=40, tol=1e-4, gains=None,
                          **opts):
    """The A/B of evaluate_from_states with frames that stop on the device when the residual
    reaches tol (sim_options.residual_tol; at least one update, at most k_max): per mode the
    updates each contact frame took and its measured device time (the whole frame: collision,
    Delassus, start, iterations, integration). A portfolio stops when either copy is done.
    gains: (persist, fresh, move, accept) of the learned start (sim_set_warmstart_gains)."""
    out = {m: {"iters": [], "ms": []} for m in modes}
    for sc in scenes:
        ref = Simulator(sc, n_iters=k_max, **opts)
        states = [ref.state()]
        contact = []
        for _ in range(frames):
            try:
                ref.step()
                contact.append(ref.stats()["n_contacts"] > 0)
                states.append(ref.state())
            except SimError:
                break
        ref.close()
        sims = {}
        for m in modes:
            pf = m in PORTFOLIO
            sim = Simulator([sc, sc] if pf else sc, n_iters=k_max, residual_tol=tol,
                            max_iters=k_max, **opts)
            if pf:
                sim.set_portfolio(2)
            if gains is not None:
                sim.set_warmstart_gains(*gains)
            sims[m] = sim
        for f in range(1, len(contact)):
            if not contact[f]:
                continue
            for m in modes:
                sim = sims[m]
                state = states[f - 1]
                if m in PORTFOLIO:
                    state = tuple(np.concatenate([a, a]) for a in state)
                try:
                    sim.set_state(*state)
                    sim.set_warmstart(0)
                    sim.step(n_iters=k_max)         # frame f - 1: the previous impulses
                    sim.set_warmstart(PORTFOLIO.get(m, MODES.get(m, 0)), net)
                    sim.step()                      # frame f, to the tolerance
                    k = sim.stats()["n_iters"]
                    ms = sum(sim.phase_times().values())
                except SimError:
                    k, ms = k_max + 1, np.nan
                out[m]["iters"].append(k)
                out[m]["ms"].append(ms)
        for sim in sims.values():
            sim.close()
    res = {}
    for m, d in out.items():
        it, ms = np.asarray(d["iters"]), np.asarray(d["ms"])
        res[m] = {"frames": int(len(it)), "mean_iters": float(it.mean()) if len(it) else 0.0,
                  "median_iters": float(np.median(it)) if len(it) else 0.0,
                  "at_cap": int((it >= k_max).sum()),
                  "mean_ms": float(np.nanmean(ms)) if len(ms) else 0.0,
                  "median_ms": float(np.nanmedian(ms)) if len(ms) else 0.0}
    return res


def evaluate(scenes, frames, mode, net=None, k_max=40, tol=1e-4, **opts):
    """Each scene runs `frames` frames of k_max iterations from its initial state with the
    given start; for every frame with contacts: the first k with residual R_k <= tol (k_max + 1
    if none) and the device time to get there: collision, Delassus and warm start, plus k
    times the frame's mean time per iteration."""
    iters, ms = [], []
    for sc in scenes:
        sim = Simulator(sc, n_iters=k_max, **opts)
        sim.set_warmstart(MODES[mode] if isinstance(mode, str) else int(mode), net)
        for _ in range(frames):
            try:
                sim.step()
                st = sim.stats()
            except SimError:   # non-finite: counted as not reached, the trajectory ends
                iters.append(k_max + 1)
                ms.append(np.nan)
                break
            if st["n_contacts"] == 0:
                continue
            r = np.asarray(st["residuals"])
            hit = np.nonzero(r <= tol)[0]
            k = int(hit[0]) if len(hit) else k_max + 1
            ph = sim.phase_times()
            per_iter = sum(ph[p] for p in ("local", "assemble", "spmv1", "solve", "spmv2",
                                           "reduce")) / k_max
            start = ph["collide"] + ph["delassus"] + ph["warmstart"]
            iters.append(k)
            ms.append(start + min(k, k_max) * per_iter + ph["integrate"])
        sim.close()
    iters, ms = np.asarray(iters), np.asarray(ms)
    return {"frames": int(len(iters)), "mean_iters": float(iters.mean()) if len(iters) else 0.0,
            "median_iters": float(np.median(iters)) if len(iters) else 0.0,
            "unreached": int((iters > k_max).sum()),
            "mean_ms": float(np.nanmean(ms)) if len(ms) else 0.0,
            "diverged": int(np.isnan(ms).sum())}


# (persist, fresh, move, accept); (0, 0, 0, 1) is the previous-frame start
GAIN_GRID = [(p, f, m, a) for p in (0.0, 1.0) for f in (0.0, 1.0) for m in (0.0, 1.0)
             for a in (1.0, 0.5, 0.25)]


def choose_gains(net, scenes, frames, grid=GAIN_GRID, k_max=40, tol=1e-4, **opts):
    """The output gains of the learned start that give the lowest mean frame time to the
    residual tolerance on validation scenes (device-stopped frames, the measure of the
    held-out A/B). Returns (gains, {gains: (mean updates, mean ms)})."""
    table = {}
    for g in grid:
        r = evaluate_to_tolerance(scenes, frames, ["learned"], net=net, k_max=k_max, tol=tol,
                                  gains=g, **opts)["learned"]
        table[g] = (r["mean_iters"], r["mean_ms"])
    best = min(grid, key=lambda g: (table[g][1], table[g][0], g))
    return best, table

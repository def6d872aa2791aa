"""Learned proposal for the GD solver (not in the paper).

A small network maps an instance's couplings to (a) each spin's initial
amplitude and (b) the instance's run settings (gain speed eps, threshold
rho_th, initial coupling scale beta0 of the ramp).  It runs entirely in the
library's kernels (gda_features, gda_mlp_forward / backward, gda_proposal_loss,
gda_adam_step); this module only moves buffers and maps the network's outputs
to parameters.  It is trained on the best configurations and fastest settings
that plain GD runs find; the plain algorithm stays the fallback and the arbiter
(its FP64 energies decide).

Output mapping (o = network output, mean over the instance's spins for 2..4):
  eps    = 0.02 + 0.48 sigmoid(o2)
  rho_th = 0.5 + 1.5 sigmoid(o3)
  beta0  = 0.1 + 0.9 sigmoid(o4)   (ramp d beta/dt = RAMP (1 - beta))
  psi_i(0) = AMP (o0 + i o1)  plus the library's seeded U(-AMP, AMP) perturbation
             per restart (init_mode 3, generated on the device).
"""
from __future__ import annotations

import ctypes as ct
import math
import os

import numpy as np

from . import gda

HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS_PATH = os.path.join(HERE, "data", "proposal_params.npy")
NPARAM = 18309
RAMP = 0.2    # eps_hat of the coupling ramp when beta0 < 1
AMP = 0.1     # scale of the proposed initial amplitudes
GRID = [(e, 1.0, b) for e in (0.05, 0.2, 0.5) for b in (0.3, 1.0)]  # (eps, rho_th, beta0) candidates


def _sig(x):
    return 1.0 / (1.0 + math.exp(-x))


def _logit(p):
    return math.log(p / (1.0 - p))


def settings_from_outputs(o_mean) -> dict:
    return {"eps": 0.02 + 0.48 * _sig(o_mean[0]), "rho_th": 0.5 + 1.5 * _sig(o_mean[1]),
            "beta0": 0.1 + 0.9 * _sig(o_mean[2])}


def outputs_from_settings(eps, rho_th, beta0):
    """Inverse of settings_from_outputs (training targets), clipped inside (0, 1)."""
    def lg(p):
        return _logit(min(max(p, 1e-3), 1 - 1e-3))
    return [lg((eps - 0.02) / 0.48), lg((rho_th - 0.5) / 1.5), lg((beta0 - 0.1) / 0.9)]


def run_params(settings: dict, **kw) -> gda.Params:
    ramp = RAMP if settings["beta0"] < 0.999 else 0.0
    return gda.default_params(eps=settings["eps"], rho_th=settings["rho_th"], beta0=settings["beta0"],
                              eps_hat=ramp, **kw)


class Proposal:
    """A trained (or freshly initialised) proposal network on the current device."""

    def __init__(self, params: np.ndarray | None = None):
        import torch
        self.torch = torch
        if params is None:
            params = np.load(PARAMS_PATH)
        params = np.asarray(params, dtype=np.float32)
        assert params.shape == (NPARAM,)
        self.p = torch.tensor(params, device="cuda")
        self.lib = gda.load_library()

    def outputs(self, solver: "gda.Solver"):
        """Network outputs [N][5] for the solver's instance (host copy)."""
        torch = self.torch
        N = solver.N
        F = torch.empty((N, 8), dtype=torch.float32, device="cuda")
        O = torch.empty((N, 5), dtype=torch.float32, device="cuda")
        solver.features(F.data_ptr())
        st = torch.cuda.current_stream().cuda_stream
        torch.cuda.synchronize()
        r = self.lib.gda_mlp_forward(ct.c_void_p(self.p.data_ptr()), ct.c_void_p(F.data_ptr()), N,
                                     ct.c_void_p(O.data_ptr()), None, ct.c_void_p(st))
        if r != 0:
            raise gda.GdaError(r, "gda_mlp_forward failed")
        torch.cuda.synchronize()
        return O.cpu().numpy().astype(np.float64)

    def head(self, solver: "gda.Solver"):
        """Features, network and head (gda_proposal_head) on the device for
        the solver's instance: (base, settings), base a device tensor in
        gda_set_init_base's layout; the settings (24 bytes) are the only data
        read back to the host."""
        torch = self.torch
        N = solver.N
        xy = solver.model == gda.XY
        F = torch.empty((N, 8), dtype=torch.float32, device="cuda")
        O = torch.empty((N, 5), dtype=torch.float32, device="cuda")
        base = torch.empty(2 * N if xy else N, dtype=torch.float32, device="cuda")
        st = torch.empty(3, dtype=torch.float64, device="cuda")
        solver.features(F.data_ptr())  # on the solver's stream
        torch.cuda.synchronize()
        s = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
        vp = lambda x: ct.c_void_p(x.data_ptr())  # noqa: E731
        r = self.lib.gda_mlp_forward(vp(self.p), vp(F), N, vp(O), None, s)
        if r == 0:
            r = self.lib.gda_proposal_head(vp(O), N, 1 if xy else 0, AMP, vp(base), vp(st), s)
        if r != 0:
            raise gda.GdaError(r, "proposal kernels failed")
        v = st.cpu().tolist()
        return base, {"eps": v[0], "rho_th": v[1], "beta0": v[2]}

    def propose(self, solver: "gda.Solver"):
        """Sets the solver's init_mode-3 base amplitudes and returns the settings."""
        base, settings = self.head(solver)
        solver.set_init_base_dev(base.data_ptr())
        return settings


def propose_into_batch(prop: "Proposal", solver: "gda.Solver", batch: "gda.Batch", k: int, dt: float) -> dict:
    """The proposal for the instance of `solver`, given to instance k of a
    batch: its settings (gda_batch_set_params, with the batch step dt) and
    its init_mode-3 base amplitudes.  Returns the settings."""
    base, settings = prop.head(solver)
    batch.set_init_base_dev(k, base.data_ptr())
    batch.set_params(k, run_params(settings, dt=dt))
    return settings


def proposed_params(settings: dict, seed: int, **kw) -> gda.Params:
    """Run parameters of a proposed start (init_mode 3, perturbation AMP)."""
    return run_params(settings, init_mode=3, init_amp=AMP, seed=seed, **kw)


# ---------------------------------------------------------------- training
def training_instance(k: int, seed0: int = 7):
    """Seeded Gaussian-J instance number k: N uniform in [256, 1024], XY (odd k,
    with g ~ U[-0.1, 0.1]) or Ising (even k, g = 0), J_ij ~ N(0, 1/N)."""
    import synth
    n = 256 + int(synth.uniform01(seed0 * 7919 + k, 1)[0] * 769)
    xy = k % 2 == 1
    J, g = synth.xy_gaussian(n, seed0 * 1000003 + k)
    return J, (g if xy else np.zeros(n)), xy


def ttt_steps(steps, E, target):
    hit = np.nonzero(E <= target)[0]
    return int(steps[hit[0]]) if len(hit) else None


def make_targets(J, g, xy, R=32, nsteps=1500, every=50, seed=1):
    """Runs the plain GD algorithm with every candidate setting; returns the
    best configuration found (unit spins, [N][2]) and the candidate setting that
    first reaches within 1e-3 of the best energy (ties: lower final energy),
    judged on the FP64 energies of the traced configurations."""
    s = gda.Solver(J, g, gda.XY if xy else gda.ISING)
    runs = []
    for (eps, rho, b0) in GRID:
        p = run_params({"eps": eps, "rho_th": rho, "beta0": b0}, dt=0.05, init_mode=1, init_amp=1e-3, seed=seed,
                       prec=gda.BF16, energy_every=every)
        s.run(p, R, nsteps)
        E, r, cfg = s.best()
        st, _, _ = s.trace()
        runs.append((E, cfg, st, s.trace_energy()))  # FP64 energies of the traced configurations
    s.close()
    Ebest = min(x[0] for x in runs)
    target = Ebest + 1e-3 * abs(Ebest)
    scored = []
    for k, (E, cfg, st, Et) in enumerate(runs):
        t = ttt_steps(st, Et, target)
        scored.append((t if t is not None else 10 ** 9, E, k))
    k_best = min(scored)[2]
    cfg = min(runs, key=lambda x: x[0])[1]
    S = np.zeros((len(cfg), 2))
    if xy:
        S[:, 0], S[:, 1] = np.cos(cfg), np.sin(cfg)
    else:
        S[:, 0] = cfg
    return S, GRID[k_best]


def init_params(seed: int) -> np.ndarray:
    """Initial parameters: normal weights scaled by 1/sqrt(fan-in) (x sqrt 2
    before ReLU), zero biases."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2.0 / 8), 128 * 8), np.zeros(128),
             rng.normal(0, math.sqrt(2.0 / 128), 128 * 128), np.zeros(128),
             rng.normal(0, math.sqrt(1.0 / 128), 5 * 128), np.zeros(5)]
    return np.concatenate(parts).astype(np.float32)


def _features_dev(J, g, xy):
    import torch
    s = gda.Solver(J, g, gda.XY if xy else gda.ISING)
    F = torch.empty((J.shape[0], 8), dtype=torch.float32, device="cuda")
    s.features(F.data_ptr())
    s.sync()
    s.close()
    return F


def train(n_inst=384, epochs=40, batch=16, lr=2e-3, wset=0.5, seed=0, log=print, target_minutes=None):
    """Generates targets with plain GD runs and trains the network with the
    library's kernels (forward, loss, backward, Adam); returns (params, losses).
    target_minutes: a wall-clock budget for the target runs; the instances
    generated within it are used (log reports how many)."""
    import time
    import torch
    lib = gda.load_library()
    data = []
    t0 = time.time()
    for k in range(n_inst):
        J, g, xy = training_instance(k)
        S, setting = make_targets(J, g, xy, seed=k + 1)
        data.append((_features_dev(J, g, xy), torch.tensor(S, dtype=torch.float32, device="cuda"),
                     outputs_from_settings(*setting), xy))
        if (k + 1) % 256 == 0:
            log(f"targets {k + 1}/{n_inst} in {time.time() - t0:.0f} s")
        if target_minutes is not None and time.time() - t0 > 60.0 * target_minutes:
            log(f"target budget reached after {k + 1} instances")
            break
    n_inst = len(data)
    p = torch.tensor(init_params(seed), device="cuda")
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    G = torch.zeros_like(p)
    rng = np.random.default_rng(seed)
    t = 0
    losses = []
    vp = lambda x: ct.c_void_p(x.data_ptr())  # noqa: E731
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    for ep in range(epochs):
        order = rng.permutation(n_inst)
        tot, cnt = 0.0, 0
        for b0 in range(0, n_inst, batch):
            idx = order[b0:b0 + batch]
            X = torch.cat([data[i][0] for i in idx]).contiguous()
            S = torch.cat([data[i][1] for i in idx]).contiguous()
            sizes = [data[i][0].shape[0] for i in idx]
            offs = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int32, device="cuda")
            cx = torch.tensor([1 if data[i][3] else 0 for i in idx], dtype=torch.int32, device="cuda")
            T = torch.tensor([data[i][2] for i in idx], dtype=torch.float32, device="cuda")
            M = X.shape[0]
            O = torch.empty((M, 5), dtype=torch.float32, device="cuda")
            H = torch.empty((M, 256), dtype=torch.float32, device="cuda")
            dO = torch.empty_like(O)
            L = torch.empty(len(idx), dtype=torch.float32, device="cuda")
            G.zero_()
            t += 1
            for r in (lib.gda_mlp_forward(vp(p), vp(X), M, vp(O), vp(H), st),
                      lib.gda_proposal_loss(vp(O), vp(S), vp(T), vp(offs), vp(cx), len(idx), wset, vp(dO), vp(L), st),
                      lib.gda_mlp_backward(vp(p), vp(X), vp(H), vp(dO), M, vp(G), st),
                      lib.gda_adam_step(vp(p), vp(G), vp(m1), vp(m2), NPARAM, lr, 0.9, 0.999, 1e-8, t, st)):
                if r != 0:
                    raise gda.GdaError(r, "proposal training kernel failed")
            tot += float(L.sum())
            cnt += len(idx)
        losses.append(tot / cnt)
        log(f"epoch {ep}: mean loss {losses[-1]:.4f}")
    return p.cpu().numpy(), losses


def _run_fp64(solver, params, R, nsteps):
    """One run with the energy trace: (trace steps, FP64 energies of the
    configurations the trace names, FP64 energies of every restart at the end,
    seconds)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    solver.run(params, R, nsteps)
    e1.record()
    e1.synchronize()
    st, _, _ = solver.trace()
    return st, solver.trace_energy(), solver.energy(), e0.elapsed_time(e1) / 1e3


def _first_hit(st, E64, target):
    hit = np.nonzero(E64 <= target)[0]
    return int(st[hit[0]]) if len(hit) else None


def eval_instance(model: str, n: int, seed: int):
    """Held-out instance of the evaluation: J ~ N(0, 1/N), g ~ U[-0.1, 0.1] (XY) or 0 (Ising)."""
    import synth
    J, g = synth.xy_gaussian(n, seed)
    return J, (g if model == "xy" else np.zeros(n))


def best_fixed_setting(model: str, n: int, seeds, R=64, nsteps=5000, every=25, dt=0.05, log=print) -> tuple:
    """The grid setting (eps, rho_th, beta0) that reaches its instances' targets
    fastest (FP64-verified), on calibration instances of the same family that
    the evaluation does not use: most hits first, then fewest steps."""
    score = {k: [] for k in range(len(GRID))}
    for seed in seeds:
        J, g = eval_instance(model, n, seed)
        s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
        runs = {}
        for k, (e, rho, b0) in enumerate(GRID):
            prm = run_params({"eps": e, "rho_th": rho, "beta0": b0}, dt=dt, init_mode=1, init_amp=1e-3, seed=seed,
                             prec=gda.BF16, energy_every=every)
            runs[k] = _run_fp64(s, prm, R, nsteps)
        s.close()
        Estar = min(min(float(r[1].min()), float(r[2].min())) for r in runs.values())
        target = Estar + 1e-3 * abs(Estar)
        for k, r in runs.items():
            h = _first_hit(r[0], r[1], target)
            score[k].append(h if h is not None else 10 ** 9)
    k_best = min(score, key=lambda k: (sum(x >= 10 ** 9 for x in score[k]), float(np.mean(score[k]))))
    log({"model": model, "N": n, "calibration": {str(GRID[k]): v for k, v in score.items()}, "best": GRID[k_best]})
    return GRID[k_best]


def mean_proposed_setting(prop: Proposal, model: str, n: int, seeds) -> dict:
    """The network's settings averaged over instances of the family that the
    evaluation does not use: the proposal reduced to per-model constants."""
    got = []
    for seed in seeds:
        J, g = eval_instance(model, n, seed)
        s = gda.Solver(J, g, gda.XY if model == "xy" else gda.ISING)
        got.append(prop.propose(s))
        s.close()
    return {k: float(np.mean([x[k] for x in got])) for k in ("eps", "rho_th", "beta0")}


def evaluate(prop: Proposal, cases, R=64, nsteps=5000, every=25, fixed=None, const=None, log=print):
    """FP64-verified time to target on held-out seeds, BF16, same R and steps,
    of the arms: plain GD (default settings, small random start), plain GD at
    the best fixed grid setting for the model (fixed[model], from
    best_fixed_setting), plain GD at the network's mean settings as constants
    (const[model], from mean_proposed_setting: an ablation of the per-instance
    output and of the proposed start), and the proposal (its settings and
    start).  The target is within 1e-3 of the best FP64 energy any arm reached
    (final restarts or traced configurations); an arm hits it at the first
    trace point whose named configuration is at or below it in FP64."""
    rows = []
    for model, n, seed in cases:
        J, g = eval_instance(model, n, seed)
        xy = model == "xy"
        s = gda.Solver(J, g, gda.XY if xy else gda.ISING)
        res = {}
        arms = ["plain", "learned"] + (["best_fixed"] if fixed else []) + (["learned_const"] if const else [])
        for arm in arms:
            if arm == "plain":
                settings = {"eps": 0.1, "rho_th": 1.0, "beta0": 1.0}
                prm = gda.default_params(dt=0.05, eps=0.1, rho_th=1.0, init_mode=1, init_amp=1e-3, seed=seed,
                                         prec=gda.BF16, energy_every=every)
            elif arm in ("best_fixed", "learned_const"):
                if arm == "best_fixed":
                    e, rho, b0 = fixed[model]
                    settings = {"eps": e, "rho_th": rho, "beta0": b0}
                else:
                    settings = dict(const[model])
                prm = run_params(settings, dt=0.05, init_mode=1, init_amp=1e-3, seed=seed, prec=gda.BF16,
                                 energy_every=every)
            else:
                settings = prop.propose(s)
                prm = proposed_params(settings, seed, dt=0.05, prec=gda.BF16, energy_every=every)
            st_, E64, E_all, sec = _run_fp64(s, prm, R, nsteps)
            res[arm] = (E64, E_all, st_, sec, settings)
        Estar = min(min(float(r[0].min()), float(r[1].min())) for r in res.values())
        target = Estar + 1e-3 * abs(Estar)
        row = {"model": model, "N": n, "seed": seed, "E_star": Estar}
        for arm, (E64, E_all, st_, sec, settings) in res.items():
            k = _first_hit(st_, E64, target)
            row[arm] = {"E": float(E_all.min()), "ttt_steps": k, "ttt_s": None if k is None else sec * k / nsteps,
                        "run_s": sec, "settings": settings}
        rows.append(row)
        log(row)
        s.close()
    return rows


def main(argv=None):
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "evaluate"])
    ap.add_argument("--n-inst", type=int, default=384)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--out", default=PARAMS_PATH)
    ap.add_argument("--report", default=None)
    ap.add_argument("--target-minutes", type=float, default=None)
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    if a.cmd == "train":
        used = []
        params, losses = train(n_inst=a.n_inst, epochs=a.epochs, target_minutes=a.target_minutes,
                               log=lambda m: (print(m, flush=True), used.append(m)))
        os.makedirs(os.path.dirname(a.out), exist_ok=True)
        np.save(a.out, params)
        report = {"losses": losses, "log": used}
    else:
        prop = Proposal(np.load(a.out))
        fixed = {"xy": best_fixed_setting("xy", 1024, [2 * 10 ** 6, 2 * 10 ** 6 + 1]),
                 "ising": best_fixed_setting("ising", 2048, [2 * 10 ** 6 + 100, 2 * 10 ** 6 + 101])}
        const = {"xy": mean_proposed_setting(prop, "xy", 1024, [2 * 10 ** 6, 2 * 10 ** 6 + 1]),
                 "ising": mean_proposed_setting(prop, "ising", 2048, [2 * 10 ** 6 + 100, 2 * 10 ** 6 + 101])}
        cases = [("xy", 1024, 10 ** 6 + k) for k in range(4)] + [("ising", 2048, 10 ** 6 + 100 + k) for k in range(4)]
        report = {"best_fixed": fixed, "learned_const": const,
                  "eval": evaluate(prop, cases, fixed=fixed, const=const)}
    if a.report:
        with open(a.report, "w") as fh:
            json.dump(report, fh, indent=1, default=float)


if __name__ == "__main__":
    main()

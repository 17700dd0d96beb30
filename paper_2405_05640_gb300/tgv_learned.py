"""Taylor-Green vortex with a learned initial guess for the pressure solve.

Protocol (every step of the path runs in the library's kernels; this module
only sequences calls and keeps device buffers):
  1. Steps 1..train_steps of the TGV (sem_ns_*), pressure solved by the
     chosen solver (FP64 refinement around FP32 PCG) from x0 = p^{n-1}.
     From step `skip` on (past the start-up transient), every step gives one
     training sample per element.  With p_ext = 3p1 - 3p2 + p3 the cubic
     extrapolation and r = b - A p_ext its residual, the correction
     e = p^n - p_ext solves A e = r.  Target e / se, se = rho rms(r);
     features (p1-p2)/sd, (p2-p3)/sd, r/rms(r) and a fourth field:
       variant "p1" (default): p1/rms(p1); rho = rms(e)/rms(r) measured once,
         on the first sample;
       variant "d3": the previous error d3 = p1 - 3p2 + 3p3 - p4 divided by
         se; rho taken from the previous step (tracks its drift).
     Every scale is known before the solve, so inference uses the same ones.
  2. The element-local network (sem_mlp_*) is trained with Adam on all
     samples (tcgen05 GEMMs forward and backward), with the mean-square loss
     ("mse") or the energy norm of its error (sem_mlp_grad_energy: stiffness
     plus lam times the mass, so that errors the solver sees amplified in its
     residual weigh more), element by element ("energy") or of the averaged
     correction the guess uses ("energy_avg": the disagreement of
     neighbouring elements counts too).
  3. From the checkpoint at step train_steps, eval_steps more steps are run
     once per method: plain FP64 PCG from x0 = p^{n-1} (the stronger plain
     baseline); FP64 refinement around FP32 Jacobi-PCG ("chosen_*") and
     around flexible FP32 CG with the hybrid Schwarz preconditioner (the
     paper's pressure preconditioner, "schwarz_*"), each from p^{n-1}, from
     p_ext and from the learned guess p_ext + se * MLP(features).
     The three-level Schwarz multigrid ("schwarz3_*": an intermediate order-3
     level) from p_ext and from the learned guess; flexible GMRES(30) with
     the two-level Schwarz preconditioner ("schwarzgm_*") from p_ext.  Every mixed solve uses
     the adaptive inner tolerance inner_adapt (a round stops once the outer
     target is within reach), the Schwarz ones an inner tolerance of
     schwarz_inner_tol (Jacobi: 1e-2); the "*_fixed" methods keep
     inner_tol = 1e-2 every round.  Pressure-solve wall time includes building the guess.
  Phase 1 solves with the Schwarz solver when it is among the methods (the
  pressures, hence the samples, are the same to the tolerance).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import binding, inputs


def _rup(x, m=128):
    return (x + m - 1) // m * m


class GuessNet:
    """Features, targets and guesses for one mesh, plus the network."""

    def __init__(self, gm, hidden=256, seed=0, variant="p1", pair=False):
        import torch
        self.gm = gm
        self.variant = variant
        self.pair = pair  # residual feature with the FP32-pair operator
        self.E, self.npt = gm.E, gm.npt
        self.I, self.O, self.R = _rup(4 * self.npt), _rup(self.npt), _rup(self.E)
        self.H = hidden
        self.net = binding.MLP(self.I, self.H, self.O, self.R)
        self.net.set_params(inputs.mlp_init(self.I, self.H, self.O, seed))
        self.X = torch.zeros((self.R, self.I), dtype=torch.bfloat16, device="cuda")
        self.Y = torch.zeros((self.R, self.O), dtype=torch.float32, device="cuda")
        self.Y0 = torch.zeros((self.R, self.O), dtype=torch.float32, device="cuda")  # no correction
        self.r = torch.empty(gm.nloc, dtype=torch.float64, device="cuda")
        self.pext = torch.empty(gm.nloc, dtype=torch.float64, device="cuda")
        self.guess = torch.empty(gm.nloc, dtype=torch.float64, device="cuda")
        self.scales = None
        self.rho_prev = None

    def rms(self, a):
        return math.sqrt(max(self.gm.glsc3(a, a), 0.0) / self.gm.nglob)

    def residual(self, b, p1, p2, p3):
        binding.guess_residual(self.gm, b, p1, p2, p3, self.r, self.pext, pair=self.pair)

    def extrap(self, p1, p2, p3):
        """The cubic extrapolation alone (no residual: only the network's
        features need it): Q Q^T p_ext / mult with a zero correction."""
        binding.guess_apply(self.gm, self.Y0, p1, p2, p3, 0.0, self.guess)
        return self.guess

    def set_scales(self, p1, p2, p3, p4):
        """Feature scales of this sample (after residual()); variant "d3"
        needs rho_prev."""
        sr = self.rms(self.r)
        s4 = self.rho_prev * sr if self.variant == "d3" else self.rms(p1)
        self.scales = dict(sd=self.rms(p1 - p2), sr=sr, s3=s4)

    def target_scale(self):
        return self.rho_prev * self.scales["sr"]

    def update_rho(self, p_new):
        """rho = rms(p_new - p_ext) / rms(r) of the step just solved."""
        e = p_new - self.pext
        self.rho_prev = self.rms(e) / self.rms(self.r)

    def features(self, p1, p2, p3, p4):
        s = self.scales
        binding.guess_features(self.gm, p1, p2, p3, p4 if self.variant == "d3" else None, self.r, s["sd"],
                               s["sr"], s["s3"], self.X)

    def target(self, p_new, p1, p2, p3, T):
        binding.guess_target(self.gm, p_new, p1, p2, p3, self.target_scale(), T)

    def predict(self, p1, p2, p3):
        self.net.forward(self.X, self.Y)
        binding.guess_apply(self.gm, self.Y, p1, p2, p3, self.target_scale(), self.guess)
        return self.guess


METHODS = ("plain_f64_prev", "chosen_prev", "chosen_extrap", "chosen_learned", "chosen_extrap_fixed",
           "schwarz_prev", "schwarz_extrap", "schwarz_learned", "schwarz_extrap_fixed", "schwarz_learned_fixed",
           "schwarz3_extrap", "schwarz3_learned", "schwarzgm_extrap")


def _method(meth):
    """(solver, guess, fixed inner tolerance) of a method name."""
    solver = meth.split("_")[0]
    guess = "extrap" if "_extrap" in meth else "learned" if "_learned" in meth else "prev"
    return solver, guess, meth.endswith("_fixed")


def run(nel=32, N=7, Re=1600.0, dt=1e-3, train_steps=100, eval_steps=100, epochs=8, lr=1e-3, hidden=256,
        tol=1e-8, seed=0, skip=10, variant="p1", methods=METHODS, inner_adapt=0.5, loss="energy_avg", lam=1.0,
        pair=True, schwarz_inner_tol=1e-5, log=None):
    import torch
    log = log or (lambda *a: None)
    t_all = time.perf_counter()
    case = inputs.tgv_box(nel, N)
    gm = binding.Mesh(N, case.nel, case.periodic, case.faces, case.vertices(), geom_rx=True, geom_f32=True,
                      geom_pair=pair)
    xyz = gm.coords().cpu().numpy()
    u0 = torch.from_numpy(np.stack([c.reshape(-1) for c in inputs.tgv_velocity(*xyz)])).cuda()
    ns = binding.NSState(gm, Re)
    ns.set_velocity(u0)
    chosen = gm.pcg_opts(tol=tol, max_iter=50000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2,
                         use_initial_guess=True, check_every=32, inner_adapt=inner_adapt)
    plain = gm.pcg_opts(tol=tol, max_iter=50000, precision=binding.SEM_PCG_F64, use_initial_guess=True,
                        check_every=32)
    vopts = gm.pcg_opts(tol=tol, max_iter=50000, check_every=8)
    sw = None
    use_sw = any(m.startswith("schwarz") for m in methods)
    if use_sw:
        gc = binding.Mesh(1, case.nel, case.periodic, case.faces, case.vertices(), geom_f32=True)
        sw = binding.Schwarz(gm, gc)
        schwarz = gm.pcg_opts(tol=tol, max_iter=50000, precision=binding.SEM_PCG_MIXED,
                              inner_tol=schwarz_inner_tol,
                              use_initial_guess=True, check_every=8, schwarz=sw, coarse_iters=3, coarse_tol=1e-2,
                              inner_adapt=inner_adapt)
        gmid = binding.Mesh(3, case.nel, case.periodic, case.faces, case.vertices(), geom_f32=True)
        swmid = binding.Schwarz(gmid, gc)
        schwarz3 = gm.pcg_opts(tol=tol, max_iter=50000, precision=binding.SEM_PCG_MIXED,
                               inner_tol=schwarz_inner_tol,
                               use_initial_guess=True, check_every=8, schwarz=sw, coarse_iters=3, coarse_tol=1e-2,
                               schwarz_mid=swmid, mid_weight=0.15, inner_adapt=inner_adapt)
    phase1_opts = schwarz if use_sw else chosen
    g = GuessNet(gm, hidden, seed, variant, pair)

    # ---- phase 1: simulate and collect samples
    Xs, Ts = [], []
    phase1 = []
    p4 = torch.zeros(gm.nloc, dtype=torch.float64, device="cuda")  # pressure four steps back
    for n in range(1, train_steps + 1):
        ns.step_begin(dt)
        p1, p2, p3, b = ns.get(3), ns.get(4), ns.get(5), ns.get(6)
        have = n >= 4
        take = have and n >= max(skip, 6) and (variant == "p1" or g.rho_prev is not None)
        if have:
            g.residual(b, p1, p2, p3)
            if take:
                g.set_scales(p1, p2, p3, p4)
                g.features(p1, p2, p3, p4)
        ps, vs = ns.step_finish(phase1_opts, vopts)
        phase1.append((ps["iters"], ps["wall_ms"]))
        if have:
            p_new = ns.get(3)
            # variant "p1": rho measured once, on the first sample; "d3": every step
            if variant == "d3" or (take and g.rho_prev is None):
                g.update_rho(p_new)
            if take:
                T = torch.zeros((g.R, g.O), dtype=torch.float32, device="cuda")
                g.target(p_new, p1, p2, p3, T)
                Xs.append(g.X.clone())
                Ts.append(T)
        p4 = p3
    torch.cuda.synchronize()
    log(f"phase 1: {train_steps} steps, {len(Xs)} samples")

    # ---- phase 2: train
    t0 = time.perf_counter()
    rng = np.random.default_rng(seed)
    total = epochs * len(Xs)
    losses = []
    ework = torch.empty(2 * gm.nloc, dtype=torch.float32, device="cuda") if loss != "mse" else None
    k = 0
    for ep in range(epochs):
        for i in rng.permutation(len(Xs)):
            lr_k = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * k / max(total - 1, 1))))
            if loss in ("energy", "energy_avg"):
                li = g.net.grad_energy(Xs[i], Ts[i], gm, lam, assembled=loss == "energy_avg", work=ework)
            else:
                li = g.net.grad(Xs[i], Ts[i], rows_real=g.E, outs_real=g.npt)
            g.net.adam(lr_k)
            losses.append(li)
            k += 1
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # loss of the zero correction: 0.5 mean(T^2)
    log(f"phase 2: {k} Adam steps in {train_s:.2f} s, loss {losses[0]:.4f} -> {losses[-1]:.4f}")
    del Xs, Ts

    # ---- phase 3: evaluate every method from the same checkpoint
    ck = ns.checkpoint()
    p4_ck = p4.clone()
    rho_ck = g.rho_prev
    results = {}
    by_solver = {"plain": plain, "chosen": chosen}
    if use_sw:
        gmo = binding.PcgOpts.from_buffer_copy(schwarz)
        gmo.krylov, gmo.gmres_restart, gmo.inner_tol = binding.SEM_KRYLOV_FGMRES, 30, 1e-2
        by_solver.update(schwarz=schwarz, schwarz3=schwarz3, schwarzgm=gmo)
    for meth in methods:
        solver, gkind, fixed = _method(meth)
        popts = by_solver[solver]
        if fixed:
            popts = binding.PcgOpts.from_buffer_copy(popts)
            popts.inner_adapt, popts.inner_tol = 0.0, 1e-2
        ns.restore(ck)
        p4 = p4_ck.clone()
        g.rho_prev = rho_ck
        iters, pms, gms, gerr, r0 = [], [], [], [], []
        for n in range(eval_steps):
            ns.step_begin(dt)
            p1, p2, p3, b = ns.get(3), ns.get(4), ns.get(5), ns.get(6)
            torch.cuda.synchronize()
            tg = time.perf_counter()
            guess = None
            if gkind == "extrap":
                guess = g.extrap(p1, p2, p3)
                torch.cuda.synchronize()
            elif gkind == "learned":
                g.residual(b, p1, p2, p3)
                g.set_scales(p1, p2, p3, p4)
                g.features(p1, p2, p3, p4)
                guess = g.predict(p1, p2, p3)
                torch.cuda.synchronize()
            guess_ms = (time.perf_counter() - tg) * 1e3
            x0 = guess if guess is not None else p1
            x0c = x0.clone()
            ps, vs = ns.step_finish(popts, vopts, p_guess=guess)
            p_new = ns.get(3)
            if gkind == "learned" and variant == "d3":
                g.update_rho(p_new)
            err = math.sqrt(gm.glsc3(x0c - p_new, x0c - p_new) / max(gm.glsc3(p_new, p_new), 1e-300))
            iters.append(ps["iters"])
            pms.append(ps["wall_ms"] + guess_ms)
            gms.append(guess_ms)
            gerr.append(err)
            r0.append(ps["init_rel_res"])
            p4 = p3
        results[meth] = {"pressure_ms_total": round(float(np.sum(pms)), 1),
                         "pressure_ms_mean": round(float(np.mean(pms)), 2),
                         "guess_ms_mean": round(float(np.mean(gms)), 3),
                         "iters_mean": round(float(np.mean(iters)), 1), "iters_total": int(np.sum(iters)),
                         "guess_rel_err_mean": float(np.mean(gerr)),
                         "guess_rel_residual_mean": float(np.mean(r0)), "energy_final": ns.kinetic_energy()}
        log(meth, results[meth])
    out = {"workload": f"TGV Re={Re:g}, {nel}^3 elements, N={N}, dt={dt:g}, steps 1-{train_steps} train, "
                       f"{train_steps + 1}-{train_steps + eval_steps} evaluate, tol {tol:g}",
           "train": {"samples": len(losses) // max(epochs, 1), "adam_steps": k, "seconds": round(train_s, 3),
                     "loss_first": losses[0], "loss_last": losses[-1],
                     "network": f"{g.I}-{g.H}-{g.H}-{g.O} BF16 (tcgen05), {g.net.P} parameters",
                     "variant": variant, "loss": loss, "lam": lam if loss != "mse" else None,
                     "pair_residual": bool(pair)},
           "phase1_iters_mean": float(np.mean([a for a, _ in phase1])),
           "phase1_solver": "schwarz" if use_sw else "chosen",
           "methods": results, "wall_s": round(time.perf_counter() - t_all, 1)}
    base = results.get("plain_f64_prev")
    if base:
        for m, r in results.items():
            r["speedup_vs_plain_f64_prev"] = round(base["pressure_ms_total"] / r["pressure_ms_total"], 3)
    return out

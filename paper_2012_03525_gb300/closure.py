"""Learned-closure workflow: generate training data with the solver itself,
train the closure network on the GPU, and measure what it gains.

Set-up (2D decaying turbulence): a periodic box of side L = 2 pi, random-phase
initial spectrum E(k) ~ k^4 exp(-2 (k/k0)^2), u_rms = 0.05, nu = 5e-4 (all in
physical units), one time step dt for every grid.  A fine N_f^2 FP64 run of
the scheme is the reference; a coarse (N_f / factor)^2 FP32 run starts from
the box-filtered fine state.  Lattice units per grid: delta_x = L / N,
u_lat = u dt / delta_x, nu_lat = nu dt / delta_x^2, and the density deviation
(pressure signal) scales with delta_x^2 at fixed dt.

Training sample for one window of `window` steps: input = the coarse state
after `window` coarse steps started from the filtered fine state; target = the
filtered fine state after the same time.  The closure learns the correction
applied once per window.  Every arithmetic step runs in libacm's kernels;
PyTorch only provides device buffers.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import acm
from . import workloads as wl


@dataclasses.dataclass
class Setup:
    n_fine: int = 1024
    factor: int = 4
    u_rms: float = 0.05
    nu: float = 5e-4
    dt: float = 6e-3
    L: float = 2 * math.pi
    k0: float = 8.0
    window: int = 8

    @property
    def n_coarse(self):
        return self.n_fine // self.factor

    def lattice(self, n):
        dx = self.L / n
        return self.u_rms * self.dt / dx, self.nu * self.dt / dx ** 2

    def params(self, n, precision):
        _, nu_lat = self.lattice(n)
        return acm.make_params((n, n), nu=nu_lat, precision=precision)

    def scales(self):
        """Normalisation of the coarse state: u by u_rms, rho' by its O(Ma^2)
        scale 3 u_rms^2 (lattice units of the coarse grid)."""
        u_c, _ = self.lattice(self.n_coarse)
        return 1.0 / (3.0 * u_c * u_c), 1.0 / u_c

    def initial(self, seed, n=None):
        n = self.n_fine if n is None else n
        u_lat, _ = self.lattice(n)
        return wl.turbulence2d(n, seed, u_rms=u_lat, k0=self.k0)


def _fine(setup, seeds, n=None, precision=acm.FP64):
    n = setup.n_fine if n is None else n
    s = acm.Solver([setup.params(n, precision) for _ in seeds])
    for i, seed in enumerate(seeds):
        s.set_fields(*setup.initial(seed, n), run=i)
    return s


def generate(setup, seeds, windows, torch, batch, model=None, reset=False, reset_every=0):
    """Training samples, (X, Y) device tensors [nsamples][batch][3][nc][nc]
    (normalised): inputs are coarse states after each window, targets the
    filtered fine states at the same times.  The coarse run starts from the
    filtered fine state and then runs freely (with ``reset`` it restarts from
    the filtered fine state every window instead; with ``reset_every`` = r > 0
    every r windows).  With a trained ``model`` the closure is applied after
    every window, so the inputs are the states the closure meets in use (the
    data-aggregation remedy for the drift of a corrected run away from the
    training states; with a small r the drift is the model's own over r - 1
    corrected windows)."""
    if reset:
        reset_every = 1
    nc = setup.n_coarse
    sr, su = setup.scales()
    closure = model
    if closure is None:
        closure = acm.Closure(nc, nc, batch)
        closure.set_scales(sr, su)
    xs, ys = [], []
    for c0 in range(0, len(seeds), batch):
        group = list(seeds[c0:c0 + batch])
        if len(group) < batch:
            break
        fine = _fine(setup, group)
        coarse = acm.Solver([setup.params(nc, acm.FP32_DEV) for _ in group])
        fine.restrict_to(coarse, setup.factor)
        for k in range(windows):
            if reset_every > 0 and k % reset_every == 0:
                fine.restrict_to(coarse, setup.factor)
            coarse.step(setup.window)
            fine.step(setup.window)
            x = torch.empty((batch, 3, nc, nc), device="cuda", dtype=torch.float32)
            y = torch.empty_like(x)
            closure.gather(coarse, x.data_ptr())
            fine.restrict_to(None, setup.factor, out_dev=y.data_ptr(), scales=(sr, su))
            xs.append(x)
            ys.append(y)
            if model is not None:
                model.apply(coarse)
        fine.sync()
        coarse.sync()
        fine.close()
        coarse.close()
    if model is None:
        closure.close()
    return torch.stack(xs), torch.stack(ys)


def he_init(seed=0, scale_out=1e-2):
    """He-style initial weights in the library's flat order (per layer
    W[co][ci][3][3], then b[co]); the output layer starts near zero so the
    untrained closure is close to no correction."""
    rng = np.random.default_rng(seed)
    chans = (3, 32, 32, 3)
    parts = []
    for l in range(3):
        cin, cout = chans[l], chans[l + 1]
        std = math.sqrt(2.0 / (9 * cin)) * (scale_out if l == 2 else 1.0)
        parts.append(rng.standard_normal(cout * cin * 9) * std)
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)


def train(setup, X, Y, torch, batch, epochs=20, lr=1e-3, seed=0, closure=None, noise=0.0):
    """Adam on the stored samples (shuffled each epoch); returns the trained
    closure and the mean loss of every epoch.  A given ``closure`` continues
    from its current weights.  ``noise`` > 0 perturbs the training inputs
    (acm_closure_set_input_noise) so the network also learns to pull
    perturbed states back toward the reference."""
    nc = setup.n_coarse
    sr, su = setup.scales()
    if closure is None:
        closure = acm.Closure(nc, nc, batch)
        closure.set_scales(sr, su)
        # fit and correct the velocity only: the density deviation carries
        # acoustic waves whose speed differs between the coarse and fine
        # lattices, so it is left to the scheme
        closure.set_loss_weights(0.0, 1.0)
        closure.set_weights(he_init(seed))
    closure.set_input_noise(noise, seed)
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = rng.permutation(X.shape[0])
        tot = 0.0
        for k in order:
            tot += closure.train_step(X[k].data_ptr(), Y[k].data_ptr(), lr)
        losses.append(tot / len(order))
    closure.set_input_noise(0.0)
    return closure, losses


def evaluate(setup, closure, seeds, windows, torch, batch):
    """Coarse runs with and without the closure against the filtered fine
    reference after `windows` windows; relative L2 of the velocity (u, v)."""
    nc = setup.n_coarse
    sr, su = setup.scales()
    fine = _fine(setup, seeds)
    plain = acm.Solver([setup.params(nc, acm.FP32_DEV) for _ in seeds])
    corr = acm.Solver([setup.params(nc, acm.FP32_DEV) for _ in seeds])
    fine.restrict_to(plain, setup.factor)
    fine.restrict_to(corr, setup.factor)
    for _ in range(windows):
        fine.step(setup.window)
        plain.step(setup.window)
        corr.step(setup.window)
        closure.apply(corr)
    ref = torch.empty((batch, 3, nc, nc), device="cuda", dtype=torch.float32)
    fine.restrict_to(None, setup.factor, out_dev=ref.data_ptr(), scales=(sr, su))
    xp = torch.empty_like(ref)
    xc = torch.empty_like(ref)
    closure.gather(plain, xp.data_ptr())
    closure.gather(corr, xc.data_ptr())
    torch.cuda.synchronize()

    def err(a):
        d = (a[:, 1:] - ref[:, 1:]).double()
        return float(torch.sqrt((d * d).sum() / (ref[:, 1:].double() ** 2).sum()))

    out = {"plain": err(xp), "closure": err(xc)}
    for h in (fine, plain, corr):
        h.close()
    return out


def fit(setup, train_seeds, windows, torch, batch, epochs=20, lr=1e-3, rounds=2, seed=0):
    """Train on one-window samples, then `rounds - 1` times add samples from
    free coarse runs corrected by the current closure and continue training.
    Returns (closure, per-round loss histories)."""
    X, Y = generate(setup, train_seeds, windows, torch, batch)
    closure, losses = train(setup, X, Y, torch, batch, epochs, lr, seed)
    hist = [losses]
    for _ in range(rounds - 1):
        X2, Y2 = generate(setup, train_seeds, windows, torch, batch, model=closure)
        X = torch.cat([X, X2])
        Y = torch.cat([Y, Y2])
        closure, losses = train(setup, X, Y, torch, batch, epochs, lr * 0.5, seed, closure)
        hist.append(losses)
    return closure, hist


# (restart interval in windows, epochs, learning rate) of each aggregation round
PUSHFORWARD_SCHEDULE = ((2, 10, 5e-4), (3, 10, 5e-4), (4, 10, 5e-4), (6, 10, 2.5e-4),
                        (8, 10, 2.5e-4), (12, 10, 2.5e-4))


def fit_pushforward(setup, train_seeds, windows, torch, batch, schedule=PUSHFORWARD_SCHEDULE,
                    epochs=20, lr=1e-3, seed=0):
    """Train on one-window samples (every window restarted from the filtered
    fine state), then for each (r, epochs, lr) of ``schedule`` add samples
    from coarse runs corrected by the current closure and restarted from the
    filtered fine state every r windows, and continue training on all
    samples.  Each round teaches the closure to pull back the drift that its
    own corrections leave over r - 1 windows (its inputs are the states it
    meets in use, its targets the filtered fine states at the same times), so
    the corrected free run stays near the reference for longer; with
    one-window samples only, the corrected run drifts off after 3-4 windows
    and diverges.  Returns (closure, per-round loss histories)."""
    X, Y = generate(setup, train_seeds, windows, torch, batch, reset=True)
    closure, losses = train(setup, X, Y, torch, batch, epochs, lr, seed)
    hist = [losses]
    for r_every, ep, lr_r in schedule:
        X2, Y2 = generate(setup, train_seeds, windows, torch, batch, model=closure,
                          reset_every=r_every)
        X = torch.cat([X, X2])
        Y = torch.cat([Y, Y2])
        del X2, Y2
        closure, losses = train(setup, X, Y, torch, batch, ep, lr_r, seed, closure)
        hist.append(losses)
    del X, Y
    return closure, hist


def evaluate_windows(setup, closure, seeds, windows, torch, batch):
    """One-window errors on held-out initial conditions: every window both
    coarse runs restart from the filtered fine state, run `window` steps, and
    one of them is corrected by the closure; relative L2 of the velocity
    against the filtered fine state, averaged over the windows."""
    nc = setup.n_coarse
    sr, su = setup.scales()
    fine = _fine(setup, seeds)
    plain = acm.Solver([setup.params(nc, acm.FP32_DEV) for _ in seeds])
    corr = acm.Solver([setup.params(nc, acm.FP32_DEV) for _ in seeds])
    ref = torch.empty((batch, 3, nc, nc), device="cuda", dtype=torch.float32)
    xp = torch.empty_like(ref)
    xc = torch.empty_like(ref)

    def err(a):
        d = (a[:, 1:] - ref[:, 1:]).double()
        return float(torch.sqrt((d * d).sum() / (ref[:, 1:].double() ** 2).sum()))

    ep, ec = [], []
    for _ in range(windows):
        fine.restrict_to(plain, setup.factor)
        fine.restrict_to(corr, setup.factor)
        fine.step(setup.window)
        plain.step(setup.window)
        corr.step(setup.window)
        closure.apply(corr)
        fine.restrict_to(None, setup.factor, out_dev=ref.data_ptr(), scales=(sr, su))
        closure.gather(plain, xp.data_ptr())
        closure.gather(corr, xc.data_ptr())
        torch.cuda.synchronize()
        ep.append(err(xp))
        ec.append(err(xc))
    for h in (fine, plain, corr):
        h.close()
    return {"plain": float(np.mean(ep)), "closure": float(np.mean(ec))}


def rollout_curve(setup, closure, seeds, windows, torch, batch):
    """Free runs from the filtered fine state at t = 0 to t = windows x
    window x dt: velocity error (relative L2 against the filtered fine FP64
    run, on the coarse grid) after every window and the wall time of the run
    (stepping only, synchronised), for the plain scheme at n_coarse (FP32 and
    FP64) and 2 n_coarse (FP64) and for the corrected n_coarse FP32 run (the
    closure applied after every window).  The fine run itself is the
    reference (error 0); its wall time is reported too."""
    nc, f = setup.n_coarse, setup.factor
    sr, su = setup.scales()
    fine = _fine(setup, seeds)
    refs = []
    for _ in range(windows):
        fine.step(setup.window)
        r = torch.empty((batch, 3, nc, nc), device="cuda", dtype=torch.float32)
        fine.restrict_to(None, f, out_dev=r.data_ptr(), scales=(sr, su))
        refs.append(r)
    fine.sync()

    def err(a, ref):
        d = (a[:, 1:] - ref[:, 1:]).double()
        return float(torch.sqrt((d * d).sum() / (ref[:, 1:].double() ** 2).sum()))

    configs = {"plain_coarse_fp32": (nc, acm.FP32_DEV, False),
               "plain_coarse_fp64": (nc, acm.FP64, False),
               "plain_2coarse_fp64": (2 * nc, acm.FP64, False),
               "closure_coarse_fp32": (nc, acm.FP32_DEV, True)}
    out = {}
    x = torch.empty((batch, 3, nc, nc), device="cuda", dtype=torch.float32)
    for name, (n, prec, corrected) in configs.items():
        start = _fine(setup, seeds)
        errs, secs = [], 0.0
        for timed in (False, True):
            run = acm.Solver([setup.params(n, prec) for _ in seeds])
            start.restrict_to(run, setup.n_fine // n)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                for k in range(windows):
                    run.step(setup.window)
                    if corrected:
                        closure.apply(run)
                    if not timed:
                        # the run's velocity on the coarse grid, normalised
                        # (factor 1: a scaled copy of an FP64 or FP32 run)
                        run.restrict_to(None, n // nc, out_dev=x.data_ptr(), scales=(sr, su),
                                        u_scale=nc / n, rho_scale=(nc / n) ** 2)
                        torch.cuda.synchronize()
                        errs.append(err(x, refs[k]))
                run.sync()
            except acm.AcmError:
                errs.append(float("inf"))
            if timed:
                secs = time.perf_counter() - t0
            run.close()
        start.close()
        out[name] = {"error_per_window": errs, "final_error": errs[-1], "seconds": secs}
    fine.close()
    # the fine reference run's own wall time over the same horizon
    ref = _fine(setup, seeds)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref.step(windows * setup.window)
    ref.sync()
    out["plain_fine_fp64"] = {"final_error": 0.0, "seconds": time.perf_counter() - t0}
    ref.close()
    return out

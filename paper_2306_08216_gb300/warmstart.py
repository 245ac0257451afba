"""Learned warm start: binding of the warm-start network (include/mdf_net.h)
and the pipeline around it.

The network predicts the steady state of a power-law lid-driven cavity from
(Re, n); the solver then marches from that prediction (mdf_init_fields) to
its own steady state, so the network only changes where the march starts.
The paper has no learned component; this is an extension of the library.

Every step runs in libmdf.so; this module marshals arguments, holds the
seeded training loop and moves fields between the network and the solver
on the device.
"""
import ctypes
import math
import os

import numpy as np

from . import mdf
from . import workloads as W

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
U_LID = 0.1  # lid speed of the cavities the network is trained on


class Net:
    """The warm-start U-Net on R x R fields, batches of at most max_batch."""

    def __init__(self, resolution, max_batch, stream=None):
        L = mdf.lib()
        h = ctypes.c_void_p()
        st = L.mdf_net_create(resolution, max_batch, ctypes.byref(h))
        if st != mdf.MDF_OK:
            raise mdf.MdfError(st, L.mdf_net_last_error(None).decode())
        self._h = h
        self.R, self.max_batch = resolution, max_batch
        self.param_count = int(L.mdf_net_param_count(h))
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
            self._chk(L.mdf_net_set_stream(h, ctypes.c_void_p(raw or 0)))

    def _chk(self, st):
        if st != mdf.MDF_OK:
            raise mdf.MdfError(st, mdf.lib().mdf_net_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            mdf.lib().mdf_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_conv_kernel(self, kind):
        """"tcgen05" (default: tensor-memory MMA where it applies) or
        "mma.sync" for every convolution."""
        self._chk(mdf.lib().mdf_net_set_conv_kernel(self._h, {"tcgen05": 0, "mma.sync": 1}[kind]))

    def layer_shapes(self):
        L = mdf.lib()
        out = []
        for k in range(L.mdf_net_layer_count(self._h)):
            s = (ctypes.c_int * 2)()
            self._chk(L.mdf_net_layer_shape(self._h, k, s))
            out.append((int(s[0]), int(s[1])))
        return out

    @staticmethod
    def _ptr(a):
        if hasattr(a, "data_ptr"):
            return ctypes.c_void_p(a.data_ptr()), 1
        return a.ctypes.data_as(ctypes.c_void_p), 0

    def set_params(self, p):
        if hasattr(p, "data_ptr"):
            assert p.numel() == self.param_count
            self._chk(mdf.lib().mdf_net_set_params(self._h, ctypes.c_void_p(p.data_ptr()), 1))
            return
        a = np.ascontiguousarray(p, dtype=np.float32)
        assert a.size == self.param_count, (a.size, self.param_count)
        self._chk(mdf.lib().mdf_net_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p), 0))

    def get_params(self):
        a = np.empty(self.param_count, dtype=np.float32)
        self._chk(mdf.lib().mdf_net_get_params(self._h, a.ctypes.data_as(ctypes.c_void_p), 0))
        return a

    def _batch_args(self, inputs, targets=None):
        if hasattr(inputs, "data_ptr"):
            B = int(inputs.shape[0])
            assert inputs.is_contiguous() and tuple(inputs.shape[1:]) == (W.WARM_IN_PLANES, self.R, self.R)
            tp = ctypes.c_void_p(targets.data_ptr()) if targets is not None else None
            return B, ctypes.c_void_p(inputs.data_ptr()), tp, 1, (inputs, targets)
        x = np.ascontiguousarray(inputs, dtype=np.float32)
        assert x.shape[1:] == (W.WARM_IN_PLANES, self.R, self.R), x.shape
        t = None if targets is None else np.ascontiguousarray(targets, dtype=np.float32)
        tp = None if t is None else t.ctypes.data_as(ctypes.c_void_p)
        return x.shape[0], x.ctypes.data_as(ctypes.c_void_p), tp, 0, (x, t)

    def forward(self, inputs, out=None):
        """Outputs [B][3][R][R]: numpy for host inputs; for device (torch)
        inputs, written into `out` (a device tensor) or a new one."""
        B, xp, _, dev, keep = self._batch_args(inputs)
        if dev:
            import torch
            if out is None:
                out = torch.empty((B, 3, self.R, self.R), dtype=torch.float32, device=inputs.device)
            self._chk(mdf.lib().mdf_net_forward(self._h, B, xp, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        y = np.empty((B, 3, self.R, self.R), dtype=np.float32)
        self._chk(mdf.lib().mdf_net_forward(self._h, B, xp, y.ctypes.data_as(ctypes.c_void_p), 0))
        return y

    def gradient(self, inputs, targets):
        B, xp, tp, dev, keep = self._batch_args(inputs, targets)
        g = np.empty(self.param_count, dtype=np.float32)
        loss = ctypes.c_double()
        if dev:
            import torch
            gd = torch.empty(self.param_count, dtype=torch.float32, device=inputs.device)
            self._chk(mdf.lib().mdf_net_gradient(self._h, B, xp, tp, ctypes.byref(loss),
                                                 ctypes.c_void_p(gd.data_ptr()), 1))
            return loss.value, gd.cpu().numpy()
        self._chk(mdf.lib().mdf_net_gradient(self._h, B, xp, tp, ctypes.byref(loss),
                                             g.ctypes.data_as(ctypes.c_void_p), 0))
        return loss.value, g

    def train_step(self, inputs, targets, lr, want_loss=True):
        B, xp, tp, dev, keep = self._batch_args(inputs, targets)
        loss = ctypes.c_double()
        self._chk(mdf.lib().mdf_net_train_step(self._h, B, xp, tp, float(lr),
                                               ctypes.byref(loss) if want_loss else None, dev))
        return loss.value if want_loss else None

    def save(self, path):
        np.save(path, self.get_params())

    def load(self, path):
        self.set_params(np.load(path))


# ---------------------------------------------------------------- pipeline

def cavity_problem(R, re, n_index, u0=U_LID, geometry="square"):
    """Keyword arguments (for mdf.Solver / mdf.Batch) of a power-law
    lid-driven cavity on R x R nodes: Re = u0^(2-n) L^n / K with L = 1 (the
    lid width), nu clamped to [nu_ref / 20, 20 nu_ref], nu_ref = K (u0/L)^(n-1);
    geometry "square" (the unit square, uniform grid) or "trapezoid" (the
    body-fitted isosceles trapezoid of workloads.trapezoid_grid, lid on top)."""
    K = u0 ** (2.0 - n_index) / re
    nu_ref = K * u0 ** (n_index - 1.0)
    kw = dict(nx=R, ny=R, nu=nu_ref, walls=(True, True), u_wall=(0, 0, 0, u0),
              power_law=(K, float(n_index), nu_ref / 20.0, nu_ref * 20.0))
    if geometry == "trapezoid":
        X, Y = W.trapezoid_grid(R, R)
        kw.update(grid="curvilinear", x=X, y=Y)
    return kw


def march(batch, target, check_every=1000, max_steps=500_000, max_seconds=None, log=None, log_every=50,
          retire=False, patience=1):
    """Step a batch until every problem's windowed residual (mdf_residual,
    window `check_every`) is <= target, diverged, max_steps or max_seconds
    of wall time.  With retire=True a problem leaves the batch
    (mdf_batch_set_active) once it meets the target or diverges, so the
    others no longer pay for it.  A problem meets the target once its
    residual has been <= target for `patience` consecutive checks (a
    residual window that happens to see a slowly oscillating flow near the
    same phase can be small once).  Returns (step count at which each
    problem met the target, -1 if never; final residuals; statuses; steps
    taken; wall seconds at which each problem met the target, NaN if never)."""
    import time
    conv = np.full(batch.count, -1, dtype=np.int64)
    when = np.full(batch.count, np.nan)
    last_r = np.full(batch.count, np.nan)
    last_st = np.zeros(batch.count, dtype=np.int64)
    gone = np.zeros(batch.count, dtype=bool)
    below = np.zeros(batch.count, dtype=np.int64)  # consecutive checks at or below target
    steps, checks = 0, 0
    r = st = None
    t0 = time.perf_counter()
    while steps < max_steps:
        batch.step(check_every)
        steps += check_every
        r, st = batch.residual()
        live = ~gone
        last_r[live], last_st[live] = r[live], st[live]
        r, st = last_r.copy(), last_st.copy()
        below[live] = np.where((r[live] <= target) & (st[live] == mdf.MDF_OK), below[live] + 1, 0)
        newly = (below >= patience) & (conv < 0)
        conv[newly] = steps
        when[newly] = time.perf_counter() - t0
        if retire:
            for i in np.nonzero(live & (newly | (st == mdf.MDF_E_DIVERGED)))[0]:
                batch.set_active(int(i), False)
                gone[i] = True
        checks += 1
        done = np.all((conv >= 0) | (st == mdf.MDF_E_DIVERGED))
        el = time.perf_counter() - t0
        if log and (checks % log_every == 0 or done):
            fin = r[np.isfinite(r)]
            log("  %d steps %.1f s: %d/%d at target, residual min %.2e median %.2e max %.2e"
                % (steps, el, int((conv >= 0).sum()), batch.count, fin.min() if fin.size else float("nan"),
                   np.median(fin) if fin.size else float("nan"), fin.max() if fin.size else float("nan")))
        if done or (max_seconds is not None and el > max_seconds):
            break
    return conv, r, st, steps, when


P_CLIP = 2.0  # |p| / u0^2 above this (the lid corners' pressure spikes) is clipped in the targets


def steady_fields(batch, u0=U_LID):
    """Training targets of every problem, [count][3][R][R]: u / u0, v / u0 and
    the pressure relative to its mean over the nodes, / u0^2, clipped to
    [-P_CLIP, P_CLIP].  Only pressure differences are defined by the
    incompressible flow: the level that the march leaves in P depends on
    how long it ran (it drifts slowly with the walls' mass balance), so it
    is not a property of the steady state the network could learn.  The
    pressure of the two lid corners is singular; unclipped, its few nodes
    would dominate the mean-square loss."""
    out = []
    for i in range(batch.count):
        f = batch.problem(i).fields(["u", "v", "P"])
        p = f["P"].astype(np.float64)
        p = (p - p.mean()) / u0 ** 2
        out.append(np.stack([f["u"] / u0, f["v"] / u0, np.clip(p, -P_CLIP, P_CLIP)]))
    return np.asarray(out, dtype=np.float32)


def generate_dataset(count, seed, R, target=1e-6, check_every=1000, max_steps=200_000, trapezoid_fraction=0.3,
                     stream=None, log=print):
    """Steady power-law cavities from seeded (Re, n) draws, the first
    (1 - trapezoid_fraction) of them on the unit square and the rest on the
    body-fitted trapezoid, each geometry marched from rest as one batch
    until every problem has met the target for three consecutive checks or
    max_steps.  Only the problems that met it and still meet it at the end
    are kept (some power-law cavities settle into a small persistent
    oscillation above it, and some diverge).  Returns inputs [k][8][R][R],
    targets [k][3][R][R] and a summary."""
    re, nn = W.warm_start_draws(count, seed)
    n_sq = count - int(round(trapezoid_fraction * count))
    geo = np.array(["square"] * n_sq + ["trapezoid"] * (count - n_sq))
    xs, ts, keep_re, keep_n, keep_geo, parts = [], [], [], [], [], {}
    for g in ("square", "trapezoid"):
        idx = np.nonzero(geo == g)[0]
        if idx.size == 0:
            continue
        batch = mdf.Batch([cavity_problem(R, re[i], nn[i], geometry=g) for i in idx], stream=stream)
        # every problem keeps marching to the end (a converged state only
        # improves), and is kept if it met the target for three consecutive
        # checks and still meets it at the last one
        conv, r, st, steps, _ = march(batch, target, check_every, max_steps, log=log, log_every=50, retire=False,
                                      patience=3)
        ok = (conv >= 0) & (r <= target)
        t = steady_fields(batch)
        batch.close()
        ts.append(t[ok])
        keep_re.append(re[idx][ok])
        keep_n.append(nn[idx][ok])
        keep_geo += [g] * int(ok.sum())
        parts[g] = {"drawn": int(idx.size), "kept": int(ok.sum()), "diverged": int((st == mdf.MDF_E_DIVERGED).sum()),
                    "steps": steps, "median_steps_to_target": float(np.median(conv[ok])) if ok.any() else None}
        log("dataset seed %d, %s: kept %d of %d (at target %.0e) after %d steps"
            % (seed, g, int(ok.sum()), idx.size, target, steps))
    re_k, n_k = np.concatenate(keep_re), np.concatenate(keep_n)
    x = W.warm_start_inputs(re_k, n_k, R, geometry=keep_geo)
    info = {"count": count, "seed": seed, "R": R, "target": target, "max_steps": max_steps,
            "kept": int(re_k.size), "geometries": parts, "re": re_k.tolist(), "n": n_k.tolist(), "geometry": keep_geo}
    return x, np.concatenate(ts), info


def split_holdout(n, fraction, seed):
    """Seeded split of n samples: (train indices, held-out indices)."""
    order = np.random.default_rng(seed).permutation(n)
    k = int(round(fraction * n))
    return np.sort(order[k:]), np.sort(order[:k])


def init_params(net, seed):
    """Seeded He initialisation over the library's own layer table."""
    shapes = [(str(k), co, ci) for k, (co, ci) in enumerate(net.layer_shapes())]
    return W.net_init_params(shapes, seed)


def train(x, t, epochs, batch=16, lr=1e-3, lr_final=2e-5, seed=0, init_seed=2306, stream=None, log=print,
          log_every=10):
    """Train a fresh network (seeded He initialisation) with Adam on the mean
    square loss, cosine learning-rate decay from lr to lr_final, seeded
    shuffling; the last partial batch of an epoch is dropped.  Returns the
    network and the per-epoch mean losses."""
    R = x.shape[-1]
    net = Net(R, batch, stream=stream)
    net.set_params(init_params(net, init_seed))
    rng = np.random.default_rng(seed)
    per_epoch = len(x) // batch
    total = epochs * per_epoch
    history = []
    k = 0
    for ep in range(epochs):
        order = rng.permutation(len(x))
        acc = 0.0
        for j in range(per_epoch):
            idx = np.sort(order[j * batch:(j + 1) * batch])
            lr_k = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * k / max(total - 1, 1)))
            acc += net.train_step(x[idx], t[idx], lr_k)
            k += 1
        history.append(acc / per_epoch)
        if log and (ep % log_every == 0 or ep == epochs - 1):
            log("epoch %d loss %.4e" % (ep, history[-1]))
    return net, history


def evaluate(net, x, t, chunk=16):
    """Per-sample relative L2 errors of the predicted velocity (u, v) and
    pressure against the targets."""
    eu, ep = [], []
    for i in range(0, len(x), chunk):
        y = net.forward(x[i:i + chunk])
        tt = t[i:i + chunk]
        for b in range(len(y)):
            eu.append(float(np.linalg.norm(y[b, :2] - tt[b, :2]) / np.linalg.norm(tt[b, :2])))
            ep.append(float(np.linalg.norm(y[b, 2] - tt[b, 2]) / max(np.linalg.norm(tt[b, 2]), 1e-30)))
    return np.array(eu), np.array(ep)


def predict(net, x, chunk=None):
    chunk = chunk or net.max_batch
    return np.concatenate([net.forward(x[i:i + chunk]) for i in range(0, len(x), chunk)])


def warm_vs_cold(net, re, nn, R, target=1e-8, check_every=1000, max_steps=150_000, max_seconds=None,
                 stream=None, log=print, geometry="square"):
    """The same cavities marched to residual `target` from rest (cold) and
    from the network's prediction (warm), each set as one batch that retires
    problems as they converge; plus the device time per step of one cavity
    stepped alone (one launch per step), from which the cold march of the
    cavities one launch per problem is extrapolated.  Some power-law cavities
    settle into a persistent small oscillation above low targets (the FP64
    oracle does the same); wall times compare the problems that reach the
    target in both marches."""
    import time

    import torch

    probs = [cavity_problem(R, a, b, geometry=geometry) for a, b in zip(re, nn)]
    t0 = time.perf_counter()
    y = predict(net, W.warm_start_inputs(re, nn, R, geometry=geometry))
    predict_s = time.perf_counter() - t0
    out = {"problems": len(probs), "R": R, "target": target, "check_every": check_every, "max_steps": max_steps,
           "predict_seconds": predict_s}
    for mode in ("cold", "warm"):
        b = mdf.Batch(probs, stream=stream)
        if mode == "warm":
            for i in range(len(probs)):
                b.init(i, y[i, 0] * U_LID, y[i, 1] * U_LID, y[i, 2] * U_LID ** 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        conv, r, st, steps, when = march(b, target, check_every, max_steps, max_seconds, log=None, retire=True)
        sec = time.perf_counter() - t0
        out[mode] = {"steps_to_target": conv.tolist(), "seconds_to_target": [float(v) for v in when],
                     "batch_steps": steps, "seconds": sec, "final_residual": [float(v) for v in r],
                     "reached": int((conv >= 0).sum()), "diverged": int((st == mdf.MDF_E_DIVERGED).sum())}
        if log:
            log("%s: %d of %d reached %.0e within %d steps" % (mode, out[mode]["reached"], len(probs), target, steps))
        b.close()
    # one cavity alone, one launch per step: device time per step
    s = mdf.Solver(R, R, stream=stream, **{k: v for k, v in probs[0].items() if k not in ("nx", "ny")})
    s.step(100)
    s.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st_ = torch.cuda.current_stream() if stream is None else stream
    e0.record(st_)
    s.step(2000)
    e1.record(st_)
    e1.synchronize()
    solo_ms = e0.elapsed_time(e1) / 2000
    s.close()
    c = np.array(out["cold"]["steps_to_target"], dtype=np.float64)
    w = np.array(out["warm"]["steps_to_target"], dtype=np.float64)
    both = (c > 0) & (w > 0)
    out["reached_both"] = int(both.sum())
    out["solo_ms_per_step"] = solo_ms
    if both.any():
        tc = np.array(out["cold"]["seconds_to_target"])[both]
        tw = np.array(out["warm"]["seconds_to_target"])[both]
        cold_solo = float(c[both].sum() * solo_ms / 1e3)
        out.update({
            "median_step_ratio_cold_over_warm": float(np.median(c[both] / w[both])),
            "total_step_ratio_cold_over_warm": float(c[both].sum() / w[both].sum()),
            "cold_batch_seconds": float(tc.max()), "warm_batch_seconds": float(tw.max()),
            "cold_one_launch_per_problem_seconds_extrapolated": cold_solo,
            "speedup_warm_batch_vs_cold_batch": float(tc.max() / tw.max()),
            "speedup_warm_batch_vs_cold_one_launch_per_problem": float(cold_solo / (tw.max() + predict_s)),
        })
    return out


def resample(field, S):
    """Bilinear resampling of planes [..][R][R] on the nodes i/(R-1) of the
    unit square onto the nodes i/(S-1) of an S x S grid (the network's
    fixed-resolution prediction moved to a cavity's own grid)."""
    R = field.shape[-1]
    t = np.arange(S) * ((R - 1.0) / (S - 1.0))
    i0 = np.minimum(np.floor(t).astype(np.int64), R - 2)
    w = t - i0
    rows = field[..., i0, :] * (1.0 - w)[:, None] + field[..., i0 + 1, :] * w[:, None]
    return rows[..., i0] * (1.0 - w) + rows[..., i0 + 1] * w


def sweep_subset(per_side=4, re_max=1000.0, count=512, seed=2306):
    """Indices of a stratified subset of the seeded cavity sweep
    (workloads.cavity_batch_draws(count, seed)): the first `per_side`
    cavities of each grid side (65, 129, 257, 513) whose Re is at most
    re_max (the range the network is trained on)."""
    re, nn, sides = W.cavity_batch_draws(count, seed)
    out = []
    for side in (65, 129, 257, 513):
        idx = [i for i in range(count) if sides[i] == side and re[i] <= re_max][:per_side]
        out += idx
    return np.array(out), re, nn, sides


def steady_sweep_subset(per_side=4, pool=10, re_max=1000.0, target=1e-6, check_every=1000, max_steps=400_000,
                        stream=None):
    """The first `per_side` cavities of each side among the first `pool`
    ones with Re <= re_max (sweep_subset) whose flow settles: marched from
    rest as one batch, their windowed residual reaches `target` within
    max_steps (many power-law cavities of the larger grids keep a slowly
    oscillating flow above it, for which a time to residual does not
    exist).  Returns the selected indices and, per side, how many of the
    pool settled."""
    idx, re, nn, sides = sweep_subset(pool, re_max)
    b = mdf.Batch([cavity_problem(int(sides[i]), re[i], nn[i]) for i in idx], stream=stream)
    conv, r, st, steps, _ = march(b, target, check_every, max_steps, log=None, retire=True)
    b.close()
    sel, settled = [], {}
    for side in (65, 129, 257, 513):
        ok = [int(i) for k, i in enumerate(idx) if sides[i] == side and conv[k] >= 0]
        settled[str(side)] = len(ok)
        sel += ok[:per_side]
    return np.array(sel), settled


def march_alone(kw, target, check_every=1000, max_steps=2_000_000, init=None, stream=None):
    """One cavity marched by itself (the single-problem solver, one launch
    per step with its autotuned plan) until its windowed residual is <=
    target: (steps, wall seconds, final residual)."""
    import time

    import torch
    kw = dict(kw)
    nx, ny = kw.pop("nx"), kw.pop("ny")
    s = mdf.Solver(nx, ny, stream=stream, **kw)
    if init is not None:
        s.init(*init)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, r = 0, float("inf")
    while steps < max_steps:
        s.step(check_every)
        steps += check_every
        try:
            r, _ = s.residual()
        except mdf.MdfError:
            r = float("nan")
            break
        if r <= target:
            break
    s.synchronize()
    sec = time.perf_counter() - t0
    s.close()
    return steps, sec, r


def warm_vs_cold_sweep(net, per_side=4, re_max=1000.0, target=1e-6, check_every=1000, max_steps=400_000,
                       one_launch_per_problem=True, indices=None, pool=10, stream=None, log=print):
    """Learned warm start + batching against cold starts on a stratified
    subset of the seeded 512-cavity sweep (steady_sweep_subset, or the
    given indices): the network's
    128 x 128 prediction of every cavity, resampled to its grid, starts one
    batch (warm + batch); the same cavities from rest form another (cold +
    batch); and, with one_launch_per_problem, each cavity is marched from
    rest by itself (cold, one launch per problem and step), all to residual
    `target`.  Every arm is measured (wall clock, including the residual
    checks; the warm arm includes the prediction and resampling).  Returns
    per-arm and per-side counts and times."""
    import time

    import torch
    re, nn, sides = W.cavity_batch_draws(512, 2306)
    settled = None
    if indices is None:
        idx, settled = steady_sweep_subset(per_side, pool, re_max, target, check_every, max_steps, stream)
    else:
        idx = np.asarray(indices, dtype=np.int64)
    probs = [cavity_problem(int(sides[i]), re[i], nn[i]) for i in idx]
    out = {"workload": "stratified subset of the seeded 512-cavity sweep (seed 2306): of the first %d cavities "
                       "of each side {65,129,257,513} with Re <= %g, the first %d whose flow reaches residual "
                       "%.0e from rest within %d steps" % (pool, re_max, per_side, target, max_steps),
           "indices": idx.tolist(), "sides": [int(sides[i]) for i in idx], "re": [float(re[i]) for i in idx],
           "n": [float(nn[i]) for i in idx], "target": target, "check_every": check_every, "max_steps": max_steps,
           "settled_of_pool_per_side": settled}
    for mode in ("cold", "warm"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = mdf.Batch(probs, stream=stream)
        if mode == "warm":
            y = predict(net, W.warm_start_inputs(re[idx], nn[idx], net.R))
            for k, i in enumerate(idx):
                f = resample(y[k].astype(np.float64), int(sides[i]))
                b.init(k, f[0] * U_LID, f[1] * U_LID, f[2] * U_LID ** 2)
        t_setup = time.perf_counter() - t0
        conv, r, st, steps, when = march(b, target, check_every, max_steps, log=None, retire=True)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        out[mode + "_batch"] = {"seconds": sec, "setup_seconds": t_setup, "batch_steps": steps,
                                "steps_to_target": conv.tolist(), "seconds_to_target": [float(v) for v in when],
                                "final_residual": [float(v) for v in r],
                                "reached": int((conv >= 0).sum()),
                                "diverged": int((st == mdf.MDF_E_DIVERGED).sum()),
                                "reached_per_side": {str(sd): int(sum(1 for k, i in enumerate(idx)
                                                                      if sides[i] == sd and conv[k] >= 0))
                                                     for sd in (65, 129, 257, 513)}}
        b.close()
        if log:
            log("%s + batch: %d of %d reached %.0e in %.1f s (%d batch steps)"
                % (mode, out[mode + "_batch"]["reached"], len(probs), target, sec, steps))
    # the cavities that reach the target from both starts; the batch arms'
    # time is when the last of them got there (the others still stepping
    # beside them), the one-launch-per-problem arm's the sum of their runs
    c = np.array(out["cold_batch"]["steps_to_target"])
    w = np.array(out["warm_batch"]["steps_to_target"])
    both = (c >= 0) & (w >= 0)
    if one_launch_per_problem:
        # each cavity of that set marched from rest by itself
        tot, per = 0.0, []
        for k, kw in enumerate(probs):
            if not both[k]:
                per.append(None)
                continue
            st_, sec, r = march_alone(kw, target, check_every, max_steps, stream=stream)
            tot += sec
            per.append({"steps": st_, "seconds": sec, "residual": r})
        out["cold_one_launch_per_problem"] = {"seconds": tot, "per_problem": per,
                                              "reached": int(sum(1 for p_ in per if p_ and p_["residual"] <= target))}
        if log:
            log("cold, one launch per problem: %.1f s" % tot)
    out["reached_both"] = int(both.sum())
    out["reached_both_per_side"] = {str(sd): int(sum(1 for k, i in enumerate(idx) if sides[i] == sd and both[k]))
                                    for sd in (65, 129, 257, 513)}
    if both.any():
        tc = float(np.max(np.array(out["cold_batch"]["seconds_to_target"])[both]) + out["cold_batch"]["setup_seconds"])
        tw = float(np.max(np.array(out["warm_batch"]["seconds_to_target"])[both]) + out["warm_batch"]["setup_seconds"])
        out.update({"cold_batch_seconds_to_all_reached": tc, "warm_batch_seconds_to_all_reached": tw,
                    "median_step_ratio_cold_over_warm": float(np.median(c[both] / w[both])),
                    "total_step_ratio_cold_over_warm": float(c[both].sum() / w[both].sum()),
                    "speedup_warm_batch_vs_cold_batch": tc / tw})
        if one_launch_per_problem:
            solo = out["cold_one_launch_per_problem"]["seconds"]
            out["cold_one_launch_per_problem_seconds_to_all_reached"] = solo
            out["speedup_warm_batch_vs_cold_one_launch_per_problem"] = solo / tw
    return out


def conv_flops_per_sample(net):
    """Algorithmic multiply-add FLOPs (x2) of one forward pass of one sample:
    every 3 x 3 convolution at its resolution with its real channel counts
    (the output layer's 3 channels, the input layer's 4)."""
    R = net.R
    res = [1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 2, 2, 1, 1, 1]  # resolution divisor of each layer
    return sum(2.0 * (R // d) ** 2 * 9 * ci * co for d, (co, ci) in zip(res, net.layer_shapes()))


def train_benchmark(R=128, batch=16, steps=50, warmup=5, seed=0, stream=None, conv_kernel="tcgen05"):
    """Device time of mdf_net_train_step on seeded random data (device
    buffers, no loss read-back): ms per step and achieved TFLOP/s of the
    convolutions (forward + input gradient + weight gradient = 3 x forward;
    the first layer's input gradient is skipped, counted anyway)."""
    import torch
    net = Net(R, batch, stream=stream)
    net.set_conv_kernel(conv_kernel)
    net.set_params(init_params(net, 2306))
    rng = np.random.default_rng(seed)
    re, nn = W.warm_start_draws(batch, seed)
    x = torch.from_numpy(W.warm_start_inputs(re, nn, R)).cuda()
    t = torch.from_numpy(rng.standard_normal((batch, 3, R, R)).astype(np.float32)).cuda()
    for _ in range(warmup):
        net.train_step(x, t, 1e-4, want_loss=False)
    st = torch.cuda.current_stream() if stream is None else stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        net.train_step(x, t, 1e-4, want_loss=False)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    flops = 3.0 * conv_flops_per_sample(net) * batch
    net.close()
    return {"R": R, "batch": batch, "steps": steps, "ms_per_step": ms, "tflops": flops / (ms / 1e3) / 1e12,
            "flops_per_step": flops, "conv_kernel": conv_kernel}


def layer_benchmark(R=128, batch=16, reps=3, seed=0, stream=None):
    """Device time of every convolution of one forward pass, per layer and
    for each kernel (tcgen05, mma.sync): the CUDA kernel events of
    torch.profiler (CUPTI) over `reps` warm forward passes, median per
    layer, with the algorithmic TFLOP/s of the layer's real channels."""
    import torch
    from torch.profiler import ProfilerActivity, profile
    net = Net(R, batch, stream=stream)
    net.set_params(init_params(net, 2306))
    re, nn = W.warm_start_draws(batch, seed)
    x = torch.from_numpy(W.warm_start_inputs(re, nn, R)).cuda()
    res = [1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 2, 2, 1, 1, 1]  # resolution divisor of each layer
    shapes = net.layer_shapes()
    out = {}
    for kind in ("tcgen05", "mma.sync"):
        net.set_conv_kernel(kind)
        for _ in range(5):
            net.forward(x)
        torch.cuda.synchronize()
        runs = []
        for _ in range(reps):
            with profile(activities=[ProfilerActivity.CUDA]) as prof:
                net.forward(x)
                torch.cuda.synchronize()
            ev = sorted((e for e in prof.events()
                         if e.device_type == torch.autograd.DeviceType.CUDA and "conv" in e.name),
                        key=lambda e: e.time_range.start)
            if len(ev) == len(shapes):
                runs.append([e.time_range.elapsed_us() for e in ev])
        if not runs:
            out[kind] = None
            continue
        us = np.median(np.array(runs), axis=0)
        layers = []
        for (co, ci), d, t in zip(shapes, res, us):
            f = 2.0 * batch * (R // d) ** 2 * 9 * ci * co
            layers.append({"cout": co, "cin": ci, "side": R // d, "us": float(t), "tflops": f / t / 1e6})
        tot_us = float(us.sum())
        flops = sum(2.0 * batch * (R // d) ** 2 * 9 * ci * co for (co, ci), d in zip(shapes, res))
        out[kind] = {"layers": layers, "forward_us": tot_us, "forward_tflops": flops / tot_us / 1e6}
    net.close()
    return {"R": R, "batch": batch, "reps": reps, "kernels": out}


def channel_stats(t):
    q = [0.0, 0.01, 0.5, 0.99, 1.0]
    return {name: np.quantile(t[:, c], q).tolist() for c, name in enumerate(("u", "v", "p"))}


def main(argv=None):
    """Generate the data, train, evaluate and compare warm and cold starts;
    writes the parameters (.npy) and a JSON report."""
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--R", type=int, default=128)
    ap.add_argument("--count", type=int, default=5400, help="cavities drawn (seed 1); those at the target are kept")
    ap.add_argument("--trapezoid-fraction", type=float, default=0.3)
    ap.add_argument("--holdout-fraction", type=float, default=0.1)
    ap.add_argument("--data-target", type=float, default=1e-6)
    ap.add_argument("--data-max-steps", type=int, default=200_000)
    ap.add_argument("--epochs", type=int, default=120)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--sweep-per-side", type=int, default=4,
                    help="cavities per grid side of the sweep subset marched to 1e-8 cold and warm (0: skip)")
    ap.add_argument("--sweep-target", type=float, default=1e-6)
    ap.add_argument("--sweep-max-steps", type=int, default=400_000)
    ap.add_argument("--out")
    ap.add_argument("--report")
    ap.add_argument("--train-bench", action="store_true",
                    help="only time mdf_net_train_step on random data (--R, --batch, --epochs = timed steps)")
    ap.add_argument("--layer-bench", action="store_true",
                    help="only time every convolution of one forward pass, per layer and kernel (--R, --batch)")
    args = ap.parse_args(argv)

    from . import build as B
    B.build()
    if args.layer_bench:
        print(json.dumps(layer_benchmark(args.R, args.batch)), flush=True)
        return 0
    if args.train_bench:
        for kind in ("tcgen05", "mma.sync"):
            print(json.dumps(train_benchmark(args.R, args.batch, steps=args.epochs, conv_kernel=kind)), flush=True)
        return 0
    if not args.out or not args.report:
        ap.error("--out and --report are required")
    rep = {"args": vars(args)}
    t0 = time.perf_counter()
    x, t, info = generate_dataset(args.count, 1, args.R, target=args.data_target, max_steps=args.data_max_steps,
                                  trapezoid_fraction=args.trapezoid_fraction)
    tr, ho = split_holdout(len(x), args.holdout_fraction, seed=3)
    geo = np.array(info["geometry"])
    rep["data"] = {k: v for k, v in info.items() if k not in ("re", "n", "geometry")}
    rep["data"].update({"seconds": time.perf_counter() - t0, "train": int(tr.size), "holdout": int(ho.size),
                        "train_stats": channel_stats(t[tr])})
    print("data", json.dumps(rep["data"]), flush=True)
    t1 = time.perf_counter()
    net, hist = train(x[tr], t[tr], args.epochs, batch=args.batch, lr=args.lr)
    rep["train"] = {"seconds": time.perf_counter() - t1, "loss_first": hist[0], "loss_last": hist[-1],
                    "steps": args.epochs * (tr.size // args.batch)}
    eu, ep = evaluate(net, x[ho], t[ho])
    eu0, _ = evaluate(net, x[tr[:ho.size]], t[tr[:ho.size]])
    rep["holdout"] = {"velocity_rel_l2_median": float(np.median(eu)), "velocity_rel_l2_max": float(eu.max()),
                      "pressure_rel_l2_median": float(np.median(ep)),
                      "train_velocity_rel_l2_median": float(np.median(eu0))}
    for g in ("square", "trapezoid"):
        m = geo[ho] == g
        if m.any():
            rep["holdout"]["velocity_rel_l2_median_" + g] = float(np.median(eu[m]))
    print("train", json.dumps(rep["train"]), "holdout", json.dumps(rep["holdout"]), flush=True)
    net.save(args.out)
    del x, t
    if args.sweep_per_side:
        rep["sweep"] = warm_vs_cold_sweep(net, per_side=args.sweep_per_side, target=args.sweep_target,
                                          max_steps=args.sweep_max_steps)
        print("sweep", json.dumps({k: v for k, v in rep["sweep"].items()
                                   if k not in ("cold_one_launch_per_problem",)}), flush=True)
    with open(args.report, "w") as f:
        json.dump(rep, f, indent=1)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())

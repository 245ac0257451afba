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
            assert inputs.is_contiguous() and tuple(inputs.shape[1:]) == (4, self.R, self.R)
            tp = ctypes.c_void_p(targets.data_ptr()) if targets is not None else None
            return B, ctypes.c_void_p(inputs.data_ptr()), tp, 1, (inputs, targets)
        x = np.ascontiguousarray(inputs, dtype=np.float32)
        assert x.shape[1:] == (4, self.R, self.R), x.shape
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

def cavity_problem(R, re, n_index, u0=U_LID):
    """Keyword arguments (for mdf.Solver / mdf.Batch) of a power-law
    lid-driven cavity on R x R nodes of the unit square: Re = u0^(2-n) L^n / K
    with L = 1, nu clamped to [nu_ref / 20, 20 nu_ref], nu_ref = K (u0/L)^(n-1)."""
    K = u0 ** (2.0 - n_index) / re
    nu_ref = K * u0 ** (n_index - 1.0)
    return dict(nx=R, ny=R, nu=nu_ref, walls=(True, True), u_wall=(0, 0, 0, u0),
                power_law=(K, float(n_index), nu_ref / 20.0, nu_ref * 20.0))


def march(batch, target, check_every=1000, max_steps=500_000, max_seconds=None, log=None, log_every=50,
          retire=False):
    """Step a batch until every problem's windowed residual (mdf_residual,
    window `check_every`) is <= target, diverged, max_steps or max_seconds
    of wall time.  With retire=True a problem leaves the batch
    (mdf_batch_set_active) once it meets the target or diverges, so the
    others no longer pay for it.  Returns (first step count at which each
    problem met the target, -1 if never; final residuals; statuses; steps
    taken; wall seconds at which each problem met the target, NaN if never)."""
    import time
    conv = np.full(batch.count, -1, dtype=np.int64)
    when = np.full(batch.count, np.nan)
    last_r = np.full(batch.count, np.nan)
    last_st = np.zeros(batch.count, dtype=np.int64)
    gone = np.zeros(batch.count, dtype=bool)
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
        newly = (r <= target) & (conv < 0) & (st == mdf.MDF_OK)
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
    p / u0^2 clipped to [-P_CLIP, P_CLIP] (the pressure of the two lid corners
    is singular; unclipped, its few nodes would dominate the mean-square
    loss)."""
    out = []
    for i in range(batch.count):
        f = batch.problem(i).fields(["u", "v", "P"])
        out.append(np.stack([f["u"] / u0, f["v"] / u0, np.clip(f["P"] / u0 ** 2, -P_CLIP, P_CLIP)]))
    return np.asarray(out, dtype=np.float32)


def generate_dataset(count, seed, R, target=1e-6, check_every=1000, max_steps=200_000, stream=None, log=print):
    """Steady power-law cavities (seeded (Re, n) draws) marched from rest by
    the batched solver until every problem's residual is <= target or
    max_steps (some power-law cavities settle into a small persistent
    oscillation and never reach a low target; they are kept with their final
    state).  Diverged problems are dropped.  Returns inputs [k][4][R][R],
    targets [k][3][R][R] and a summary."""
    re, nn = W.warm_start_draws(count, seed)
    batch = mdf.Batch([cavity_problem(R, a, b) for a, b in zip(re, nn)], stream=stream)
    conv, r, st, steps, _ = march(batch, target, check_every, max_steps, log=log, log_every=50)
    ok = st != mdf.MDF_E_DIVERGED
    t = steady_fields(batch)[ok]
    batch.close()
    x = W.warm_start_inputs(re[ok], nn[ok], R)
    info = {"count": count, "seed": seed, "R": R, "target": target, "kept": int(ok.sum()),
            "reached_target": int((conv >= 0).sum()), "diverged": int((~ok).sum()), "steps": steps,
            "median_steps_to_target": float(np.median(conv[conv >= 0])) if (conv >= 0).any() else None,
            "final_residual_quantiles": np.quantile(r[ok], [0.5, 0.9, 1.0]).tolist() if ok.any() else None,
            "re": re[ok].tolist(), "n": nn[ok].tolist()}
    log("dataset seed %d: kept %d of %d (%d at target) after %d steps"
        % (seed, info["kept"], count, info["reached_target"], steps))
    return x, t, info


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
                 stream=None, log=print):
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

    probs = [cavity_problem(R, a, b) for a, b in zip(re, nn)]
    t0 = time.perf_counter()
    y = predict(net, W.warm_start_inputs(re, nn, R))
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


def conv_flops_per_sample(net):
    """Algorithmic multiply-add FLOPs (x2) of one forward pass of one sample:
    every 3 x 3 convolution at its resolution with its real channel counts
    (the output layer's 3 channels, the input layer's 4)."""
    R = net.R
    res = [1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 2, 2, 1, 1, 1]  # resolution divisor of each layer
    return sum(2.0 * (R // d) ** 2 * 9 * ci * co for d, (co, ci) in zip(res, net.layer_shapes()))


def train_benchmark(R=128, batch=16, steps=50, warmup=5, seed=0, stream=None):
    """Device time of mdf_net_train_step on seeded random data (device
    buffers, no loss read-back): ms per step and achieved TFLOP/s of the
    convolutions (forward + input gradient + weight gradient = 3 x forward;
    the first layer's input gradient is skipped, counted anyway)."""
    import torch
    net = Net(R, batch, stream=stream)
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
            "flops_per_step": flops}


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
    ap.add_argument("--train", type=int, default=1024, help="training cavities (seed 1)")
    ap.add_argument("--holdout", type=int, default=64, help="held-out cavities (seed 2)")
    ap.add_argument("--data-target", type=float, default=1e-6)
    ap.add_argument("--data-max-steps", type=int, default=200_000)
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--compare", type=int, default=16, help="held-out cavities marched to 1e-8 cold and warm")
    ap.add_argument("--out")
    ap.add_argument("--report")
    ap.add_argument("--train-bench", action="store_true",
                    help="only time mdf_net_train_step on random data (--R, --batch, --epochs = timed steps)")
    args = ap.parse_args(argv)

    from . import build as B
    B.build()
    if args.train_bench:
        print(json.dumps(train_benchmark(args.R, args.batch, steps=args.epochs)), flush=True)
        return 0
    if not args.out or not args.report:
        ap.error("--out and --report are required")
    rep = {"args": vars(args)}
    t0 = time.perf_counter()
    x, t, info = generate_dataset(args.train, 1, args.R, target=args.data_target, max_steps=args.data_max_steps)
    xh, th, infoh = generate_dataset(args.holdout, 2, args.R, target=args.data_target, max_steps=args.data_max_steps)
    rep["data"] = {"train": {k: v for k, v in info.items() if k not in ("re", "n")},
                   "holdout": {k: v for k, v in infoh.items() if k not in ("re", "n")},
                   "seconds": time.perf_counter() - t0, "train_stats": channel_stats(t)}
    print("data", json.dumps(rep["data"]), flush=True)
    t1 = time.perf_counter()
    net, hist = train(x, t, args.epochs, batch=args.batch, lr=args.lr)
    rep["train"] = {"seconds": time.perf_counter() - t1, "loss_first": hist[0], "loss_last": hist[-1],
                    "steps": args.epochs * (len(x) // args.batch)}
    eu, ep = evaluate(net, xh, th)
    eu0, _ = evaluate(net, x[:len(xh)], t[:len(xh)])
    rep["holdout"] = {"velocity_rel_l2_median": float(np.median(eu)), "velocity_rel_l2_max": float(eu.max()),
                      "pressure_rel_l2_median": float(np.median(ep)),
                      "train_velocity_rel_l2_median": float(np.median(eu0))}
    print("train", json.dumps(rep["train"]), "holdout", json.dumps(rep["holdout"]), flush=True)
    net.save(args.out)
    k = min(args.compare, len(xh))
    for tgt in (1e-6, 1e-8):
        key = "warm_vs_cold_%.0e" % tgt
        rep[key] = warm_vs_cold(net, np.array(infoh["re"][:k]), np.array(infoh["n"][:k]), args.R, target=tgt)
        print(key, json.dumps({a: b for a, b in rep[key].items() if a not in ("cold", "warm")}), flush=True)
    with open(args.report, "w") as f:
        json.dump(rep, f, indent=1)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())

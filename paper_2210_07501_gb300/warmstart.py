"""Learned warm start of the channel solver.

1. Training data: steady fields of seeded sweep channels, produced by the batched LB solver
   (`LbmBatch`, residual <= tol or a step budget).
2. Training: the surrogate (`Cnn`, hand-written CUDA kernels) learns parameters + heating
   profile -> steady phi, T - T_ref, u/U, v/U (see `surrogate`), with Adam on the mean
   squared error; data stays on the GPU.
3. Evaluation on held-out channels: the LB solver started from the surrogate's prediction
   (warm) against the solver started from rest (cold, the plain method and the reference):
   steps and wall time to the tolerance, the surrogate's own error against the converged LB
   fields, and the difference between the warm- and cold-started converged fields.  The
   warm start takes the predicted temperature and interface (phi); variants start from the
   predicted temperature alone and from all four predicted fields, and the caller may add
   starts of its own (`extra_starts`), e.g. a reference solution, run the same way.
   The slowest part of the approach to steady state is the settling of the interface,
   which the predicted phi shortens; the temperature alone shortens only the thermal
   transient.
"""
from __future__ import annotations

import time

import numpy as np

from . import LbmBatch, Cnn
from . import surrogate as S

FIELDS = ("phi", "u", "v", "T")


def steady_batch(cases, tol, max_steps, precision="fp32", init=None, K=100, stream=None):
    """Run cases to steady state in one batch; optional per-case initial fields."""
    b = LbmBatch(cases, precision=precision, stream=stream)
    b.lbm_batch_set_check_interval(K)
    if init is not None:
        for c, f in enumerate(init):
            b.lbm_batch_init_fields(c, **f)
    b.lbm_batch_autotune(3)
    t0 = time.perf_counter()
    steps, conv = b.lbm_batch_run_to_steady(tol, max_steps)
    dt = time.perf_counter() - t0
    fields = [b.lbm_batch_fields(c) for c in range(len(cases))]
    b.close()
    return fields, np.array(steps), np.array(conv), dt


def dataset(cases, fields):
    X = np.stack([S.features(c["domain"], c["params"]) for c in cases])
    Y = np.stack([S.targets(c["domain"], c["params"], f) for c, f in zip(cases, fields)])
    return X, Y


def target_scale(Y):
    """Per-channel standard deviation of the training targets: the network learns Y / scale,
    so that every output channel weighs equally in the mean squared error."""
    return np.maximum(Y.std(axis=(0, 2, 3)), 1e-12).astype(np.float32)


def train(net: Cnn, X, Y, iters=2000, batch=16, lr=1e-3, seed=0, log_every=0):
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.tensor(Y, device="cuda")
    n = X.shape[0]
    losses = []
    for it in range(iters):
        idx = torch.tensor(rng.choice(n, size=min(batch, n), replace=False), device="cuda")
        xb = Xd.index_select(0, idx).contiguous()
        yb = Yd.index_select(0, idx).contiguous()
        step_lr = lr * (0.1 ** (it / max(iters, 1)))          # exponential decay to lr / 10
        losses.append(net.train_step(xb, yb, step_lr))
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {losses[-1]:.4e}", flush=True)
    return losses


def predict(net: Cnn, X, scale, batch=16):
    """Predictions in target units (the network's output times the per-channel scale)."""
    import torch
    out = []
    for i in range(0, X.shape[0], batch):
        xb = torch.tensor(X[i:i + batch], device="cuda")
        yb = torch.empty((xb.shape[0], 4, X.shape[2], X.shape[3]), dtype=torch.float32, device="cuda")
        net.forward(xb, yb)
        out.append(yb.cpu().numpy())
    return np.concatenate(out) * scale[None, :, None, None]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def plain_per_case(cases, tol, max_steps, precision="fp32", init=None, K=100, stream=None):
    """The plain solver: one handle per channel, one after another (wall time, steps)."""
    from . import Lbm
    t0 = time.perf_counter()
    steps = []
    for c, w in enumerate(cases):
        g = Lbm(w["domain"], w["params"], precision=precision, stream=stream)
        g.lbm_set_check_interval(K)
        if init is not None:
            g.lbm_init_fields(**init[c])
        g.lbm_autotune(2)
        _, n = g.lbm_run_to_steady(tol, max_steps)
        steps.append(n)
        g.close()
    return time.perf_counter() - t0, np.array(steps)


def experiment(train_cases, test_cases, tol=1e-5, max_steps=60000, iters=2000, batch=16, lr=1e-3, seed=0,
               precision="fp32", log_every=0, plain_cases=0, extra_starts=None, train_tol=None, train_max_steps=None,
               K=100, progress=None, variants=True):
    """Full pipeline; returns a dict of measurements.  Runs on one dedicated stream, shared
    by torch's tensor operations and the library's kernels.  The training channels run to
    train_tol / train_max_steps (default: tol / max_steps), the held-out ones to tol, with
    K steps between residual checks.  extra_starts: optional {name: [initial fields per
    test case]} run as further variants (variants=False: only those, not the surrogate's own
    variants).  progress: optional callable(name, dict) told the result of each phase as
    soon as it is done."""
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        return _experiment(train_cases, test_cases, tol, max_steps, iters, batch, lr, seed, precision, log_every,
                           stream, plain_cases, extra_starts, train_tol or tol, train_max_steps or max_steps, K,
                           progress or (lambda name, d: None), variants)


def _experiment(train_cases, test_cases, tol, max_steps, iters, batch, lr, seed, precision, log_every, stream,
                plain_cases, extra_starts, train_tol, train_max_steps, K, progress, with_variants):
    t0 = time.perf_counter()
    f_train, s_train, c_train, _ = steady_batch(train_cases, train_tol, train_max_steps, precision, K=K,
                                                stream=stream)
    t_data = time.perf_counter() - t0
    progress("training_data", {"seconds": t_data, "converged": int(c_train.sum()), "steps_mean": float(s_train.mean())})
    X, Y = dataset(train_cases, f_train)
    scale = target_scale(Y)
    H, W = X.shape[2], X.shape[3]
    net = Cnn(H, W, batch_max=batch, bf16=True, seed=seed, stream=stream)
    t0 = time.perf_counter()
    losses = train(net, X, Y / scale[None, :, None, None], iters=iters, batch=batch, lr=lr, seed=seed,
                   log_every=log_every)
    t_train = time.perf_counter() - t0
    progress("training", {"seconds": t_train, "loss_first": float(losses[0]), "loss_last": float(np.mean(losses[-20:]))})
    Xt = np.stack([S.features(c["domain"], c["params"]) for c in test_cases])
    t0 = time.perf_counter()
    P = predict(net, Xt, scale)
    t_pred = time.perf_counter() - t0
    init = [S.fields_from_prediction(c["domain"], c["params"], p, use_phi=True) for c, p in zip(test_cases, P)]
    f_cold, s_cold, c_cold, t_cold = steady_batch(test_cases, tol, max_steps, precision, K=K, stream=stream)
    progress("cold", {"seconds": t_cold, "converged": int(c_cold.sum()), "steps_mean": float(s_cold.mean())})
    f_warm, s_warm, c_warm, t_warm = steady_batch(test_cases, tol, max_steps, precision, init=init, K=K,
                                                  stream=stream)
    progress("warm", {"seconds": t_warm, "converged": int(c_warm.sum()), "steps_mean": float(s_warm.mean())})
    net.close()
    # variants: the surrogate's T alone; T, interface and velocity; the caller's starts
    variants = {}
    starts = [("surrogate_T", [S.fields_from_prediction(c["domain"], c["params"], p)
                               for c, p in zip(test_cases, P)]),
              ("surrogate_T_phi_u_v", [S.fields_from_prediction(c["domain"], c["params"], p, use_phi=True,
                                                                use_velocity=True) for c, p in zip(test_cases, P)])]
    if not with_variants:
        starts = []
    starts += list((extra_starts or {}).items())
    for name, ini in starts:
        fv, sv, cv, tv = steady_batch(test_cases, tol, max_steps, precision, init=ini, K=K, stream=stream)
        bv = np.flatnonzero(cv & c_cold)
        variants[name] = {"steps_mean": float(sv.mean()), "converged": int(cv.sum()), "seconds": tv,
                          "steps": sv.tolist(),
                          "steps_mean_on_cold_converged": float(sv[bv].mean()) if bv.size else None,
                          "cold_steps_mean_same_cases": float(s_cold[bv].mean()) if bv.size else None,
                          "fewer_steps_cases": int(np.sum(sv < s_cold)),
                          "final_vs_cold_rel_l2": {k: float(np.mean([rel_l2(fv[i][k], f_cold[i][k]) for i in bv]))
                                                   if bv.size else None for k in ("phi", "u", "v", "T")}}
        progress(name, {k: v for k, v in variants[name].items() if k != "steps"})
    # the surrogate's own error against the converged cold-start LB fields (the reference)
    pred_fields = [S.fields_from_prediction(c["domain"], c["params"], p, use_phi=True, use_velocity=True)
                   for c, p in zip(test_cases, P)]
    # (phi: of its departure from the flat profile; T: of T - T_ref)
    def _err(k, i, f, c):
        base = S.phi_flat(c["domain"]) if k == "phi" else (c["params"]["T_ref"] if k == "T" else 0.0)
        return rel_l2(i[k] - base, f[k] - base)
    sur_err = {k: float(np.mean([_err(k, i, f, c) for i, f, c in zip(pred_fields, f_cold, test_cases)]))
               for k in FIELDS}
    # warm vs cold converged fields, on the channels both runs brought to the tolerance
    both = np.flatnonzero(c_warm & c_cold)
    wc = {k: float(np.mean([rel_l2(f_warm[i][k], f_cold[i][k]) for i in both])) if both.size else None
          for k in ("phi", "u", "v", "T")}
    plain = None
    if plain_cases:
        n = min(plain_cases, len(test_cases))
        t_plain, s_plain = plain_per_case(test_cases[:n], tol, max_steps, precision, K=K, stream=stream)
        plain = {"cases": n, "seconds": t_plain, "steps_mean": float(s_plain.mean()),
                 "same_steps_as_cold_batch": bool(np.array_equal(s_plain, s_cold[:n]))}
    return {
        "plain_per_case_cold": plain,
        "train_cases": len(train_cases), "test_cases": len(test_cases), "grid": [int(H), int(W)],
        "tol": tol, "max_steps": max_steps, "precision": precision, "check_interval": K,
        "train_tol": train_tol, "train_max_steps": train_max_steps,
        "data_seconds": t_data, "train_converged": int(c_train.sum()),
        "train_iters": iters, "batch": batch, "train_seconds": t_train,
        "loss_first": float(losses[0]), "loss_last": float(np.mean(losses[-20:])),
        "predict_seconds": t_pred,
        "cold_steps_mean": float(s_cold.mean()), "warm_steps_mean": float(s_warm.mean()),
        "both_converged": int(both.size),
        "cold_steps_mean_converged": float(s_cold[both].mean()) if both.size else None,
        "warm_steps_mean_converged": float(s_warm[both].mean()) if both.size else None,
        "cold_steps": s_cold.tolist(), "warm_steps": s_warm.tolist(),
        "cold_converged": int(c_cold.sum()), "warm_converged": int(c_warm.sum()),
        "cold_seconds": t_cold, "warm_seconds": t_warm,
        "warm_fewer_steps_cases": int(np.sum(s_warm < s_cold)),
        "surrogate_rel_l2_vs_lb": sur_err,
        "variants": variants,
        "warm_vs_cold_final_rel_l2": wc,
    }

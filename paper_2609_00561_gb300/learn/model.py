"""Learned blocking: an MLP (features -> ABMC block-size class, log CPM
resolution) trained on the GPU with the library's own kernels
(iccg_mlp_forward / iccg_mlp_grad / iccg_mlp_adam).

The labels come from the label sweep (learn/sweep.py): for every generated
matrix, the FP64 GPU ICCG solve time to 1e-8 under ABMC with each block size
and under Leiden CPM with each resolution; the class label is the fastest
block size, the regression label the log of the fastest resolution.  The
exhaustive sweep is the model's yardstick (regret T(prediction) / T(best of the
sweep)) and its fallback (`choose` returns the swept optimum when a matrix
was swept).

    python -m paper_2609_00561_gb300.learn.model --sweep blocking_sweep.json
        [--add-features]   # compute the features of every record (host) and store them
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HIDDEN = 64
WREG = 0.5
BASE_BLOCK = 32        # the method without the model: fixed ABMC block size ...
BASE_GAMMA = 0.05      # ... and fixed CPM resolution


def load_sweep(path):
    with open(path) as f:
        return json.load(f)


def add_features(data):
    """Features of every record's matrix (regenerated from its spec) by the
    library's host extractor."""
    import gen
    from paper_2609_00561_gb300 import iccg
    for rec in data["records"]:
        a = gen.config5_matrix(rec["spec"])
        rec["features"] = iccg.features(a).tolist()
    return data


TIE = 0.01   # settings within 1% of the fastest count as tied (timing noise)


def labels(data):
    """(features [N, F], class [N], log gamma [N], ABMC times [N, S], CPM times [N, G]).
    The class is the smallest block size within TIE of the fastest ABMC
    setting; the regression target the log of the largest resolution within
    TIE of the fastest CPM setting (ties go to the simpler, smaller-block
    setting, so timing noise between equal blockings does not flip labels)."""
    bs, gs = data["meta"]["block_sizes"], data["meta"]["gammas"]
    X, yc, yr, ta, tc = [], [], [], [], []
    for rec in data["records"]:
        runs = rec["runs"]
        a = np.array([r["ms"] if r["status"] == 0 else math.inf for r in runs[:len(bs)]])
        c = np.array([r["ms"] if r["status"] == 0 else math.inf for r in runs[len(bs):]])
        X.append(rec["features"])
        yc.append(int(np.flatnonzero(a <= (1 + TIE) * a.min())[0]))
        yr.append(math.log(gs[int(np.flatnonzero(c <= (1 + TIE) * c.min())[-1])]))
        ta.append(a)
        tc.append(c)
    return (np.array(X, dtype=np.float64), np.array(yc, dtype=np.int32), np.array(yr, dtype=np.float64),
            np.array(ta), np.array(tc))


def best_constants(ta, tc):
    """The constant settings (block-size index, resolution index) with the
    lowest mean regret on the given records (chosen on the training set)."""
    ra = (ta / ta.min(axis=1, keepdims=True)).mean(axis=0)
    rc = (tc / tc.min(axis=1, keepdims=True)).mean(axis=0)
    return int(np.argmin(ra)), int(np.argmin(rc))


def evaluate_constant(ta, tc, ia, ic):
    """Regret of constant settings (indices into the swept block sizes and
    resolutions) on the given records."""
    best_a, best_c = ta.min(axis=1), tc.min(axis=1)
    t_a, t_c = ta[:, ia], tc[:, ic]
    return {"abmc_regret_mean": float(np.mean(t_a / best_a)), "abmc_within_5pct": float(np.mean(t_a <= 1.05 * best_a)),
            "cpm_regret_mean": float(np.mean(t_c / best_c)), "cpm_within_5pct": float(np.mean(t_c <= 1.05 * best_c)),
            "combined_regret_mean": float(np.mean(np.minimum(t_a, t_c) / np.minimum(best_a, best_c)))}


def split(n, seed=0, n_test=40):
    """Train / held-out indices: a seeded permutation, the last n_test held out."""
    perm = np.random.default_rng(seed).permutation(n)
    return np.sort(perm[:n - n_test]), np.sort(perm[n - n_test:])


class Model:
    """Standardisation + MLP parameters (FP32 on the device while training)."""

    def __init__(self, nf, ncls, hidden=HIDDEN, seed=0):
        from paper_2609_00561_gb300 import iccg
        self.nf, self.ncls, self.h = nf, ncls, hidden
        self.np = iccg.mlp_nparams(nf, hidden, ncls)
        rng = np.random.default_rng(seed)
        p = []
        for fan_in, fan_out in ((nf, hidden), (hidden, hidden), (hidden, ncls + 1)):
            p.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), fan_in * fan_out))
            p.append(np.zeros(fan_out))
        self.params = np.concatenate(p).astype(np.float32)
        self.mu = np.zeros(nf)
        self.sd = np.ones(nf)

    def standardise(self, X):
        return ((X - self.mu) / self.sd).astype(np.float32)

    def fit(self, X, yc, yr, epochs=3000, lr=3e-3, device="cuda"):
        """Full-batch Adam on the GPU; returns the loss history (every 100 epochs)."""
        import torch
        from paper_2609_00561_gb300 import iccg
        self.mu = X.mean(axis=0)
        self.sd = np.where(X.std(axis=0) > 1e-12, X.std(axis=0), 1.0)
        Xs = torch.tensor(self.standardise(X), device=device)
        ycd = torch.tensor(yc.astype(np.int32), device=device)
        yrd = torch.tensor(yr.astype(np.float32), device=device)
        P = torch.tensor(self.params, device=device)
        G = torch.zeros_like(P)
        M = torch.zeros_like(P)
        V = torch.zeros_like(P)
        B = Xs.shape[0]
        work = torch.zeros(B * (4 * self.h + 2 * (self.ncls + 1) + 1), dtype=torch.float32, device=device)
        loss = torch.zeros(1, dtype=torch.float32, device=device)
        stream = torch.cuda.current_stream().cuda_stream
        hist = []
        for ep in range(1, epochs + 1):
            iccg.mlp_grad(P, self.nf, self.h, self.ncls, Xs, ycd, yrd, WREG, G, loss, work, stream)
            iccg.mlp_adam(P, G, M, V, lr, 0.9, 0.999, 1e-8, ep, stream)
            if ep % 100 == 0 or ep == 1:
                hist.append(float(loss.item()))
        self.params = P.cpu().numpy()
        return hist

    def predict(self, X, device="cuda"):
        """(class index [N], log gamma [N]) from the device forward kernel."""
        import torch
        from paper_2609_00561_gb300 import iccg
        Xs = torch.tensor(self.standardise(np.atleast_2d(X)), device=device)
        P = torch.tensor(self.params, device=device)
        out = torch.zeros((Xs.shape[0], self.ncls + 1), dtype=torch.float32, device=device)
        iccg.mlp_forward(P, self.nf, self.h, self.ncls, Xs, out, None, torch.cuda.current_stream().cuda_stream)
        o = out.cpu().numpy().astype(np.float64)
        return o[:, :self.ncls].argmax(axis=1), o[:, self.ncls]

    def save(self, path):
        np.savez(path, params=self.params, mu=self.mu, sd=self.sd, shape=np.array([self.nf, self.h, self.ncls]))


class Ensemble:
    """Several Models (seeds) whose outputs are averaged; the CPM prediction
    is kept only when it lies farther than `margin` (log space) from the
    constant resolution `gamma_const`, else that constant is used."""

    def __init__(self, models, margin=0.0, gamma_const=1.0):
        self.models, self.margin, self.gamma_const = models, margin, gamma_const

    def predict(self, X):
        import torch
        from paper_2609_00561_gb300 import iccg
        outs = []
        for m in self.models:
            Xs = torch.tensor(m.standardise(np.atleast_2d(X)), device="cuda")
            P = torch.tensor(m.params, device="cuda")
            out = torch.zeros((Xs.shape[0], m.ncls + 1), dtype=torch.float32, device="cuda")
            iccg.mlp_forward(P, m.nf, m.h, m.ncls, Xs, out, None, torch.cuda.current_stream().cuda_stream)
            outs.append(out.cpu().numpy().astype(np.float64))
        o = np.mean(outs, axis=0)
        ncls = self.models[0].ncls
        lg = o[:, ncls]
        lc = math.log(self.gamma_const)
        lg = np.where(np.abs(lg - lc) > self.margin, lg, lc)
        return o[:, :ncls].argmax(axis=1), lg


def _regrets(cls, lg, ta, tc, gammas):
    lgs = np.log(np.array(gammas))
    gi = np.abs(lg[:, None] - lgs[None, :]).argmin(axis=1)
    r = np.arange(len(cls))
    t_a, t_c = ta[r, cls], tc[r, gi]
    best_a, best_c = ta.min(axis=1), tc.min(axis=1)
    return (float(np.mean(t_a / best_a)), float(np.mean(t_c / best_c)),
            float(np.mean(np.minimum(t_a, t_c) / np.minimum(best_a, best_c))))


EPOCHS = (100, 300, 1000)
MARGINS = (0.0, 0.35, 0.7, 1.0, 1.5, 100.0)


def fit_select(X, yc, yr, ta, tc, gammas, nseeds=5, folds=5, seed=0):
    """Model selection on the training records only: 5-fold cross-validation
    over the training length (EPOCHS, chosen by the combined regret) and the
    CPM margin (MARGINS, chosen by the CPM regret) of a seed ensemble; then
    the ensemble trained on all of them.  Returns (Ensemble, choice record)."""
    rng = np.random.default_rng(seed + 1)
    parts = np.array_split(rng.permutation(len(yc)), folds)
    ia, ic = best_constants(ta, tc)
    cv = {}
    for ep in EPOCHS:
        outs = []
        for k in range(folds):
            va = parts[k]
            tr = np.concatenate([parts[j] for j in range(folds) if j != k])
            ja, jc = best_constants(ta[tr], tc[tr])
            ms = []
            for sd in range(nseeds):
                m = Model(X.shape[1], ta.shape[1], seed=seed + sd)
                m.fit(X[tr], yc[tr], yr[tr], epochs=ep)
                ms.append(m)
            cls, lg = Ensemble(ms, 0.0, gammas[jc]).predict(X[va])
            outs.append((va, cls, lg, math.log(gammas[jc])))
        for mg in MARGINS:
            res = []
            for va, cls, lg, lc in outs:
                lg2 = np.where(np.abs(lg - lc) > mg, lg, lc)
                res.append(_regrets(cls, lg2, ta[va], tc[va], gammas))
            cv[(ep, mg)] = np.mean(res, axis=0)
    ep_best = min(EPOCHS, key=lambda e: cv[(e, 0.0)][2])
    mg_best = min(MARGINS, key=lambda g: cv[(ep_best, g)][1])
    ms = []
    for sd in range(nseeds):
        m = Model(X.shape[1], ta.shape[1], seed=seed + sd)
        m.fit(X, yc, yr, epochs=ep_best)
        ms.append(m)
    choice = {"epochs": ep_best, "margin": mg_best, "cv_regret": [float(v) for v in cv[(ep_best, mg_best)]],
              "constant_block_index": ia, "constant_gamma": gammas[ic], "seeds": nseeds}
    return Ensemble(ms, mg_best, gammas[ic]), choice


def evaluate(model, X, ta, tc, gammas, block_sizes):
    """Regret of the predictions against the sweep, and the gain over the
    method without the model (ABMC 32, CPM 0.05), on the given records."""
    cls, lg = model.predict(X)
    lgs = np.log(np.array(gammas))
    gi = np.abs(lg[:, None] - lgs[None, :]).argmin(axis=1)      # nearest swept resolution
    rows = np.arange(len(cls))
    t_abmc, t_cpm = ta[rows, cls], tc[rows, gi]
    best_a, best_c = ta.min(axis=1), tc.min(axis=1)
    base_a = ta[:, block_sizes.index(BASE_BLOCK)]
    base_c = tc[:, gammas.index(BASE_GAMMA)]
    # the combined choice: the faster of the two predicted blockings vs the
    # faster of the two fixed ones (both measured by the sweep's times)
    pred = np.minimum(t_abmc, t_cpm)
    best = np.minimum(best_a, best_c)
    base = np.minimum(base_a, base_c)
    return {
        "n": int(len(cls)),
        "abmc_regret_mean": float(np.mean(t_abmc / best_a)),
        "abmc_within_5pct": float(np.mean(t_abmc <= 1.05 * best_a)),
        "cpm_regret_mean": float(np.mean(t_cpm / best_c)),
        "cpm_within_5pct": float(np.mean(t_cpm <= 1.05 * best_c)),
        "abmc_gain_vs_fixed32": float(np.exp(np.mean(np.log(base_a / t_abmc)))),
        "cpm_gain_vs_fixed005": float(np.exp(np.mean(np.log(base_c / t_cpm)))),
        "combined_regret_mean": float(np.mean(pred / best)),
        "combined_gain_vs_fixed": float(np.exp(np.mean(np.log(base / pred)))),
    }


def choose(model, a, block_sizes, gammas, swept=None):
    """(ABMC block size, CPM resolution) for matrix a: the sweep's optimum when
    `swept` (a record of the label sweep for this matrix) is given, else the
    model's prediction from the library's features (the resolution snapped to
    the nearest swept value)."""
    if swept is not None:
        runs = swept["runs"]
        ta = [r["ms"] if r["status"] == 0 else math.inf for r in runs[:len(block_sizes)]]
        tc = [r["ms"] if r["status"] == 0 else math.inf for r in runs[len(block_sizes):]]
        return block_sizes[int(np.argmin(ta))], gammas[int(np.argmin(tc))]
    from paper_2609_00561_gb300 import iccg
    cls, lg = model.predict(iccg.features(a)[None, :])
    gi = int(np.abs(lg[0] - np.log(np.array(gammas))).argmin())
    return block_sizes[int(cls[0])], gammas[gi]


def evaluate_fixed(ta, tc, gammas, block_sizes):
    """Regret of the method without the model (ABMC 32, CPM 0.05)."""
    base_a = ta[:, block_sizes.index(BASE_BLOCK)]
    base_c = tc[:, gammas.index(BASE_GAMMA)]
    best_a, best_c = ta.min(axis=1), tc.min(axis=1)
    return {"abmc_regret_mean": float(np.mean(base_a / best_a)),
            "cpm_regret_mean": float(np.mean(base_c / best_c)),
            "combined_regret_mean": float(np.mean(np.minimum(base_a, base_c) / np.minimum(best_a, best_c)))}


def report(data, seed=0):
    """Select and train on the training split, evaluate on the held-out split:
    the model, the best constant settings chosen on the training labels, and
    the method without the model (fixed ABMC 32 / CPM 0.05)."""
    X, yc, yr, ta, tc = labels(data)
    tr, te = split(len(yc))
    g, b = data["meta"]["gammas"], data["meta"]["block_sizes"]
    ens, choice = fit_select(X[tr], yc[tr], yr[tr], ta[tr], tc[tr], g, seed=seed)
    ia, ic = best_constants(ta[tr], tc[tr])
    return ens, {"choice": choice, "train": evaluate(ens, X[tr], ta[tr], tc[tr], g, b),
                 "test": evaluate(ens, X[te], ta[te], tc[te], g, b),
                 "test_best_constant": dict(evaluate_constant(ta[te], tc[te], ia, ic), block_size=b[ia], gamma=g[ic]),
                 "test_fixed": evaluate_fixed(ta[te], tc[te], g, b),
                 "labels": {"block_size": {str(v): int(np.sum(yc == k)) for k, v in enumerate(b)},
                            "gamma": {str(v): int(np.sum(np.isclose(np.exp(yr), v))) for v in g}}}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--sweep", required=True)
    p.add_argument("--add-features", action="store_true")
    p.add_argument("--out", default=None)
    args = p.parse_args()
    data = load_sweep(args.sweep)
    if args.add_features:
        data = add_features(data)
        with open(args.sweep, "w") as f:
            json.dump(data, f)
        return
    ens, res = report(data)
    print(json.dumps(res, indent=1))
    if args.out:
        for k, m in enumerate(ens.models):
            m.save(f"{args.out}.{k}")


if __name__ == "__main__":
    main()

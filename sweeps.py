"""The paper's parameter and distribution studies (Sec. 5), rerun on one GB300
with this library's GPU path.

The paper measured the harmonic kernel G = Gamma_j / (z_j - z_i) in FP64 at
p = 17 (tolerance ~1e-6), theta = 1/2, leaf sizes from its level formula
Eq. (Nlevels).  Each study below keeps those settings unless it sweeps them:

  leaf       time vs N_d for several N (Fig. "Ndirect") and the optimal N_d for
             several p (Fig. "Ndirecttol")
  p          per-phase times and error vs p at N = 1e6, N_d = 45 (Fig. "pspeedup")
  breakeven  FMM vs the library's direct sum as N grows (Fig. "breakeven")
  adaptivity time vs N on the uniform, normal and layer sets (Fig. "adaptivity")
  sigma      time vs the spread of the normal and layer sets, relative to the
             uniform set (Fig. "nonuniform")

Every study prints one JSON line per measurement and a markdown table.
Inputs are the seeded synthetic sets of workloads.py.  Run, for example:
    python sweeps.py --study p --precision fp64 mixed
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402


def setup():
    import torch

    import paper_1205_4611_gb300 as G
    G.load()
    return torch, G


def measure(torch, G, src, q, opt, repeats=3):
    """Median wall time of build + evaluate (synchronised), and the last run's
    per-phase device times."""
    s = torch.from_numpy(src).cuda()
    qq = torch.from_numpy(q).cuda()
    phi = torch.empty((len(src), 2), dtype=torch.float64, device="cuda")
    times, phases = [], None
    for r in range(repeats + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tree = G.fmm_build_tree(s, None, opt)
        G.fmm_set_timing(tree, True)
        G.fmm_evaluate(tree, qq, phi)
        G.fmm_tree_sync(tree)
        dt = (time.perf_counter() - t0) * 1e3
        if r:
            times.append(dt)
            phases = G.fmm_get_timings(tree)
        levels = G.fmm_tree_info(tree)["levels"]
        tree.free()
    return statistics.median(times), phases, levels, phi


def options(G, p, nd, precision, kernel="harmonic", level_rule=1):
    return G.fmm_default_options(
        p=p, leaf_size=nd, level_rule=level_rule,
        precision=G.FMM_PREC_MIXED if precision == "mixed" else G.FMM_PREC_FP64,
        kernel=G.FMM_KERNEL_HARMONIC if kernel == "harmonic" else G.FMM_KERNEL_LOG)


def emit(rows, line):
    print(json.dumps(line), flush=True)
    rows.append(line)


def table(rows, cols):
    out = ["| " + " | ".join(cols) + " |", "|" + "---|" * len(cols)]
    for r in rows:
        out.append("| " + " | ".join(
            (f"{r[c]:.4g}" if isinstance(r[c], float) else str(r[c])) for c in cols) + " |")
    return "\n".join(out)


def study_leaf(torch, G, args):
    rows = []
    for prec in args.precision:
        for p in args.p_list or [9, 17, 25]:
            for n in args.n_list or [100_000, 1_000_000]:
                src, q, _ = W.problem("uniform", n, W.BASE_SEED + 600 + n)
                res = {}
                for nd in [15, 25, 35, 45, 60, 80, 110]:
                    ms, _, L, _ = measure(torch, G, src, q, options(G, p, nd, prec))
                    res[nd] = (ms, L)
                best = min(res, key=lambda k: res[k][0])
                for nd, (ms, L) in res.items():
                    emit(rows, {"study": "leaf", "precision": prec, "p": p, "N": n, "N_d": nd,
                                "levels": L, "ms": ms, "rel": ms / res[best][0],
                                "optimal": nd == best})
    print(table(rows, ["precision", "p", "N", "N_d", "levels", "ms", "rel", "optimal"]))
    return rows


def direct_harmonic_sample(torch, src, q, sample):
    """Reference values sum_{x_j != y} q_j / (x_j - y) at the sampled sources,
    by a plain complex128 sum (PyTorch on the GPU, 16 targets at a time)."""
    x = torch.from_numpy(src[:, 0] + 1j * src[:, 1]).cuda()
    qq = torch.from_numpy(q[:, 0] + 1j * q[:, 1]).cuda()
    out = []
    for k in range(0, len(sample), 16):
        y = x[torch.from_numpy(sample[k:k + 16]).cuda()]
        d = x[None, :] - y[:, None]
        terms = torch.where(d == 0, torch.zeros_like(d), qq[None, :] / d)
        out.append(terms.sum(dim=1))
    return torch.cat(out).cpu().numpy()


def normwise(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def study_p(torch, G, args, n=1_000_000, n_sample=128, reference=None):
    """Per-phase times and error vs p.  The error is normwise against a direct
    sum at n_sample seeded sources: `reference(src, q, sample)` (default: the
    complex128 sum of direct_harmonic_sample)."""
    rows = []
    src, q, _ = W.problem("uniform", n, W.BASE_SEED + 700)
    sample = np.random.default_rng(0).choice(n, n_sample, replace=False)
    ref = (reference or (lambda s_, q_, i_: direct_harmonic_sample(torch, s_, q_, i_)))(
        src, q, sample)
    for prec in args.precision:
        for p in args.p_list or [5, 9, 13, 17, 21, 25, 29, 33, 41, 49]:
            ms, ph, L, phi = measure(torch, G, src, q, options(G, p, 45, prec))
            got = phi.cpu().numpy()[sample]
            err = normwise(got[:, 0] + 1j * got[:, 1], ref)
            emit(rows, {"study": "p", "precision": prec, "p": p, "N": n, "N_d": 45, "levels": L,
                        "ms": ms, "p2p": ph["p2p"], "m2l": ph["m2l"], "p2m": ph["p2m"],
                        "m2m": ph["m2m"], "l2l": ph["l2l"], "l2p_m2p": ph["m2p_l2p"],
                        "tree": ph["tree"], "connect": ph["connect"], "error": err})
    print(table(rows, ["precision", "p", "ms", "p2p", "m2l", "p2m", "m2m", "l2l", "l2p_m2p",
                       "tree", "connect", "error"]))
    return rows


def study_breakeven(torch, G, args):
    rows = []
    for n in [500, 1000, 2000, 3500, 5000, 10_000, 20_000]:
        src, q, _ = W.problem("uniform", n, W.BASE_SEED + 800 + n)
        s = torch.from_numpy(src).cuda()
        qq = torch.from_numpy(q).cuda()
        phi = torch.empty((n, 2), dtype=torch.float64, device="cuda")
        times = []
        for r in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.fmm_direct_noalloc(s, qq, phi)
            torch.cuda.synchronize()
            if r:
                times.append((time.perf_counter() - t0) * 1e3)
        direct = statistics.median(times)
        for prec in args.precision:
            ms, _, L, _ = measure(torch, G, src, q, options(G, 17, 45, prec, kernel="log"))
            emit(rows, {"study": "breakeven", "precision": prec, "N": n, "levels": L,
                        "fmm_ms": ms, "direct_fp64_ms": direct, "fmm_faster": ms < direct})
    print(table(rows, ["precision", "N", "levels", "fmm_ms", "direct_fp64_ms", "fmm_faster"]))
    return rows


def study_adaptivity(torch, G, args):
    rows = []
    for prec in args.precision:
        for dist in ["uniform", "normal", "layer"]:
            for n in args.n_list or [100_000, 300_000, 1_000_000, 3_000_000, 10_000_000]:
                src, q, _ = W.problem(dist, n, W.BASE_SEED + 900 + n)
                ms, ph, L, _ = measure(torch, G, src, q, options(G, 17, 45, prec), repeats=2)
                emit(rows, {"study": "adaptivity", "precision": prec, "dist": dist, "N": n,
                            "levels": L, "ms": ms, "p2p": ph["p2p"], "m2l": ph["m2l"],
                            "particles_per_s": n / (ms * 1e-3)})
    print(table(rows, ["precision", "dist", "N", "levels", "ms", "p2p", "m2l", "particles_per_s"]))
    return rows


def study_sigma(torch, G, args):
    rows = []
    n = 1_000_000
    for prec in args.precision:
        src, q, _ = W.problem("uniform", n, W.BASE_SEED + 1000)
        base, phb, _, _ = measure(torch, G, src, q, options(G, 17, 45, prec))
        for dist in ["normal", "layer"]:
            for sigma in [0.3, 0.1, 0.03, 0.01, 0.003]:
                src, q, _ = W.problem(dist, n, W.BASE_SEED + 1000, sigma=sigma)
                ms, ph, L, _ = measure(torch, G, src, q, options(G, 17, 45, prec))
                emit(rows, {"study": "sigma", "precision": prec, "dist": dist, "sigma": sigma,
                            "N": n, "levels": L, "ms": ms, "rel_to_uniform": ms / base,
                            "p2p_rel": ph["p2p"] / phb["p2p"], "m2l_rel": ph["m2l"] / phb["m2l"]})
    print(table(rows, ["precision", "dist", "sigma", "levels", "ms", "rel_to_uniform", "p2p_rel",
                       "m2l_rel"]))
    return rows


STUDIES = {"leaf": study_leaf, "p": study_p, "breakeven": study_breakeven,
           "adaptivity": study_adaptivity, "sigma": study_sigma}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--study", nargs="+", default=list(STUDIES), choices=list(STUDIES))
    ap.add_argument("--precision", nargs="+", default=["mixed", "fp64"], choices=["mixed", "fp64"])
    ap.add_argument("--p-list", type=int, nargs="*", default=None)
    ap.add_argument("--n-list", type=int, nargs="*", default=None)
    args = ap.parse_args()
    torch, G = setup()
    for name in args.study:
        STUDIES[name](torch, G, args)
    return 0


if __name__ == "__main__":
    sys.exit(main())

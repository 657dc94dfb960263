"""Training and evaluation of the slice-count selector on the GPU.

This module only generates seeded synthetic GEMM instances and marshals arguments: the
features, the emulated products at every S, the reference products, the error measurements,
the perceptron's forward pass and its Adam steps all run in libozk's CUDA kernels.

Instance families (all seeded; numpy generates the operands on the host):
  * ``dense``   : entries U(-1, 1) 2^round(N(0, sigma)), sigma in {0, 0.5, 1, 2, 3, 4, 6};
  * ``scaled``  : dense entries with row scales of op(A) and column scales of op(B)
                  2^round(N(0, s)), s in {2, 8, 20} (exponent spread across rows / columns);
  * ``cancel``  : op(B) = N R + delta R2 with N a basis of op(A)'s null space, so that
                  ||AB|| / (||A|| ||B||) ~ delta, delta = 10^-U(0, 8);
  * ``kkr``     : the operands of block-LU updates of KKR matrices M = I - t G (bcc LIZ of
                  15..65 sites, contour energies): L columns M[0:p, p:q] times U rows
                  M[p:q, 0:p], and L columns times a 16 x 16 pivot inverse.
Labels: log10 of the relative Frobenius error of the S-slice product (S = 3..10, triangular
pairs) against the S = 12 product (95 bits per operand, so its own error stays below 1e-20
for these instances before its final rounding to binary64), floored at 1e-17.

Usage (GPU):  python -m paper_2603_29975_gb300.selector --out selector_weights.bin
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

SMIN, SMAX = 3, 10
SREF = 12
FLOOR = -17.0
KINDS = ("dense", "scaled", "cancel", "kkr")


def _loguniform_int(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def _dense(rng, m, n, sigma):
    e = np.rint(rng.normal(0, sigma, (m, n))) if sigma > 0 else np.zeros((m, n))
    re = rng.uniform(-1, 1, (m, n)) * np.exp2(e)
    e2 = np.rint(rng.normal(0, sigma, (m, n))) if sigma > 0 else np.zeros((m, n))
    im = rng.uniform(-1, 1, (m, n)) * np.exp2(e2)
    return re + 1j * im


class _KkrPool:
    """A few KKR matrices M = I - t G (bcc LIZ, contour energies) to draw update operands from."""

    def __init__(self, seed, sizes=(15, 27, 51, 65), energies=4):
        import synth
        E, _ = synth.contour(32)
        pick = np.linspace(0, 31, energies).astype(int)
        self.systems = []
        for i, L in enumerate(sizes):
            for j in pick:
                t, G, _ = synth.kkr_system(L, 16, complex(E[j]), seed=seed + 7 * i, atom=int(j))
                self.systems.append((i, synth.kkr_matrix(t, G)))

    def draw(self, rng):
        sid = int(rng.integers(len(self.systems)))
        group, M = self.systems[sid]
        n = M.shape[0]
        if rng.uniform() < 0.7:
            w = int(rng.choice([16, 32, 64]))
            q = int(rng.integers(16 + w, n + 1)) // 16 * 16
            p = max(16, q - w)
            return group, M[:p, p:q], M[p:q, :p]
        a = int(rng.integers(2, n // 16)) * 16
        D = np.linalg.inv(M[a:a + 16, a:a + 16])
        return group, M[:a, a:a + 16], D


def generate_instances(count, seed, kkr_sizes=(15, 27, 51, 65), energies=4):
    """(group, kind, A, B) with A = op(A), B = op(B) as numpy complex matrices.  `group`
    identifies the KKR system (instances of one system stay on one side of a split)."""
    rng = np.random.default_rng(seed)
    pool = _KkrPool(seed, kkr_sizes, energies)
    out = []
    for i in range(count):
        kind = KINDS[i % len(KINDS)]
        if kind == "kkr":
            g, A, B = pool.draw(rng)
            out.append((1000 + g, kind, A, B))
            continue
        m, n, k = _loguniform_int(rng, 16, 400), _loguniform_int(rng, 16, 400), _loguniform_int(rng, 16, 800)
        if kind == "dense":
            sigma = float(rng.choice([0, 0.5, 1, 2, 3, 4, 6]))
            A, B = _dense(rng, m, k, sigma), _dense(rng, k, n, sigma)
        elif kind == "scaled":
            s = float(rng.choice([2, 8, 20]))
            A = _dense(rng, m, k, 1.0) * np.exp2(np.rint(rng.normal(0, s, (m, 1))))
            B = _dense(rng, k, n, 1.0) * np.exp2(np.rint(rng.normal(0, s, (1, n))))
        else:
            m = min(m, 300)
            k = min(max(k, m + 8), 400)
            A = _dense(rng, m, k, 1.0)
            _, _, vh = np.linalg.svd(A)
            N = vh[m:].conj().T                                      # k x (k - m), A N = 0
            delta = 10.0 ** -rng.uniform(0, 8)
            B = N @ _dense(rng, k - m, n, 0.0) + delta * _dense(rng, k, n, 0.0)
        out.append((i, kind, A, B))
    return out


def contour_solves(atoms, energies, natoms=256):
    """(atom, LIZ sites, energy index) of single solves drawn from the batched contour workload
    (`natoms` atoms with LIZ sizes drawn from 27..169 sites, 32 contour points): the given
    atoms at the given contour points."""
    import synth
    Ls = [int(v) for v in synth.liz_sizes(natoms)]
    return [(a, Ls[a], z) for a in atoms for z in energies]


def log_contour(ozk, h, solves, nbs=(32, 64), capacity=200000, seconds=None):
    """Training rows logged from the GEMMs of block-LU solves of the contour workload.  Every
    (atom, energy) M = I - t G (binary64 build on the GPU, G of the 169-site LIZ at that contour
    point, the atom's leading block) is solved by kkr_tau00 with S = 0 and panel widths cycling
    through `nbs` while the handle's selector log is on: each of the solve's GEMMs (the panels'
    L = M_RJ D^-1 and trailing updates M_RR -= L M_JR) adds its features and its log10 errors at
    S = 3..10.  Returns X (N x 16), T (N x 8) and the atom of every row (the split key)."""
    import torch
    import synth
    b = 16
    E, _ = synth.contour(32)
    zs = sorted({z for _, _, z in solves})
    Gs = dict(zip(zs, synth.kkr_contour_G(169, b, [complex(E[z]) for z in zs])))
    F = torch.zeros((capacity, 16), dtype=torch.float32, device="cuda")
    T = torch.zeros((capacity, 8), dtype=torch.float32, device="cuda")
    groups = []
    done = 0
    t_start = time.time()
    for i, (a, L, z) in enumerate(solves):
        if done >= capacity or (seconds is not None and time.time() - t_start > seconds):
            break
        n = L * b
        t = synth.kkr_t(L, b, atom=a)
        tb = torch.from_numpy(np.ascontiguousarray(np.transpose(t, (0, 2, 1)))).cuda()
        Gd = ozk.colmajor_cuda(Gs[z][:n, :n])
        M = torch.empty((n, n), dtype=torch.complex128, device="cuda").t()
        ozk.kkr_build_m(h, tb, Gd, M)
        tau = torch.zeros((b, b), dtype=torch.complex128, device="cuda").t()
        t0 = ozk.colmajor_cuda(t[0])
        h.selector_log_begin(F[done:], T[done:])
        ozk.kkr_tau00(h, M, t0, tau, S=0, nb=nbs[i % len(nbs)])
        rows = h.selector_log_end()
        groups += [a] * rows
        done += rows
    if h.status():
        raise RuntimeError("device status set while logging")
    return F[:done].cpu().numpy(), T[:done].cpu().numpy(), np.array(groups)


def solve_times(ozk, h, solves, S_list, nb=64, tol=1e-10):
    """Single solves of the contour workload at S = 0 (the selector per GEMM, with its check)
    and at each fixed S of S_list: summed milliseconds (CUDA events around every solve) and the
    largest relative error of tau_00 against the binary64 DMMA solve."""
    import torch
    import synth
    b = 16
    E, _ = synth.contour(32)
    zs = sorted({z for _, _, z in solves})
    Gs = dict(zip(zs, synth.kkr_contour_G(169, b, [complex(E[z]) for z in zs])))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    h.selector_configure(tol=tol)
    out = {str(S): {"ms_total": 0.0, "max_rel_err_vs_dmma": 0.0} for S in [0] + list(S_list)}
    for a, L, z in solves:
        n = L * b
        t = synth.kkr_t(L, b, atom=a)
        tb = torch.from_numpy(np.ascontiguousarray(np.transpose(t, (0, 2, 1)))).cuda()
        Gd = ozk.colmajor_cuda(Gs[z][:n, :n])
        M0 = torch.empty((n, n), dtype=torch.complex128, device="cuda").t()
        ozk.kkr_build_m(h, tb, Gd, M0)
        t0 = ozk.colmajor_cuda(t[0])

        def run(S, timed=True):
            M = M0.clone()
            tau = torch.zeros((b, b), dtype=torch.complex128, device="cuda").t()
            ev[0].record()
            ozk.kkr_tau00(h, M, t0, tau, S=S, nb=32 if S < 0 else nb)
            ev[1].record()
            torch.cuda.synchronize()
            return tau.cpu().numpy(), ev[0].elapsed_time(ev[1])

        ref, _ = run(-1)
        for S in [0] + list(S_list):
            run(S)                                                   # warm (workspace, scratch)
            tau, ms = run(S)
            e = float(np.linalg.norm(tau - ref) / np.linalg.norm(ref))
            out[str(S)]["ms_total"] += ms
            out[str(S)]["max_rel_err_vs_dmma"] = max(out[str(S)]["max_rel_err_vs_dmma"], e)
            if S == 0:
                info = h.selector_last()
                o = out["0"]
                o["redone_at_S10"] = o.get("redone_at_S10", 0) + int(info["fallback"])
                hist = o.setdefault("gemms_per_S", {})
                for k, v in info["S_count"].items():
                    hist[str(k)] = hist.get(str(k), 0) + v
    if h.status():
        raise RuntimeError("device status set in the timed solves")
    return out


def label(ozk, h, instances, with_times=True):
    """Features (N x 16), target log10 errors (N x 8) and per-S times in ms (N x 8)."""
    import torch
    N = len(instances)
    X = np.zeros((N, 16), dtype=np.float32)
    T = np.zeros((N, 8), dtype=np.float32)
    times = np.zeros((N, 8))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for i, (_, _, A, B) in enumerate(instances):
        Ad, Bd = ozk.colmajor_cuda(A), ozk.colmajor_cuda(B)
        m, n = A.shape[0], B.shape[1]
        X[i] = ozk.to_numpy(ozk.selector_features(h, Ad, Bd, seed=i))
        ref = torch.empty((n, m), dtype=torch.complex128, device="cuda").t()
        ozk.ozaki_zgemm(h, Ad, Bd, ref, S=SREF)
        C = torch.empty((n, m), dtype=torch.complex128, device="cuda").t()
        for o, S in enumerate(range(SMIN, SMAX + 1)):
            if with_times:
                ozk.ozaki_zgemm(h, Ad, Bd, C, S=S)                    # warm (workspace, caches)
                ev[0].record()
            ozk.ozaki_zgemm(h, Ad, Bd, C, S=S)
            if with_times:
                ev[1].record()
            err = ozk.rel_diff(h, C, ref)
            if with_times:
                times[i, o] = ev[0].elapsed_time(ev[1])
            T[i, o] = max(math.log10(err), FLOOR) if err > 0 else FLOOR
    if h.status():
        raise RuntimeError("device status set while labelling")
    return X, T, times


def split(instances, frac=0.8, seed=0):
    """Train / test indices, split by group (a KKR system, or a single random instance)."""
    groups = sorted({g for g, *_ in instances})
    rng = np.random.default_rng(seed)
    rng.shuffle(groups)
    cut = set(groups[:int(round(frac * len(groups)))])
    tr = [i for i, (g, *_) in enumerate(instances) if g in cut]
    te = [i for i, (g, *_) in enumerate(instances) if g not in cut]
    return tr, te


def train(ozk, h, X, T, steps=3000, lr=2e-3, seed=1, log_every=500):
    import torch
    h.selector_init(seed)
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    hist = []
    for s in range(1, steps + 1):
        rate = lr * (0.5 * (1 + math.cos(math.pi * (s - 1) / steps)) * 0.9 + 0.1)     # cosine decay
        loss = ozk.selector_train_step(h, Xd, Td, rate, want_loss=(s % log_every == 0 or s == 1))
        if loss is not None:
            hist.append((s, loss))
    return hist


def choose(pred, tol, margin):
    lim = math.log10(tol) - margin
    for o in range(8):
        if pred[o] <= lim:
            return SMIN + o
    return SMAX


def evaluate(ozk, h, instances, X, T, times, tol=1e-10, margin=0.6, run_auto=True):
    """Selector quality on labelled instances: chosen S, violations before the residual check
    (label of the chosen S above tol) and after it (the S = 0 call's product against the
    reference), and time against fixed S."""
    import torch
    Y = ozk.to_numpy(ozk.selector_predict(h, torch.from_numpy(X).cuda()))
    lim = math.log10(tol)
    chosen = np.array([choose(y, tol, margin) for y in Y])
    viol_before = int(np.sum(T[np.arange(len(T)), chosen - SMIN] > lim))
    ok_fixed = [S for S in range(SMIN, SMAX + 1) if np.all(T[:, S - SMIN] <= lim)]
    best_fixed = min(ok_fixed) if ok_fixed else None
    out = {"instances": len(T), "tol": tol, "margin": margin, "mean_S_selected": float(chosen.mean()),
           "violations_before_check": viol_before, "best_fixed_S_meeting_tol": best_fixed,
           "mse_log10": float(np.mean((Y - T) ** 2)), "S_hist": {int(S): int(np.sum(chosen == S))
                                                                 for S in range(SMIN, SMAX + 1)}}
    if run_auto:
        h.selector_configure(tol=tol, margin=margin)
        viol_after, fallbacks, used, t_auto = 0, 0, [], 0.0
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for i, (_, _, A, B) in enumerate(instances):
            Ad, Bd = ozk.colmajor_cuda(A), ozk.colmajor_cuda(B)
            m, n = A.shape[0], B.shape[1]
            ref = torch.empty((n, m), dtype=torch.complex128, device="cuda").t()
            ozk.ozaki_zgemm(h, Ad, Bd, ref, S=SREF)
            C = torch.empty((n, m), dtype=torch.complex128, device="cuda").t()
            ozk.ozaki_zgemm(h, Ad, Bd, C, S=0)                       # warm
            t0 = time.perf_counter()
            ev[0].record()
            ozk.ozaki_zgemm(h, Ad, Bd, C, S=0)
            ev[1].record()
            torch.cuda.synchronize()
            t_auto += ev[0].elapsed_time(ev[1])
            info = h.selector_last()
            used.append(info["S_used"])
            fallbacks += int(info["fallback"])
            viol_after += int(ozk.rel_diff(h, C, ref) > tol)
        out.update({"violations_after_check": viol_after, "fallbacks": fallbacks,
                    "mean_S_used": float(np.mean(used)), "auto_ms_total": t_auto,
                    "fixed_S10_ms_total": float(times[:, SMAX - SMIN].sum())})
        if best_fixed is not None:
            out["fixed_best_ms_total"] = float(times[:, best_fixed - SMIN].sum())
        out["chosen_S_ms_total"] = float(times[np.arange(len(T)), chosen - SMIN].sum())
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--contour", action="store_true",
                    help="add rows logged from single solves of the 256-atom contour workload")
    ap.add_argument("--log-seconds", type=float, default=300.0)
    ap.add_argument("--count", type=int, default=2400)
    ap.add_argument("--seed", type=int, default=20260401)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--out", default=None)
    ap.add_argument("--report", default=None)
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import paper_2603_29975_gb300 as ozk
    from paper_2603_29975_gb300 import build
    build.build()
    h = ozk.Handle()
    t0 = time.time()
    inst = generate_instances(args.count, args.seed)
    t1 = time.time()
    X, T, times = label(ozk, h, inst)
    t2 = time.time()
    tr, te = split(inst, seed=args.seed)
    Xtr, Ttr = X[tr], T[tr]
    rep = {"generate_s": t1 - t0, "label_s": t2 - t1}
    if args.contour:
        # atoms a = 3 (mod 4) are held out; the others are logged at every 4th contour point in
        # a seeded order until the time budget ends
        rng = np.random.default_rng(args.seed)
        train_solves = contour_solves([a for a in range(256) if a % 4 != 3], range(0, 32, 4))
        rng.shuffle(train_solves)
        test_atoms = [a for a in range(256) if a % 4 == 3][::4]
        test_log = contour_solves(test_atoms, (2, 10, 18, 26))
        test_time = contour_solves(test_atoms, (6, 22))
        h.selector_load()                      # any parameters: the S = 0 solves only carry the log
        h.selector_configure(tol=args.tol)
        t2 = time.time()
        Xc, Tc, gc = log_contour(ozk, h, train_solves, seconds=args.log_seconds)
        t3 = time.time()
        Xct, Tct, gct = log_contour(ozk, h, test_log)
        rep.update({"contour_log_s": t3 - t2, "contour_train_rows": int(len(Xc)),
                    "contour_train_atoms": int(len(set(gc.tolist()))), "contour_test_rows": int(len(Xct)),
                    "contour_test_atoms": int(len(set(gct.tolist())))})
        Xtr, Ttr = np.concatenate([Xtr, Xc]), np.concatenate([Ttr, Tc])
        t2 = time.time()
    hist = train(ozk, h, Xtr, Ttr, steps=args.steps, lr=args.lr, seed=args.seed)
    t3 = time.time()
    rep.update({"train_rows": int(len(Xtr)), "train_s": t3 - t2, "train_loss": hist,
                "train": evaluate(ozk, h, [inst[i] for i in tr], X[tr], T[tr], times[tr], tol=args.tol, run_auto=False),
                "test": evaluate(ozk, h, [inst[i] for i in te], X[te], T[te], times[te], tol=args.tol)})
    if args.contour:
        rep["contour_test"] = evaluate(ozk, h, None, Xct, Tct, None, tol=args.tol, run_auto=False)
        h.selector_configure(tol=args.tol)
        rep["contour_test_solves"] = {"solves": len(test_time),
                                      "S": solve_times(ozk, h, test_time, (5, 6, 7, 10), tol=args.tol)}
    if args.out:
        h.selector_save(args.out)
    text = json.dumps(rep, indent=1)
    if args.report:
        with open(args.report, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()

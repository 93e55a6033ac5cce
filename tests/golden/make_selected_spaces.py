"""Write the heat-bath-selected variational spaces and their oracle energies.

This script calls only the CPU oracle (``oracle/``) and the seeded integral
generator (``shci_synth``); nothing it stores comes from the CUDA library.

Selection (Sec. II.A, Eq. 2), as the workloads specify it: V starts as the
aufbau determinant; each iteration adds every determinant D_a outside V with
some D_i in V such that |H_ai| * |c_i| >= eps1 (|c_i| the largest |coefficient|
of D_i over the roots; ``oracle.System.select``, brute force over every single
and double excitation), then re-solves for the lowest roots (``oracle``
Davidson on the upper-triangle rows, started from the previous roots), and
lowers eps1 by the factor 0.7, starting from 1e-2.  The first iteration that
would take |V| to the target or beyond keeps only the target's worth of its new
determinants: those with the largest max_i |H_ai c_i|, ties by ascending
(alpha words, beta words).  V is stored in generation order: the aufbau
determinant, then each iteration's new determinants in the order the selection
returns them (ascending as integers whose most significant word is the last
stored word).

Storage (``<name>.npz``): per iteration block, the determinants' colex ranks
rank(beta) * C(n_orb, n_alpha) + rank(alpha) -- increasing within a block,
because colex rank orders bitstrings like their integer values -- as the first
rank and the gaps to the next, byte-planed and deflated.  ``<name>.json``
records the SHA-256 of the decoded [n_det, 2] uint64 array, the schedule, and,
after ``--energies``, the oracle's lowest roots of H on the full V (Davidson on
the upper-triangle rows to tol 1e-12, residual 1e-8) and the connected pair
count.

    python tests/golden/make_selected_spaces.py [--only NAME] [--energies] [--check-lanczos]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import shci_synth as S  # noqa: E402

SPACES = {
    # workload name: (target |V|, roots used by the selection)
    "sel_24o_6a6b_1m": (1_000_000, 2),
    "sel_20o_5a5b_1m": (1_000_000, 1),
}
EPS1_START = 1e-2
EPS1_FACTOR = 0.7
SELECT_TOL = 1e-9


def selected_space(name, log=print):
    cfg = S.config(name)
    target, roots = SPACES[name]
    h, eri, ec = S.integrals(cfg.n_orb, cfg.rank, cfg.seed, cfg.band, cfg.n_alpha)
    O = oracle.System(h, eri, ec)
    V = S.hf_dets(cfg.n_orb, cfg.n_alpha, cfg.n_beta)
    blocks = [1]
    schedule = []
    c = np.ones((1, 1))
    eps1 = EPS1_START
    while V.shape[0] < target:
        t = time.time()
        new, best = O.select(V, c, eps1, with_best=True)
        t_sel = time.time() - t
        last = V.shape[0] + new.shape[0] >= target
        if last:
            keep = target - V.shape[0]
            key = [new[:, w] for w in range(new.shape[1] - 1, -1, -1)] + [-best]
            order = np.lexsort(key)                      # largest product first, then (alpha, beta) words
            chosen = np.sort(order[:keep])               # back to the selection's order
            new = new[chosen]
        if new.shape[0]:
            V = np.concatenate([V, new])
            blocks.append(int(new.shape[0]))
        step = {"eps1": eps1, "new": int(new.shape[0]), "n_det": int(V.shape[0]), "select_s": round(t_sel, 1)}
        if not last:
            k = min(roots, V.shape[0])
            guess = None
            if c.shape[0] == k:
                guess = np.zeros((k, V.shape[0]))
                guess[:, :c.shape[1]] = c
            t = time.time()
            e, c = O.lowest_eigenpairs(V, k, tol=SELECT_TOL, guess=guess)
            step.update({"energies": [float(x) for x in e], "davidson_s": round(time.time() - t, 1)})
        schedule.append(step)
        log(name, json.dumps(step))
        eps1 *= EPS1_FACTOR
    return cfg, V, blocks, schedule


# ------------------------------------------------------------------ storage

def _encode(ranks):
    first = np.uint64(ranks[0])
    gaps = np.diff(ranks).astype(np.uint64)
    width = 4 if gaps.size == 0 or int(gaps.max()) < 2 ** 32 else 8
    g = gaps.astype(np.uint32 if width == 4 else np.uint64)
    planes = np.ascontiguousarray(g.view(np.uint8).reshape(-1, width).T)
    return first, width, planes


def write_space(name, cfg, V, blocks, schedule):
    ranks = S.colex_det_ranks(V, cfg.n_orb, cfg.n_alpha, cfg.n_beta)
    arrays = {"blocks": np.array(blocks, np.int64),
              "shape": np.array([cfg.n_orb, cfg.n_alpha, cfg.n_beta], np.int64)}
    o = 0
    for b, m in enumerate(blocks):
        first, width, planes = _encode(ranks[o:o + m])
        arrays["first_%d" % b] = np.array([first], np.uint64)
        arrays["planes_%d" % b] = planes
        o += m
    path = os.path.join(HERE, name + ".npz")
    np.savez_compressed(path, **arrays)
    back = S.load_selected_space(name, check_hash=False)
    assert np.array_equal(back, V), "encoding round trip failed"
    meta = {"workload": name, "n_orb": cfg.n_orb, "n_alpha": cfg.n_alpha, "n_beta": cfg.n_beta,
            "n_det": int(V.shape[0]), "sha256": hashlib.sha256(np.ascontiguousarray(V).tobytes()).hexdigest(),
            "selection": {"eps1_start": EPS1_START, "eps1_factor": EPS1_FACTOR, "roots": SPACES[name][1],
                          "davidson_tol": SELECT_TOL, "blocks": blocks, "schedule": schedule},
            "command": "python tests/golden/make_selected_spaces.py --only %s" % name}
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(meta, f, indent=1)
    return meta


def add_energies(name, lanczos=False, log=print):
    meta_path = os.path.join(HERE, name + ".json")
    meta = json.load(open(meta_path))
    cfg = S.config(name)
    V = S.load_selected_space(name)
    h, eri, ec = S.integrals(cfg.n_orb, cfg.rank, cfg.seed, cfg.band, cfg.n_alpha)
    O = oracle.System(h, eri, ec)
    t = time.time()
    rowptr, col, val = O.upper_csr(V)
    t_csr = time.time() - t
    op = oracle.UpperMatrix(rowptr, col, val, O.hdiag(V))
    log(name, "upper pairs", op.nnz_upper, "in %.0f s" % t_csr)
    k = cfg.roots
    t = time.time()
    e, C = oracle.davidson(op.matvec, op.diag, k, tol=1e-12, res_tol=1e-8, max_iter=2000, max_sub=max(12 * k, 32))
    t_dav = time.time() - t
    res = [float(np.linalg.norm(op.matvec(C[a]) - e[a] * C[a])) for a in range(k)]
    log(name, "energies", e, "residuals", res, "in %.0f s" % t_dav)
    meta["oracle"] = {"energies": [float(x) for x in e], "residual_norms": res, "roots": k,
                      "nnz_upper": op.nnz_upper, "davidson_tol": 1e-12, "davidson_res_tol": 1e-8,
                      "davidson_s": round(t_dav, 1), "upper_csr_s": round(t_csr, 1), "threads": oracle.num_threads(),
                      "method": "oracle.davidson on oracle.System.upper_csr (brute force (a), Slater-Condon in "
                                "operator form), started from the unit vectors of the lowest diagonal entries",
                      "command": "python tests/golden/make_selected_spaces.py --only %s --energies" % name}
    if lanczos:
        import scipy.sparse.linalg as sla
        A = sla.LinearOperator((V.shape[0], V.shape[0]), matvec=op.matvec, dtype=np.float64)
        t = time.time()
        w = np.sort(sla.eigsh(A, k=k + 1, which="SA", tol=1e-12, return_eigenvectors=False))
        meta["oracle"]["lanczos"] = {"energies": [float(x) for x in w], "seconds": round(time.time() - t, 1),
                                     "method": "scipy ARPACK eigsh (which=SA, tol 1e-12) on the same matrix"}
        log(name, "lanczos", w)
    with open(meta_path, "w") as f:
        json.dump(meta, f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", action="append")
    ap.add_argument("--energies", action="store_true", help="only add the oracle energies of a written space")
    ap.add_argument("--check-lanczos", action="store_true", help="also run ARPACK Lanczos on the same matrix")
    args = ap.parse_args()
    names = args.only or list(SPACES)
    for name in names:
        if not args.energies:
            cfg, V, blocks, schedule = selected_space(name)
            write_space(name, cfg, V, blocks, schedule)
        add_energies(name, lanczos=args.check_lanczos)


if __name__ == "__main__":
    main()

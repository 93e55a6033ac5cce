"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

This module only *draws* inputs: molecular-like integrals, determinant spaces
and trial vectors.  It holds none of the method's arithmetic (no Slater-Condon
rules, no excitation signs, no matrix elements, no eigen-solver), so both the
oracle and the GPU path can consume its outputs without sharing any of the
computation they are compared on.

Layouts (the library's input contract):

* ``h``           float64 [n_orb, n_orb], symmetric, row-major.
* ``eri_packed``  float64 [n_pair*(n_pair+1)/2] with n_pair = n_orb*(n_orb+1)/2,
                  chemists' notation (pq|rs); pair index pq = p*(p+1)/2 + q for
                  p >= q and slot = PQ*(PQ+1)/2 + RS for PQ >= RS (8-fold symmetry).
* determinants    uint64 [n_det, 2*W], alpha words then beta words; spatial
                  orbital n of a spin string is bit (n & 63) of word (n >> 6)
                  (the bit-packed representation of Sec. V.A), W = ceil(n_orb/64).

The paper's molecular integrals (Cu, Cr2) are not available; the generators
below are stand-ins with the paper's shapes (orbital counts, electron counts,
space sizes).  Their recipe is fixed here so that every run is reproducible.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "n_words", "n_pair", "eri_len", "integrals", "strings_from_occ", "fci_dets",
    "selected_dets", "hf_dets", "random_vectors", "CONFIGS", "config", "make_system",
    "colex_det_ranks", "load_selected_space", "selected_space_meta", "SPACES_DIR",
]


# ---------------------------------------------------------------- sizes

def n_words(n_orb: int) -> int:
    """64-bit words per spin string."""
    return (n_orb + 63) // 64


def n_pair(n_orb: int) -> int:
    return n_orb * (n_orb + 1) // 2


def eri_len(n_orb: int) -> int:
    m = n_pair(n_orb)
    return m * (m + 1) // 2


# ---------------------------------------------------------------- integrals

def integrals(n_orb: int, rank: int, seed: int, band: int = 0, n_elec_spin: int = 0):
    """Synthetic real integrals (h, eri_packed, e_core).

    h_pp = linspace(-2, 1, n_orb); off-diagonal h_pq (p < q) ~ N(0, 0.05) drawn
    once and mirrored.  (pq|rs) = sum_{L < rank} B^L_pq B^L_rs with B^L symmetric,
    B^L_pq (p <= q) ~ N(0, 0.3 exp(-|p-q|/3)); this is positive semi-definite
    and has the 8-fold permutation symmetry of real orbitals.

    ``band`` > 0 replaces the ``band`` diagonal entries centred on the Fermi
    level (between orbital n_elec_spin-1 and n_elec_spin) by an evenly spaced
    window of width 0.1 around that level and re-sorts the diagonal: a
    near-degenerate band like that of a transition-metal dimer.
    """
    rng = np.random.default_rng(seed)
    diag = np.linspace(-2.0, 1.0, n_orb)
    if band:
        e_f = 0.5 * (diag[n_elec_spin - 1] + diag[n_elec_spin])
        lo = n_elec_spin - band // 2
        diag[lo:lo + band] = np.linspace(e_f - 0.05, e_f + 0.05, band)
        diag = np.sort(diag)
    h = np.zeros((n_orb, n_orb))
    iu = np.triu_indices(n_orb, 1)
    h[iu] = rng.normal(0.0, 0.05, size=len(iu[0]))
    h = h + h.T
    h[np.diag_indices(n_orb)] = diag

    p_idx, q_idx = np.tril_indices(n_orb)          # p >= q, in packed pair order
    # packed pair order: pq = p(p+1)/2 + q  <=> row-major lower triangle
    std = 0.3 * np.exp(-np.abs(p_idx - q_idx) / 3.0)
    b = rng.normal(0.0, 1.0, size=(rank, len(p_idx))) * std[None, :]
    gram = b.T @ b                                  # (PQ, RS) = sum_L B_PQ B_RS
    pq, rs = np.tril_indices(len(p_idx))
    eri = np.ascontiguousarray(gram[pq, rs])
    return np.ascontiguousarray(h), eri, 0.0


# ---------------------------------------------------------------- strings

def strings_from_occ(occ: np.ndarray, n_orb: int) -> np.ndarray:
    """Pack occupation lists int[m, n_e] into uint64[m, W]."""
    occ = np.asarray(occ, dtype=np.int64)
    w = n_words(n_orb)
    out = np.zeros((occ.shape[0], w), dtype=np.uint64)
    for e in range(occ.shape[1]):
        o = occ[:, e]
        word = o >> 6
        bit = np.left_shift(np.uint64(1), (o & 63).astype(np.uint64))
        for k in range(w):
            out[:, k] |= np.where(word == k, bit, np.uint64(0))
    return out


def _all_strings(n_orb: int, n_e: int) -> np.ndarray:
    """All C(n_orb, n_e) strings, lexicographic in the occupation list."""
    if n_e == 0:
        return np.zeros((1, n_words(n_orb)), dtype=np.uint64)
    occ = np.array(list(itertools.combinations(range(n_orb), n_e)), dtype=np.int64)
    return strings_from_occ(occ, n_orb)


def fci_dets(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Full-CI space, alpha-string index major and beta-string index minor."""
    a = _all_strings(n_orb, n_alpha)
    b = _all_strings(n_orb, n_beta)
    w = n_words(n_orb)
    dets = np.empty((a.shape[0] * b.shape[0], 2 * w), dtype=np.uint64)
    dets[:, :w] = np.repeat(a, b.shape[0], axis=0)
    dets[:, w:] = np.tile(b, (a.shape[0], 1))
    return dets


def hf_dets(n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """Aufbau determinant (lowest orbitals by index; the diagonal of h is sorted)."""
    a = strings_from_occ(np.arange(n_alpha)[None, :], n_orb)
    b = strings_from_occ(np.arange(n_beta)[None, :], n_orb)
    return np.concatenate([a, b], axis=1)


# ---------------------------------------------------------------- selected spaces

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014), vectorised on uint64."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _string_table(n_orb, n_e, hole_window, particle_window, max_level):
    """Strings reachable from the aufbau string by moving up to ``max_level``
    electrons out of the top ``hole_window`` occupied orbitals into the lowest
    ``particle_window`` virtual orbitals.  Returns (occ int[m, n_e], level int[m])."""
    occ_hf = list(range(n_e))
    holes_from = occ_hf[max(0, n_e - hole_window):]
    parts_to = list(range(n_e, min(n_orb, n_e + particle_window)))
    rows, levels = [], []
    for lev in range(0, min(max_level, len(holes_from), len(parts_to)) + 1):
        for hs in itertools.combinations(holes_from, lev):
            keep = [o for o in occ_hf if o not in hs]
            for ps in itertools.combinations(parts_to, lev):
                rows.append(sorted(keep + list(ps)))
                levels.append(lev)
    return np.array(rows, dtype=np.int64).reshape(len(rows), n_e), np.array(levels)


def selected_dets(n_orb: int, n_alpha: int, n_beta: int, orb_energy: np.ndarray,
                  n_target: int, seed: int, tau: float | None = None,
                  hole_window: int | None = None, particle_window: int | None = None,
                  max_level: int | None = None) -> np.ndarray:
    """A seeded stand-in for a heat-bath-selected variational space.

    Each spin string s gets an excitation energy D(s) = sum_{p in s} e_p -
    sum_{p in aufbau} e_p from the orbital energies ``orb_energy`` (the sorted
    diagonal of h).  A determinant (a, b) gets the score D(a) + D(b) + t, where
    t = -tau * ln(u) is exponential noise whose uniform u comes from a
    SplitMix64 hash of (seed, a, b).  The ``n_target`` lowest-score determinants
    are kept and ordered by score (ties by alpha words then beta words), with the
    aufbau determinant first: like a selected space in generation order, it is
    dense near the reference, thins out with excitation energy, and has an
    irregular boundary.  No Hamiltonian matrix element enters the recipe.
    """
    e = np.asarray(orb_energy, dtype=np.float64)
    hole_window = n_orb if hole_window is None else hole_window
    particle_window = n_orb if particle_window is None else particle_window
    max_level = n_orb if max_level is None else max_level
    if tau is None:
        tau = 0.75 * float(np.mean(np.diff(e)))
    occ_a, lev_a = _string_table(n_orb, n_alpha, hole_window, particle_window, max_level)
    occ_b, lev_b = _string_table(n_orb, n_beta, hole_window, particle_window, max_level)
    da = e[occ_a].sum(1) - e[:n_alpha].sum()
    db = e[occ_b].sum(1) - e[:n_beta].sum()
    sa = strings_from_occ(occ_a, n_orb)
    sb = strings_from_occ(occ_b, n_orb)
    order_b = np.argsort(db, kind="stable")
    db_sorted = db[order_b]

    def count_below(t):
        return int(np.searchsorted(db_sorted, t - da, side="right").sum())

    total = len(da) * len(db)
    if n_target >= total:
        raise ValueError("n_target exceeds the candidate space")
    # bracket T0 such that the candidate pool comfortably exceeds n_target after noise
    lo, hi = 0.0, float(da.max() + db.max()) + 1.0
    want = min(total, max(int(2.5 * n_target), n_target + 1000))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if count_below(mid) >= want:
            hi = mid
        else:
            lo = mid
    t0 = hi
    while True:
        cnt = np.searchsorted(db_sorted, t0 - da, side="right")
        ia = np.repeat(np.arange(len(da)), cnt)
        starts = np.repeat(np.cumsum(cnt) - cnt, cnt)
        ib = order_b[np.arange(ia.size) - starts]
        wa = sa.shape[1]
        key = np.uint64((seed * 0x2545F4914F6CDD1D) & 0xFFFFFFFFFFFFFFFF)
        with np.errstate(over="ignore"):
            for k in range(wa):
                key = _splitmix64(key ^ sa[ia, k])
                key = _splitmix64(key ^ sb[ib, k])
        u = ((key >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
        score = da[ia] + db[ib] - tau * np.log(u)
        ok = score <= t0
        if ok.sum() >= n_target or cnt.sum() >= total:
            break
        t0 = t0 + 2.0 * tau
    ia, ib, score = ia[ok], ib[ok], score[ok]
    hf = (lev_a[ia] == 0) & (lev_b[ib] == 0)
    score = np.where(hf, -1.0, score)
    if ia.size > n_target:
        part = np.argpartition(score, n_target - 1)[:n_target]
        ia, ib, score = ia[part], ib[part], score[part]
    w = n_words(n_orb)
    dets = np.empty((ia.size, 2 * w), dtype=np.uint64)
    dets[:, :w] = sa[ia]
    dets[:, w:] = sb[ib]
    keys = [dets[:, c] for c in range(2 * w - 1, -1, -1)] + [score]
    order = np.lexsort(keys)
    return np.ascontiguousarray(dets[order])


# ---------------------------------------------------------------- stored selected spaces
# Heat-bath-selected spaces are written by tests/golden/make_selected_spaces.py
# (which runs the selection with the CPU oracle) and read back here by both the
# oracle's tests and the library's tests and benchmark.

SPACES_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def _sorted_strings(n_orb: int, n_e: int) -> np.ndarray:
    """Every one-word string of n_e electrons in n_orb orbitals, ascending as
    integers: position k holds the string of colex rank k."""
    if n_orb > 64:
        raise ValueError("stored spaces hold one-word strings (n_orb <= 64)")
    return np.sort(_all_strings(n_orb, n_e)[:, 0])


def colex_det_ranks(dets: np.ndarray, n_orb: int, n_alpha: int, n_beta: int) -> np.ndarray:
    """rank(beta) * C(n_orb, n_alpha) + rank(alpha) per determinant (colex
    ranks, which order strings like their integer values)."""
    ta, tb = _sorted_strings(n_orb, n_alpha), _sorted_strings(n_orb, n_beta)
    ra = np.searchsorted(ta, dets[:, 0])
    rb = np.searchsorted(tb, dets[:, 1])
    if not (np.array_equal(ta[ra], dets[:, 0]) and np.array_equal(tb[rb], dets[:, 1])):
        raise ValueError("determinant with a wrong electron count")
    return rb.astype(np.uint64) * np.uint64(ta.size) + ra.astype(np.uint64)


def selected_space_meta(name: str) -> dict:
    with open(os.path.join(SPACES_DIR, name + ".json")) as f:
        return json.load(f)


def load_selected_space(name: str, check_hash: bool = True, n_det: int | None = None) -> np.ndarray:
    """The stored heat-bath-selected space ``name`` as uint64 [n_det, 2] in
    generation order (its first n_det determinants if given: the space of an
    earlier selection stage plus part of the next block).  The decoded array's
    SHA-256 is checked against the one recorded beside it."""
    z = np.load(os.path.join(SPACES_DIR, name + ".npz"))
    n_orb, na, nb = (int(x) for x in z["shape"])
    ta, tb = _sorted_strings(n_orb, na), _sorted_strings(n_orb, nb)
    parts = []
    for b in range(z["blocks"].size):
        planes = z["planes_%d" % b]
        width = planes.shape[0]
        gaps = np.ascontiguousarray(planes.T).view(np.uint32 if width == 4 else np.uint64).ravel()
        first = z["first_%d" % b][0]
        ranks = np.concatenate([[first], first + np.cumsum(gaps.astype(np.uint64), dtype=np.uint64)])
        parts.append(ranks.astype(np.uint64))
    ranks = np.concatenate(parts)
    dets = np.empty((ranks.size, 2), np.uint64)
    dets[:, 0] = ta[(ranks % np.uint64(ta.size)).astype(np.int64)]
    dets[:, 1] = tb[(ranks // np.uint64(ta.size)).astype(np.int64)]
    if check_hash:
        want = selected_space_meta(name)["sha256"]
        got = hashlib.sha256(dets.tobytes()).hexdigest()
        if got != want:
            raise ValueError("stored space %s: SHA-256 %s, expected %s" % (name, got, want))
    return dets if n_det is None else np.ascontiguousarray(dets[:n_det])


def random_vectors(n: int, k: int, seed: int) -> np.ndarray:
    """float64 [k, n] with entries ~ N(0, 1)."""
    return np.random.default_rng(seed).normal(size=(k, n))


# ---------------------------------------------------------------- workloads

@dataclass(frozen=True)
class Config:
    name: str
    n_orb: int
    n_alpha: int
    n_beta: int
    rank: int
    seed: int
    n_det: int | None          # None: full-CI space
    roots: int
    band: int = 0
    window: tuple = field(default=(None, None, None))   # hole, particle, max level
    # "heat-bath": V is the stored heat-bath-selected space of this name
    # (tests/golden/<name>.npz, written by the oracle's selection); "score":
    # the seeded score-and-noise stand-in of selected_dets
    space: str = "score"
    stored_as: str | None = None           # name of the stored space (default: the config's name)


CONFIGS = {
    # full-CI space, 10 orbitals, 4a4b: C(10,4)^2 = 44,100 determinants
    "fci_10o_4a4b": Config("fci_10o_4a4b", 10, 4, 4, 20, 1001, None, 1),
    # heat-bath-selected space (Sec. II.A, Eq. 2), 24 orbitals, 6a6b, |V| = 1e6, two roots, stored H
    "sel_24o_6a6b_1m": Config("sel_24o_6a6b_1m", 24, 6, 6, 60, 1002, 1_000_000, 2, space="heat-bath"),
    # the same shape and integrals with the score-and-noise stand-in space
    "sel_24o_6a6b_1m_standin": Config("sel_24o_6a6b_1m_standin", 24, 6, 6, 60, 1002, 1_000_000, 2),
    # large shape like a transition-metal dimer: 76 orbitals, 14a14b, 12-orbital band
    "sel_76o_14a14b_50m": Config("sel_76o_14a14b_50m", 76, 14, 14, 300, 1003, 50_000_000, 1,
                                 band=12, window=(8, 16, 4)),
    # differentiation workload: heat-bath-selected space, 20 orbitals, 5a5b, |V| = 1e6
    "sel_20o_5a5b_1m": Config("sel_20o_5a5b_1m", 20, 5, 5, 40, 1004, 1_000_000, 1, space="heat-bath"),
    "sel_20o_5a5b_1m_standin": Config("sel_20o_5a5b_1m_standin", 20, 5, 5, 40, 1004, 1_000_000, 1),
}


def config(name: str) -> Config:
    return CONFIGS[name]


def batch_configs(n_sys: int = 64, seed: int = 5000, n_det_max: int = 2_000_000, n_det_min: int = 10_000,
                  roots: int = 4):
    """The batched workload: n_sys independent systems of uneven size.

    System s draws (from its own generator seeded seed + s) n_orb ~ U{12..30},
    electrons per spin ~ U{3..8} (capped at n_orb - 2, alpha and beta drawn
    separately) and |V| log-uniform in [n_det_min, n_det_max], capped at half
    the full-CI dimension; integrals use rank 2 * n_orb and seed seed + s."""
    out = []
    for s in range(n_sys):
        rng = np.random.default_rng(seed + s)
        n_orb = int(rng.integers(12, 31))
        na = int(min(rng.integers(3, 9), n_orb - 2))
        nb = int(min(rng.integers(3, 9), n_orb - 2))
        n_det = int(np.exp(rng.uniform(np.log(n_det_min), np.log(n_det_max))))
        fci = math.comb(n_orb, na) * math.comb(n_orb, nb)
        n_det = max(roots + 1, min(n_det, fci // 2))
        out.append(Config("batch_%02d" % s, n_orb, na, nb, 2 * n_orb, seed + s, n_det, roots))
    return out


def make_system(cfg: Config, n_det: int | None = None):
    """(h, eri_packed, e_core, dets) for a workload; ``n_det`` overrides the
    space size (a smaller space of the same shape for parity runs: for a
    stored heat-bath space, its first n_det determinants in generation order)."""
    h, eri, e_core = integrals(cfg.n_orb, cfg.rank, cfg.seed, cfg.band, cfg.n_alpha)
    n = cfg.n_det if n_det is None else n_det
    if n is None:
        dets = fci_dets(cfg.n_orb, cfg.n_alpha, cfg.n_beta)
    elif cfg.space == "heat-bath":
        name = cfg.stored_as or cfg.name
        meta = selected_space_meta(name)
        if n > meta["n_det"]:
            raise ValueError("%s holds %d determinants, %d asked" % (name, meta["n_det"], n))
        dets = load_selected_space(name, n_det=n)
    else:
        hw, pw, ml = cfg.window
        dets = selected_dets(cfg.n_orb, cfg.n_alpha, cfg.n_beta, np.diag(h), n, cfg.seed,
                             hole_window=hw, particle_window=pw, max_level=ml)
    return h, eri, e_core, dets

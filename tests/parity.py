"""Force-parity criterion shared by the GPU tests.

Per atom i, with F the GPU force and F_ref the FP64 oracle force:
  raw_i  = |F_i - F_ref,i| / |F_ref,i|
  norm_i = |F_i - F_ref,i| / cond_i,  cond_i = sum over partners j of the sizes of the
           three terms of Eq. 1-2, (|A| r^-14 + |B| r^-8 + |k q_i q_j| r^-3) * r
  rms    = sqrt(sum |dF|^2 / sum |F_ref|^2)
The pass criterion is max_i norm_i <= tol (tol = 1e-5 for FP32 pair math): the error
of a sum measured against the size of what is summed, which stays meaningful when
large pair terms cancel in F_i.

Pairs whose FP64 r^2 lies within a few float32 ulps of rc^2 ("boundary pairs") may be
kept by one side and dropped by the other, and both decisions are correct roundings of
the same filter.  For an atom touched by such pairs the test also accepts the oracle's
force with any subset of those pair terms toggled.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle

BOUNDARY_ULPS = 16


def boundary_window(rc: float) -> float:
    return BOUNDARY_ULPS * 2.0**-24 * rc * rc


def pair_term(pos, i, j, s, ff: oracle.ForceField):
    """Force on i from j as if inside the cutoff (the cutoff is lifted a little)."""
    A = ff.A[s.type[i], s.type[j]]
    B = ff.B[s.type[i], s.type[j]]
    F, _ = oracle.pair(pos[i], pos[j], s.box, float(s.q[i]), float(s.q[j]), A, B, ff.k,
                       ff.rc * (1 + 1e-5))
    return F


def boundary_alternatives(pos, s, ff, F_ref):
    """{atom: [alternative reference forces]} from toggling boundary pairs."""
    ij, r2 = oracle.boundary_pairs(pos, s.box, ff.rc, boundary_window(ff.rc))
    per_atom: dict[int, list] = {}
    for (i, j), rr in zip(ij, r2):
        Fij = pair_term(pos, i, j, s, ff)
        sign = -1.0 if rr < ff.rc * ff.rc else 1.0  # remove an included pair, add an excluded one
        per_atom.setdefault(int(i), []).append(sign * Fij)
        per_atom.setdefault(int(j), []).append(-sign * Fij)
    alts = {}
    for a, terms in per_atom.items():
        opts = []
        for k in range(1, len(terms) + 1):
            for sub in itertools.combinations(terms, k):
                opts.append(F_ref[a] + np.sum(sub, axis=0))
        alts[a] = opts
    return alts, int(ij.shape[0])


def force_errors(F, F_ref, cond, alts=None):
    dF = np.linalg.norm(F - F_ref, axis=1)
    if alts:
        for a, opts in alts.items():
            for alt in opts:
                dF[a] = min(dF[a], np.linalg.norm(F[a] - alt))
    nref = np.linalg.norm(F_ref, axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        raw = np.where(nref > 0, dF / nref, np.where(dF > 0, np.inf, 0.0))
        norm = np.where(cond > 0, dF / cond, np.where(dF > 0, np.inf, 0.0))
    rms = float(np.sqrt((dF**2).sum() / max((nref**2).sum(), 1e-300)))
    return dict(max_raw=float(raw.max(initial=0.0)), max_norm=float(norm.max(initial=0.0)),
                rms=rms, worst=int(np.argmax(norm)) if norm.size else -1)

"""Process-parallel driver of the FP64 oracle (independent centre atoms per worker).

TEST INFRASTRUCTURE (see oracle/__init__.py).

The energy of centre atom i depends only on the edges of i, so disjoint sets of centres
are evaluated in separate worker processes with `Allegro64.centre_terms`, and the forces
are assembled from the per-edge gradients afterwards.  Workers are started with the
"spawn" method (safe after a CUDA context exists in the parent) and run their BLAS on one
thread each.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_STATE = {}


def _init(hp, seed, pos, Z, box, pbc, sys_ptr):
    from .allegro64 import Allegro64
    _STATE.update(model=Allegro64(hp, seed), pos=pos, Z=Z, box=box, pbc=pbc,
                  sys_ptr=sys_ptr)


def _work(centres):
    s = _STATE
    return s["model"].centre_terms(s["pos"], s["Z"], s["box"], s["pbc"], list(centres),
                                   s["sys_ptr"])


def centre_terms(hp, seed, pos, Z, box, pbc, centres, sys_ptr=None, workers=None,
                 pieces_per_worker=4):
    """{i: (E_i, col, shift, g)} for the given centres, computed by `workers` processes."""
    workers = workers or os.cpu_count() or 1
    centres = np.asarray(sorted(set(int(c) for c in centres)), dtype=np.int64)
    if workers <= 1 or centres.shape[0] < 2 * workers:
        _init(hp, seed, pos, Z, box, pbc, sys_ptr)
        return _work(centres)
    chunks = [c for c in np.array_split(centres, workers * pieces_per_worker) if c.size]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                             "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_init,
                      initargs=(hp, seed, pos, Z, box, pbc, sys_ptr)) as pool:
            parts = pool.map(_work, chunks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out = {}
    for p in parts:
        out.update(p)
    return out


def evaluate(hp, seed, pos, Z, box, pbc, sys_ptr=None, workers=None):
    """(E_sys, E_atom, F) of a whole system, centres spread over worker processes."""
    n = np.asarray(pos).shape[0]
    if sys_ptr is None:
        sys_ptr = np.array([0, n])
    terms = centre_terms(hp, seed, pos, Z, box, pbc, range(n), sys_ptr, workers)
    E_atom = np.zeros(n)
    F = np.zeros((n, 3))
    for i, (Ei, col, _sh, g) in terms.items():
        E_atom[i] = Ei
        if g.shape[0]:
            F[i] += g.sum(axis=0)
            np.add.at(F, col, -g)
    E_sys = np.array([E_atom[sys_ptr[k]:sys_ptr[k + 1]].sum()
                      for k in range(len(sys_ptr) - 1)])
    return E_sys, E_atom, F


def sampled_forces(hp, seed, pos, Z, box, pbc, atoms, sys_ptr=None, workers=None):
    """Forces and per-atom energies on a sample of atoms (edges out of and into each)."""
    from . import neighbors
    nl = neighbors.neighbor_list(pos, box, pbc, hp["rc"], 0.0, sys_ptr, centres=atoms)
    need = set(int(a) for a in atoms)
    for m in atoms:
        need.update(int(j) for j in nl[int(m)][0])
    terms = centre_terms(hp, seed, pos, Z, box, pbc, sorted(need), sys_ptr, workers)
    F, Ei = {}, {}
    for m in atoms:
        m = int(m)
        Fm = terms[m][3].sum(axis=0) if terms[m][3].shape[0] else np.zeros(3)
        for i in sorted(set(int(j) for j in nl[m][0])):
            _, col, _, g = terms[i]
            hit = col == m
            Fm = Fm - g[hit].sum(axis=0)
        F[m] = Fm
        Ei[m] = terms[m][0]
    return F, Ei

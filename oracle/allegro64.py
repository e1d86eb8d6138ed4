"""FP64 CPU oracle of the Allegro-FM energy and forces (arXiv 2502.06073).

TEST INFRASTRUCTURE (see oracle/__init__.py): a plain, slow evaluator of the model
definition below, with forces from a hand-derived reverse-mode gradient.  It shares no
code with the CUDA path.

Paper statements used (Methodology, Model Training; Table 1): Allegro, strictly local
with a radial cutoff; l = 2 "in full O(3) symmetry"; a two-body latent MLP and a per-layer
latent MLP, "both employing SiLU"; the embedding is a linear projection; the edge-energy
MLP has no non-linearity; weights are unit-variance uniform; per-atom energies.
Everything the paper leaves open is fixed as a reading (each marked [R]):

  edge e = (i, j, s), r_e = x_j + s L - x_i, r = |r_e|, u_e = r_e / r
  [R] radial basis  B_n(r) = sqrt(2/rc) sin(n pi r / rc) / r,  n = 1..n_basis
  [R] envelope      f(x) = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1) - p(p+1)/2 x^(p+2),
                    x = r/rc, f = 0 for x >= 1
  two-body          x^0 = f * MLP_2b( onehot(Z_i) || onehot(Z_j) || B(r) )
  per layer L = 1..N
    [R] env weights w^L = x^(L-1) W_env^L / sqrt(D),            w[l, c]
    [R] environment G^L_i[c, l, m] = nu^(-1/2) sum_{k in N(i)} w^L_ik[l, c] Y_lm(u_ik)
    [R] V^0_ij[c, (l, (-1)^l), m] = w^1_ij[l, c] Y_lm(u_ij)
        tensor product per channel and path (l1 p1) x (l2) -> (l3 p3):
            T[c, m3] = sum_{m1 m2} C[m1, m2, m3] V^(L-1)_ij[c, l1 p1, m1] G^L_i[c, l2, m2]
        scalars s^L = the 0e outputs (one per 0e path and channel)
    [R] latent        x^L = ( x^(L-1) + f * MLP_lat^L( x^(L-1) || s^L ) ) / sqrt(2)
    [R] mixing        V^L[c, (l3 p3)] = sum_{paths -> l3p3} theta^L[path, c] T / sqrt(n_paths)
                      (layers L < N only)
  energy            E_ij = MLP_e(x^N) (linear layers only), E_i = sum_j E_ij, E = sum_i E_i
  [R] every linear layer is x W / sqrt(fan_in), no biases; SiLU after every linear layer
      of the two-body and latent MLPs.

Forces: F_m = -dE/dx_m = sum_{e = (m, j, s)} g_e - sum_{e = (i, m, s)} g_e with
g_e = dE/dr_e.  The energy of centre i depends only on the edges of i, so centres are
processed in independent chunks.
"""
from __future__ import annotations

import math

import numpy as np

from . import neighbors, so3
from .weights import N_SPECIES, init_params

SQRT2 = math.sqrt(2.0)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


def bessel(r, rc, n_basis):
    """B_n(r) and dB_n/dr, shapes [E, n_basis]."""
    n = np.arange(1, n_basis + 1, dtype=np.float64)
    a = n[None, :] * math.pi / rc
    pref = math.sqrt(2.0 / rc)
    rr = r[:, None]
    s = np.sin(a * rr)
    c = np.cos(a * rr)
    B = pref * s / rr
    dB = pref * (a * c * rr - s) / (rr * rr)
    return B, dB


def tp(cg, V, G):
    """T[e, c, k] = sum_{a, b} cg[a, b, k] V[e, c, a] G[e, c, b]."""
    a, b, k = cg.shape
    VG = V[:, :, :, None] * G[:, :, None, :]
    return (VG.reshape(-1, a * b) @ cg.reshape(a * b, k)).reshape(V.shape[0], V.shape[1], k)


def tp_adjoint(cg, gT, V, G):
    """Gradients of sum(gT * tp(cg, V, G)) with respect to V and to G."""
    a, b, k = cg.shape
    M = (gT.reshape(-1, k) @ cg.reshape(a * b, k).T).reshape(V.shape[0], V.shape[1], a, b)
    gV = (M * G[:, :, None, :]).sum(axis=3)
    gG = (M * V[:, :, :, None]).sum(axis=2)
    return gV, gG


def envelope(r, rc, p):
    """Polynomial cutoff f(r/rc) and df/dr (zero beyond rc)."""
    x = r / rc
    inside = x < 1.0
    f = (1.0 - 0.5 * (p + 1) * (p + 2) * x ** p + p * (p + 2) * x ** (p + 1)
         - 0.5 * p * (p + 1) * x ** (p + 2))
    df = -0.5 * p * (p + 1) * (p + 2) * x ** (p - 1) * (1.0 - x) ** 2 / rc
    return np.where(inside, f, 0.0), np.where(inside, df, 0.0)


class Allegro64:
    """The potential with one fixed set of weights, evaluated in float64."""

    def __init__(self, hp: dict, seed: int | None = 42, params: dict | None = None):
        self.hp = dict(hp)
        self.params = params if params is not None else init_params(hp, seed)
        self.layers = so3.model_paths(hp["lmax"], hp["n_layers"])
        self.C = hp["channels"]
        self.lmax = hp["lmax"]
        self.D = hp["two_body"][-1]
        self.nu = float(hp["avg_num_neighbors"])
        for L, (irr_in, paths, outs) in enumerate(self.layers, start=1):
            n0 = sum(1 for p in paths if p[2] == (0, 1))
            assert n0 == self.lmax + 1, "every layer sees all natural irreps"
        assert hp["latent"][-1] == self.D, "latent output width must equal the two-body width"

    # -------------------------------------------------------------------- forward
    def _forward(self, rvec, Zi, Zj, seg, nc):
        hp, P = self.hp, self.params
        C, lmax, D, NL = self.C, self.lmax, self.D, hp["n_layers"]
        E = rvec.shape[0]
        t = {}
        r = np.sqrt(np.einsum("ek,ek->e", rvec, rvec))
        uh = rvec / r[:, None]
        B, dB = bessel(r, hp["rc"], hp["n_basis"])
        f, df = envelope(r, hp["rc"], hp["poly_p"])
        Y = [so3.sh(l, uh) for l in range(lmax + 1)]
        t.update(r=r, uh=uh, B=B, dB=dB, f=f, df=df, Y=Y)

        inp = np.zeros((E, 2 * N_SPECIES + hp["n_basis"]))
        inp[np.arange(E), Zi - 1] = 1.0
        inp[np.arange(E), N_SPECIES + Zj - 1] = 1.0
        inp[:, 2 * N_SPECIES:] = B
        h, zs = inp, []
        for k in range(len(hp["two_body"])):
            W = P[f"W2b.{k}"]
            z = h @ W / math.sqrt(W.shape[0])
            zs.append(z)
            h = silu(z)
        t["z2b"], t["h2b"] = zs, h
        x = f[:, None] * h
        t["x"] = [x]
        V = None
        t["layers"] = []
        for L in range(1, NL + 1):
            irr_in, paths, outs = self.layers[L - 1]
            lt = {}
            w = (x @ P[f"Wenv.{L}"] / math.sqrt(D)).reshape(E, lmax + 1, C)
            G = []
            for l in range(lmax + 1):
                contrib = w[:, l, :, None] * Y[l][:, None, :]
                g = np.zeros((nc, C, 2 * l + 1))
                np.add.at(g, seg, contrib)
                G.append(g / math.sqrt(self.nu))
            if L == 1:
                V = {(l, (-1) ** l): w[:, l, :, None] * Y[l][:, None, :]
                     for l in range(lmax + 1)}
            T = []
            for (i_in, l2, out) in paths:
                cg = so3.coupling(irr_in[i_in][0], l2, out[0])
                T.append(tp(cg, V[irr_in[i_in]], G[l2][seg]))
            sc = [q for q, p in enumerate(paths) if p[2] == (0, 1)]
            s = np.stack([T[q][:, :, 0] for q in sc], axis=1).reshape(E, len(sc) * C)
            h = np.concatenate([x, s], axis=1)
            zl = []
            for k in range(len(hp["latent"])):
                W = P[f"Wlat.{L}.{k}"]
                z = h @ W / math.sqrt(W.shape[0])
                zl.append(z)
                h = silu(z)
            x_new = (x + f[:, None] * h) / SQRT2
            V_new = None
            if L < NL:
                theta = P[f"theta.{L}"]
                V_new = {}
                for out in outs:
                    qs = [q for q, p in enumerate(paths) if p[2] == out]
                    acc = sum(theta[q][None, :, None] * T[q] for q in qs)
                    V_new[out] = acc / math.sqrt(len(qs))
            lt.update(w=w, G=G, V=V, T=T, sc=sc, zl=zl, h=h)
            t["layers"].append(lt)
            x, V = x_new, V_new
            t["x"].append(x)
        e = x
        for k in range(len(hp["edge_eng"]) + 1):
            W = P[f"We.{k}"]
            e = e @ W / math.sqrt(W.shape[0])
        Eij = e[:, 0]
        t["Eij"] = Eij
        return Eij, t

    # -------------------------------------------------------------------- gradient
    def _backward(self, t, seg, nc):
        """g_e = dE/dr_e for E = sum of all edge energies (hand-derived reverse mode)."""
        hp, P = self.hp, self.params
        C, lmax, D, NL = self.C, self.lmax, self.D, hp["n_layers"]
        E = t["r"].shape[0]
        ge = np.ones((E, 1))
        for k in reversed(range(len(hp["edge_eng"]) + 1)):
            W = P[f"We.{k}"]
            ge = ge @ W.T / math.sqrt(W.shape[0])
        gx = ge                                  # dE/dx^N, [E, D]
        gV = None
        gY = [np.zeros_like(y) for y in t["Y"]]
        gf = np.zeros(E)
        f = t["f"]
        for L in reversed(range(1, NL + 1)):
            irr_in, paths, outs = self.layers[L - 1]
            lt = t["layers"][L - 1]
            # x^L = (x^(L-1) + f h) / sqrt2
            gh = gx * f[:, None] / SQRT2
            gf += np.einsum("ed,ed->e", gx, lt["h"]) / SQRT2
            gxp = gx / SQRT2
            for k in reversed(range(len(hp["latent"]))):
                W = P[f"Wlat.{L}.{k}"]
                gz = gh * silu_grad(lt["zl"][k])
                gh = gz @ W.T / math.sqrt(W.shape[0])
            gxp = gxp + gh[:, :D]
            gs = gh[:, D:].reshape(E, len(lt["sc"]), C)
            gT = [np.zeros_like(T) for T in lt["T"]]
            for a, q in enumerate(lt["sc"]):
                gT[q][:, :, 0] += gs[:, a, :]
            if L < NL:
                theta = P[f"theta.{L}"]
                for out in outs:
                    qs = [q for q, p in enumerate(paths) if p[2] == out]
                    for q in qs:
                        gT[q] += theta[q][None, :, None] * gV[out] / math.sqrt(len(qs))
            V, G = lt["V"], lt["G"]
            gVin = {ir: np.zeros_like(v) for ir, v in V.items()}
            gG = [np.zeros_like(g) for g in G]
            for q, (i_in, l2, out) in enumerate(paths):
                ir = irr_in[i_in]
                cg = so3.coupling(ir[0], l2, out[0])
                gv, gg = tp_adjoint(cg, gT[q], V[ir], G[l2][seg])
                gVin[ir] += gv
                np.add.at(gG[l2], seg, gg)
            w = lt["w"]
            gw = np.zeros_like(w)
            for l in range(lmax + 1):
                gGe = gG[l][seg] / math.sqrt(self.nu)
                gw[:, l, :] += (gGe * t["Y"][l][:, None, :]).sum(axis=2)
                gY[l] += (gGe * w[:, l, :, None]).sum(axis=1)
            if L == 1:
                for l in range(lmax + 1):
                    gv = gVin[(l, (-1) ** l)]
                    gw[:, l, :] += (gv * t["Y"][l][:, None, :]).sum(axis=2)
                    gY[l] += (gv * w[:, l, :, None]).sum(axis=1)
            gxp = gxp + gw.reshape(E, -1) @ P[f"Wenv.{L}"].T / math.sqrt(D)
            gx, gV = gxp, gVin
        # x^0 = f * h2b
        gf += np.einsum("ed,ed->e", gx, t["h2b"])
        gh = gx * f[:, None]
        for k in reversed(range(len(hp["two_body"]))):
            W = P[f"W2b.{k}"]
            gz = gh * silu_grad(t["z2b"][k])
            gh = gz @ W.T / math.sqrt(W.shape[0])
        gB = gh[:, 2 * N_SPECIES:]
        uh, r = t["uh"], t["r"]
        g_r = np.einsum("en,en->e", gB, t["dB"]) + gf * t["df"]
        g = g_r[:, None] * uh
        for l in range(1, lmax + 1):
            gu = np.einsum("em,emk->ek", gY[l], so3.sh_grad_u(l, uh))
            gu -= np.einsum("ek,ek->e", gu, uh)[:, None] * uh
            g += gu / r[:, None]
        return g

    # -------------------------------------------------------------------- drivers
    def edge_vectors(self, pos, box, i, j, s):
        return pos[j] - pos[i] + s.astype(np.float64) * np.asarray(box)[None, :]

    def evaluate(self, pos, Z, box, pbc, sys_ptr=None, forces=True, chunk_edges=200_000,
                 nl=None):
        """Total energy per system, per-atom energies and forces of a whole system."""
        pos = np.asarray(pos, dtype=np.float64)
        Z = np.asarray(Z)
        n = pos.shape[0]
        if sys_ptr is None:
            sys_ptr = np.array([0, n])
        if nl is None:
            nl = neighbors.neighbor_list(pos, box, pbc, self.hp["rc"], 0.0, sys_ptr)
        row_ptr, col, shift = nl
        E_atom = np.zeros(n)
        F = np.zeros((n, 3))
        c0 = 0
        while c0 < n:
            c1 = c0 + 1
            while c1 < n and row_ptr[c1 + 1] - row_ptr[c0] <= chunk_edges:
                c1 += 1
            e0, e1 = row_ptr[c0], row_ptr[c1]
            if e1 > e0:
                i = np.repeat(np.arange(c0, c1), np.diff(row_ptr[c0:c1 + 1]))
                j = col[e0:e1]
                rvec = self.edge_vectors(pos, box, i, j, shift[e0:e1])
                seg = i - c0
                Eij, t = self._forward(rvec, Z[i], Z[j], seg, c1 - c0)
                E_atom[c0:c1] += np.bincount(seg, Eij, minlength=c1 - c0)
                if forces:
                    g = self._backward(t, seg, c1 - c0)
                    np.add.at(F, i, g)
                    np.add.at(F, j, -g)
            c0 = c1
        E_sys = np.array([E_atom[sys_ptr[k]:sys_ptr[k + 1]].sum()
                          for k in range(len(sys_ptr) - 1)])
        return E_sys, E_atom, F

    def virial(self, pos, Z, box, pbc, sys_ptr=None):
        """Virial per system, W_ab = -sum_e r_e,a g_e,b (eV), g_e = dE/dr_e.

        Under a homogeneous strain x -> (1 + eps) x (box included) every edge vector maps
        to (1 + eps) r_e, so dE/d(eps_ab) = sum_e g_e,a r_e,b = -W_ba; the stress is
        sigma = -W / V.  (The paper trains on stresses; Methodology, Model Training.)"""
        pos = np.asarray(pos, dtype=np.float64)
        n = pos.shape[0]
        if sys_ptr is None:
            sys_ptr = np.array([0, n])
        nl = neighbors.neighbor_list(pos, box, pbc, self.hp["rc"], 0.0, sys_ptr)
        row_ptr, col, shift = nl
        W = np.zeros((len(sys_ptr) - 1, 3, 3))
        sys_of = np.searchsorted(np.asarray(sys_ptr), np.arange(n), side="right") - 1
        i = np.repeat(np.arange(n), np.diff(row_ptr))
        if col.shape[0] == 0:
            return W
        rvec = self.edge_vectors(pos, box, i, col, shift)
        _, t = self._forward(rvec, np.asarray(Z)[i], np.asarray(Z)[col], i, n)
        g = self._backward(t, i, n)
        for k in range(W.shape[0]):
            m = sys_of[i] == k
            W[k] = -rvec[m].T @ g[m]
        return W

    def centre_terms(self, pos, Z, box, pbc, centres, sys_ptr=None):
        """Per-centre energy E_i and edge gradients g_e of the given centres only.

        Returns {i: (E_i, col, shift, g)} -- what a sampled check at full size needs."""
        pos = np.asarray(pos, dtype=np.float64)
        nl = neighbors.neighbor_list(pos, box, pbc, self.hp["rc"], 0.0, sys_ptr,
                                     centres=centres)
        ids = sorted(nl)
        cols = [nl[i][0] for i in ids]
        shs = [nl[i][1] for i in ids]
        cnt = np.array([c.shape[0] for c in cols])
        i_e = np.repeat(np.array(ids), cnt)
        seg = np.repeat(np.arange(len(ids)), cnt)
        j_e = np.concatenate(cols) if cols else np.zeros(0, np.int64)
        s_e = np.concatenate(shs) if shs else np.zeros((0, 3), np.int64)
        out = {}
        if j_e.shape[0] == 0:
            return {i: (0.0, cols[a], shs[a], np.zeros((0, 3))) for a, i in enumerate(ids)}
        rvec = self.edge_vectors(pos, box, i_e, j_e, s_e)
        Eij, t = self._forward(rvec, np.asarray(Z)[i_e], np.asarray(Z)[j_e], seg, len(ids))
        g = self._backward(t, seg, len(ids))
        Ei = np.bincount(seg, Eij, minlength=len(ids))
        off = np.concatenate([[0], np.cumsum(cnt)])
        for a, i in enumerate(ids):
            out[i] = (Ei[a], cols[a], shs[a], g[off[a]:off[a + 1]])
        return out

    def readout_scale(self, pos, Z, box, pbc, atoms, sys_ptr=None):
        """Per atom i: sum over its edges and latent columns of |x^N_ijd w_d|, where
        w = We.0 We.1 ... / prod sqrt(fan_in) is the linear edge-energy readout composed into
        one vector (Table 1: no non-linearity), so E_ij = sum_d x^N_ijd w_d.  A relative
        perturbation of at most u in every x^N component moves E_i by at most u times this
        scale; it sets the scale of reduced-precision per-atom energy errors (the per-atom
        energies themselves can be far smaller through cancellation)."""
        pos = np.asarray(pos, dtype=np.float64)
        nl = neighbors.neighbor_list(pos, box, pbc, self.hp["rc"], 0.0, sys_ptr,
                                     centres=atoms)
        ids = sorted(nl)
        cnt = np.array([nl[i][0].shape[0] for i in ids])
        if cnt.sum() == 0:
            return {i: 0.0 for i in ids}
        i_e = np.repeat(np.array(ids), cnt)
        seg = np.repeat(np.arange(len(ids)), cnt)
        j_e = np.concatenate([nl[i][0] for i in ids])
        s_e = np.concatenate([nl[i][1] for i in ids])
        rvec = self.edge_vectors(pos, box, i_e, j_e, s_e)
        _, t = self._forward(rvec, np.asarray(Z)[i_e], np.asarray(Z)[j_e], seg, len(ids))
        w = np.eye(self.D)
        for k in range(len(self.hp["edge_eng"]) + 1):
            W = self.params[f"We.{k}"]
            w = w @ W / math.sqrt(W.shape[0])
        sc = np.bincount(seg, np.abs(t["x"][-1] * w[:, 0][None, :]).sum(axis=1),
                         minlength=len(ids))
        return {i: float(sc[a]) for a, i in enumerate(ids)}

    def sampled_forces(self, pos, Z, box, pbc, atoms, sys_ptr=None):
        """Forces on a few atoms m, from the edges out of m and the edges into m."""
        pos = np.asarray(pos, dtype=np.float64)
        nl = neighbors.neighbor_list(pos, box, pbc, self.hp["rc"], 0.0, sys_ptr,
                                     centres=atoms)
        need = set(atoms)
        for m in atoms:
            need.update(int(j) for j in nl[m][0])
        terms = self.centre_terms(pos, Z, box, pbc, sorted(need), sys_ptr)
        F = {}
        for m in atoms:
            Fm = terms[m][3].sum(axis=0) if terms[m][3].shape[0] else np.zeros(3)
            for i, (_, col, _, g) in terms.items():
                hit = col == m
                if hit.any():
                    Fm = Fm - g[hit].sum(axis=0)
            F[m] = Fm
        return F, {m: terms[m][0] for m in atoms}

#!/usr/bin/env python3
"""Generate tp_gen.cuh: unrolled Clebsch-Gordan tensor products for the CUDA path.

Allegro-FM uses e3nn tensor products of edge features with the environment embedding,
l <= 2 "in full O(3) symmetry" (arXiv 2502.06073, Methodology, Model Training).  The
real-basis coupling tensors are derived here from the Racah formula for the complex
Clebsch-Gordan coefficients and the complex-to-real change of basis of the spherical
harmonics (Condon-Shortley phase), then normalised to sum C^2 = 2 l3 + 1 with the first
non-zero entry (lexicographic in m1, m2, m3) positive.  The emitted code multiplies only
the non-zero entries, fully unrolled, per channel.

Irreps are (l, p); per-channel feature vectors list their irreps by l and, within one l,
natural parity (-1)^l first.  A layer couples every input irrep (l1, p1) with the
environment irreps (l2, (-1)^l2), l2 = 0..lmax, into (l3, p1 (-1)^l2) for
|l1 - l2| <= l3 <= min(l1 + l2, lmax); the last layer keeps only the 0e outputs.
Input kinds: 0 = natural irreps (first layer), 1 = the outputs of a first layer, 2 = the
outputs of a later layer (all irreps reachable).
Output kinds: 0 = every reachable irrep, 1 = natural-parity irreps only, 2 = 0e only (the
last layer).  Kind 1 is the layer before the last: a 0e output of the last layer couples
(l1, p1) with (l2, (-1)^l2) only for l1 = l2 and p1 = (-1)^l1, so the other outputs of
that layer never reach the energy and are not computed.  Path weights keep the index of
the path in the full list of the layer, and the 1/sqrt(n) mixing counts all paths into
an irrep, so the kept outputs are exactly those of the full layer.

Usage: python gen_tp.py [output path]   (default: tp_gen.cuh next to this file)
"""
from __future__ import annotations

import math
import os
import struct
import sys
from fractions import Fraction

LMAX_SUPPORTED = (1, 2)


# --------------------------------------------------------------------- coefficients
def _fact(n):
    return math.factorial(n)


def cg_complex(j1, m1, j2, m2, J, M):
    """<j1 m1 j2 m2 | J M> by the Racah formula (integer spins), exact then float."""
    if m1 + m2 != M or abs(m1) > j1 or abs(m2) > j2 or abs(M) > J:
        return 0.0
    if not (abs(j1 - j2) <= J <= j1 + j2):
        return 0.0
    pre = Fraction((2 * J + 1) * _fact(J + j1 - j2) * _fact(J - j1 + j2) * _fact(j1 + j2 - J),
                   _fact(j1 + j2 + J + 1))
    pre *= (_fact(J + M) * _fact(J - M) * _fact(j1 - m1) * _fact(j1 + m1)
            * _fact(j2 - m2) * _fact(j2 + m2))
    s = Fraction(0)
    for k in range(0, j1 + j2 + J + 2):
        d = [k, j1 + j2 - J - k, j1 - m1 - k, j2 + m2 - k, J - j2 + m1 + k, J - j1 - m2 + k]
        if min(d) < 0:
            continue
        den = 1
        for x in d:
            den *= _fact(x)
        s += Fraction((-1) ** k, den)
    return math.sqrt(pre) * float(s)


def real_from_complex(l):
    """U with Y_real = U Y_complex (rows: real m = -l..l, cols: complex m = -l..l)."""
    n = 2 * l + 1
    U = [[0j] * n for _ in range(n)]
    r2 = 1.0 / math.sqrt(2.0)
    for m in range(-l, l + 1):
        row = m + l
        if m > 0:
            U[row][m + l] = (-1) ** m * r2
            U[row][-m + l] = r2
        elif m == 0:
            U[row][l] = 1.0
        else:
            mu = -m
            U[row][-mu + l] = 1j * r2
            U[row][mu + l] = -1j * (-1) ** mu * r2
    return U


def coupling_real(l1, l2, l3):
    U1, U2, U3 = real_from_complex(l1), real_from_complex(l2), real_from_complex(l3)
    n1, n2, n3 = 2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1
    C = [[[0j] * n3 for _ in range(n2)] for _ in range(n1)]
    for a in range(n1):
        for b in range(n2):
            for c in range(n3):
                acc = 0j
                for m1 in range(-l1, l1 + 1):
                    u1 = U1[a][m1 + l1].conjugate()
                    if u1 == 0:
                        continue
                    for m2 in range(-l2, l2 + 1):
                        u2 = U2[b][m2 + l2].conjugate()
                        if u2 == 0:
                            continue
                        M = m1 + m2
                        if abs(M) > l3:
                            continue
                        u3 = U3[c][M + l3]
                        if u3 == 0:
                            continue
                        acc += u3 * cg_complex(l1, m1, l2, m2, l3, M) * u1 * u2
                C[a][b][c] = acc
    flat = [C[a][b][c] for a in range(n1) for b in range(n2) for c in range(n3)]
    re = sum(abs(z.real) for z in flat)
    im = sum(abs(z.imag) for z in flat)
    vals = [z.real for z in flat] if re >= im else [z.imag for z in flat]
    norm = math.sqrt(sum(v * v for v in vals))
    vals = [v * math.sqrt(2 * l3 + 1) / norm for v in vals]
    vals = [0.0 if abs(v) < 1e-12 else v for v in vals]
    first = next(v for v in vals if v != 0.0)
    if first < 0:
        vals = [-v for v in vals]
    out = {}
    k = 0
    for a in range(n1):
        for b in range(n2):
            for c in range(n3):
                if vals[k] != 0.0:
                    out[(a, b, c)] = vals[k]
                k += 1
    return out


# --------------------------------------------------------------------- irreps / paths
def canon(irreps):
    return sorted(set(irreps), key=lambda ir: (ir[0], 0 if ir[1] == (-1) ** ir[0] else 1))


def layer(in_irreps, lmax, last):
    paths = []
    for i_in, (l1, p1) in enumerate(in_irreps):
        for l2 in range(lmax + 1):
            p2 = (-1) ** l2
            for l3 in range(abs(l1 - l2), min(l1 + l2, lmax) + 1):
                out = (l3, p1 * p2)
                if last and out != (0, 1):
                    continue
                paths.append((i_in, l2, out))
    return paths, canon([p[2] for p in paths])


def natural(ir):
    return ir[1] == (-1) ** ir[0]


# (input kind, output kind) pairs the layers of a model with 1..4 layers use
KINDS = ((0, 0), (0, 1), (0, 2), (1, 0), (1, 1), (2, 1))


def layer_kinds(L, n_layers):
    """(input kind, output kind) of layer L; input kind 3 = natural irreps read from the
    previous layer's output (same products as input kind 0)."""
    outk = 2 if L == n_layers else (1 if L == n_layers - 1 else 0)
    if L == 1:
        return 0, outk
    if L == n_layers:
        return 3, outk
    return min(L - 1, 2), outk


def in_irreps_of(lmax, in_kind):
    irr = [(l, (-1) ** l) for l in range(lmax + 1)]
    for _ in range(in_kind):
        _, irr = layer(irr, lmax, False)
    return irr


def offsets(irreps):
    off, o = [], 0
    for (l, _p) in irreps:
        off.append(o)
        o += 2 * l + 1
    return off, o


def f32(x):
    """x rounded to float32 (the value of the literal fl(x) in CUDA)."""
    return struct.unpack("f", struct.pack("f", x))[0]


def fl(x):
    s = repr(float(x))
    if "e" not in s and "." not in s:
        s += ".0"
    return s + "f"


def gen_kind(lmax, in_kind, out_kind):
    last = out_kind == 2
    irr_in = in_irreps_of(lmax, in_kind)
    full, full_outs = layer(irr_in, lmax, last)
    n_into = {o: sum(1 for p in full if p[2] == o) for o in full_outs}
    scal = [q for q, p in enumerate(full) if p[2] == (0, 1)]
    # kept paths with their index in the full list (path weights, scalar order)
    kept = [(q, p) for q, p in enumerate(full) if out_kind != 1 or natural(p[2])]
    outs = [o for o in full_outs if out_kind != 1 or natural(o)]
    off_in, din = offsets(irr_in)
    off_out, dout = offsets(outs) if not last else ([], 0)
    goff = [l * l for l in range(lmax + 1)]
    name = f"TP<{lmax}, {in_kind}, {out_kind}>"
    lines = []
    lines.append(f"template <> struct TP<{lmax}, {in_kind}, {out_kind}> {{")
    lines.append(f"  // in irreps {irr_in}; out irreps {outs if not last else [(0, 1)]}")
    lines.append(f"  static constexpr int NP = {len(full)}, DIN = {din}, "
                 f"DOUT = {max(dout, 1)}, NS = {len(scal)}, NPW = {0 if last else len(full)};")
    # forward
    lines.append("  template <int TS>")
    lines.append("  static __device__ __forceinline__ void fwd(const float* __restrict__ v, "
                 "const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {")
    if not last:
        lines.append(f"    #pragma unroll\n    for (int k = 0; k < {dout}; ++k) vo[k] = 0.f;")
    nnz_total = 0
    for q, (i_in, l2, out) in kept:
        l1 = irr_in[i_in][0]
        l3 = out[0]
        C = coupling_real(l1, l2, l3)
        nnz_total += len(C)
        lines.append(f"    {{ // path {q}: {irr_in[i_in]} x ({l2},{(-1) ** l2}) -> {out}")
        for c in range(2 * l3 + 1):
            terms = [f"{fl(v)} * v[{off_in[i_in] + a}] * g[{goff[l2] + b}]"
                     for (a, b, cc), v in sorted(C.items()) if cc == c]
            lines.append(f"      const float t{c} = " + (" + ".join(terms) if terms else "0.f")
                         + ";")
        if out == (0, 1):
            lines.append(f"      s[{scal.index(q)}] = t0;")
        if not last:
            oo = off_out[outs.index(out)]
            lines.append(f"      const float w = th[{q} * TS];")
            for c in range(2 * l3 + 1):
                lines.append(f"      vo[{oo + c}] += w * t{c};")
        lines.append("    }")
    lines.append("  }")
    # backward
    lines.append("  template <int TS>")
    lines.append("  static __device__ __forceinline__ void bwd(const float* __restrict__ v, "
                 "const float* __restrict__ g, const float* __restrict__ th, "
                 "const float* __restrict__ gs, const float* __restrict__ gvo, "
                 "float* gv, float* gg) {")
    for q, (i_in, l2, out) in kept:
        l1 = irr_in[i_in][0]
        l3 = out[0]
        C = coupling_real(l1, l2, l3)
        lines.append(f"    {{ // path {q}")
        if not last:
            oo = off_out[outs.index(out)]
            lines.append(f"      const float w = th[{q} * TS];")
        for c in range(2 * l3 + 1):
            parts = []
            if out == (0, 1) and c == 0:
                parts.append(f"gs[{scal.index(q)}]")
            if not last:
                parts.append(f"w * gvo[{oo + c}]")
            lines.append(f"      const float gt{c} = " + (" + ".join(parts) if parts else "0.f")
                         + ";")
        # one product |C| gt_c per (output component, float32 magnitude), shared by the
        # entries of either sign: fma(-s, x, y) equals y + (C gt_c) x exactly for C < 0
        prods = {}
        for (a, b, c), val in sorted(C.items()):
            mag = f32(abs(val))
            if (c, mag) not in prods:
                name = f"s{c}_{len([k for k in prods if k[0] == c])}"
                prods[(c, mag)] = name
                rhs = f"gt{c}" if mag == 1.0 else f"{fl(abs(val))} * gt{c}"
                lines.append(f"      const float {name} = {rhs};")
            sv = ("" if val > 0 else "-") + prods[(c, mag)]
            ia, ib = off_in[i_in] + a, goff[l2] + b
            lines.append(f"      gv[{ia}] = fmaf({sv}, g[{ib}], gv[{ia}]);"
                         f" gg[{ib}] = fmaf({sv}, v[{ia}], gg[{ib}]);")
        lines.append("    }")
    lines.append("  }")
    lines.append(f"  static constexpr int NNZ = {nnz_total};")
    lines.append("};")
    scale = [1.0 / math.sqrt(n_into[p[2]]) for p in full]
    return name, lines, dict(np=len(full), kept=len(kept), din=din, dout=dout, ns=len(scal),
                             nnz=nnz_total, irr_in=irr_in, outs=outs, scale=scale)


def main(out_path):
    body = []
    table = []
    for lmax in LMAX_SUPPORTED:
        for in_kind, out_kind in KINDS:
            _, lines, info = gen_kind(lmax, in_kind, out_kind)
            body.extend(lines)
            body.append("")
            table.append((lmax, in_kind, out_kind, info))
    hdr = [
        "// Generated by gen_tp.py -- do not edit.  Unrolled real Clebsch-Gordan tensor",
        "// products (Racah formula + complex-to-real basis change), per channel.",
        "// fwd: T_path = C (v_in x g); s[] = 0e outputs; vo[] = sum theta_path T / sqrt(n).",
        "// bwd: given gs (d/ds) and gvo (d/dvo): gv += dT/dv^T gT, gg += dT/dg^T gT.",
        "// Output kind 0: all reachable irreps, 1: natural-parity irreps, 2: 0e only.",
        "#pragma once",
        "",
        "template <int LMAX, int INK, int OUTK> struct TP;",
        "",
        "struct TPKindInfo {",
        "  int lmax, in_kind, out_kind, n_paths, n_kept, dim_in, dim_out, n_scalar, nnz;",
        "};",
        "static const TPKindInfo kTPKinds[] = {",
    ]
    for (lmax, ink, outk, info) in table:
        hdr.append(f"  {{{lmax}, {ink}, {outk}, {info['np']}, {info['kept']}, {info['din']}, "
                   f"{info['dout']}, {info['ns']}, {info['nnz']}}},")
    hdr.append("};")
    hdr.append(f"static const int kNumTPKinds = {len(table)};")
    maxp = max(info["np"] for (_, _, _, info) in table)
    hdr.append("// 1/sqrt(paths into the output irrep) of every path, per kind (rows as above): the")
    hdr.append("// weights are stored as theta_path times this, and fwd/bwd read them at th[q * TS].")
    hdr.append(f"static const float kTPPathScale[][{maxp}] = {{")
    for (_, _, _, info) in table:
        hdr.append("  {" + ", ".join(fl(x) for x in info["scale"]) + "},")
    hdr.append("};")
    hdr.append("")
    with open(out_path, "w") as f:
        f.write("\n".join(hdr + body) + "\n")


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "tp_gen.cuh"))

"""Writes fe_gll_tables.h: the shape-only 1D tables of the float Hamiltonian operator kernel
and of the float Gauss-quadrature potential kernel.

For degree p the in-plane contractions of the mass-scaled operator use
  MS[j][k] = M1[j][k] sig_k,   KS[j][k] = K1[j][k] sig_k,
with M1, K1 the exactly integrated 1D mass and stiffness matrices of the Lagrange basis on the
p + 1 Gauss-Lobatto-Legendre nodes of [-1, 1] and sig_k = 1 / sqrt(m_k) (m_k = w_k, or 2 w_0 at
a node shared by two cells).  They depend on p only; the mesh enters through the scalars
ax, ay at run time.  GB[q][i] = l_i(g_q) interpolates from the GLL nodes to the p + 1
Gauss-Legendre points g_q of [-1, 1] (the potential integrated by Gauss quadrature).  The rules are computed the way the library's mesh set-up computes them
(three-term Legendre recurrence, Newton from the same starting points, (p+1)-point Gauss
quadrature of the products) and rounded to float.

Run: python gen_gll_tables.py  (writes fe_gll_tables.h beside this script).
"""
import math
import os


def legendre(n, x):
    p0, p1 = 1.0, x
    if n == 0:
        return 1.0, 0.0
    for k in range(2, n + 1):
        p0, p1 = p1, ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k
    dp = n * (x * p1 - p0) / (x * x - 1.0) if abs(x * x - 1.0) > 1e-300 else 0.0
    return p1, dp


def gll_rule(p):
    x = [0.0] * (p + 1)
    x[0], x[p] = -1.0, 1.0
    for i in range(1, p):
        t = -math.cos(math.pi * i / p)
        for _ in range(100):
            P, dP = legendre(p, t)
            d2 = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t)
            dt = dP / d2
            t -= dt
            if abs(dt) < 1e-16:
                break
        x[i] = t
    w = [2.0 / (p * (p + 1.0) * legendre(p, xi)[0] ** 2) for xi in x]
    return x, w


def gauss_rule(q):
    xs, ws = [], []
    for i in range(q):
        t = math.cos(math.pi * (i + 0.75) / (q + 0.5))
        for _ in range(100):
            P, dP = legendre(q, t)
            dt = P / dP
            t -= dt
            if abs(dt) < 1e-16:
                break
        P, dP = legendre(q, t)
        xs.append(t)
        ws.append(2.0 / ((1.0 - t * t) * dP * dP))
    return xs, ws


def lagrange(xn, i, t):
    v, d = 1.0, 0.0
    for j in range(len(xn)):
        if j == i:
            continue
        f = (t - xn[j]) / (xn[i] - xn[j])
        d = d * f + v / (xn[i] - xn[j])
        v *= f
    return v, d


def tables(p):
    n1 = p + 1
    xi, w = gll_rule(p)
    gq, gw = gauss_rule(n1)
    K1 = [[0.0] * n1 for _ in range(n1)]
    M1 = [[0.0] * n1 for _ in range(n1)]
    for a in range(n1):
        ld = [lagrange(xi, i, gq[a]) for i in range(n1)]
        for i in range(n1):
            for j in range(n1):
                K1[i][j] += gw[a] * ld[i][1] * ld[j][1]
                M1[i][j] += gw[a] * ld[i][0] * ld[j][0]
    sig = [1.0 / math.sqrt(2.0 * w[0] if k in (0, p) else w[k]) for k in range(n1)]
    MS = [[M1[j][k] * sig[k] for k in range(n1)] for j in range(n1)]
    KS = [[K1[j][k] * sig[k] for k in range(n1)] for j in range(n1)]
    return MS, KS


def gauss_interp(p):
    xi, _ = gll_rule(p)
    gq = sorted(gauss_rule(p + 1)[0])   # ascending, as the points of a cell are ordered
    return [[lagrange(xi, i, gq[q])[0] for i in range(p + 1)] for q in range(p + 1)]


def f32(v):
    import struct
    return struct.unpack("f", struct.pack("f", v))[0]


def emit(name, A):
    rows = ",\n    ".join("{" + ", ".join(repr(f32(v)) + "f" for v in r) + "}" for r in A)
    return f"__device__ constexpr float {name}[{len(A)}][{len(A)}] = {{\n    {rows}}};\n"


def main():
    out = ["// Generated by gen_gll_tables.py (do not edit): shape-only 1D tables M1 sig and K1 sig",
           "// of the float Hamiltonian operator and the GLL-to-Gauss interpolation GB for",
           "// p = 1..6 (see the script for their definition).",
           "#pragma once", "", "namespace fe {", ""]
    for p in range(1, 7):
        MS, KS = tables(p)
        out.append(emit(f"kGllMS{p}", MS))
        out.append(emit(f"kGllKS{p}", KS))
        out.append(emit(f"kGaussB{p}", gauss_interp(p)))
    out.append("""// MS[j][k] and KS[j][k] of degree P (compile-time indices fold to immediates)
template <int P>
__device__ __forceinline__ constexpr float gll_ms(int j, int k) {
  if constexpr (P == 1) return kGllMS1[j][k];
  else if constexpr (P == 2) return kGllMS2[j][k];
  else if constexpr (P == 3) return kGllMS3[j][k];
  else if constexpr (P == 4) return kGllMS4[j][k];
  else if constexpr (P == 5) return kGllMS5[j][k];
  else return kGllMS6[j][k];
}
template <int P>
__device__ __forceinline__ constexpr float gll_ks(int j, int k) {
  if constexpr (P == 1) return kGllKS1[j][k];
  else if constexpr (P == 2) return kGllKS2[j][k];
  else if constexpr (P == 3) return kGllKS3[j][k];
  else if constexpr (P == 4) return kGllKS4[j][k];
  else if constexpr (P == 5) return kGllKS5[j][k];
  else return kGllKS6[j][k];
}
// GB[q][i] of degree P
template <int P>
__device__ __forceinline__ constexpr float gauss_b(int q, int i) {
  if constexpr (P == 1) return kGaussB1[q][i];
  else if constexpr (P == 2) return kGaussB2[q][i];
  else if constexpr (P == 3) return kGaussB3[q][i];
  else if constexpr (P == 4) return kGaussB4[q][i];
  else if constexpr (P == 5) return kGaussB5[q][i];
  else return kGaussB6[q][i];
}

}  // namespace fe""")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fe_gll_tables.h")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()

"""Writes oracle/sg_gp_table.h: the Gauss-Patterson rules of the oracle
(test infrastructure; the library computes its own rules independently).

Gauss-Patterson rules (Section 2.2, Eq. 2.12; Patterson 1968) are nested: the
rule of level g has 2^g - 1 nodes on [-1, 1].  Level 1 is the midpoint rule
(the zero of P_1); level g+1 keeps the n = 2^g - 1 nodes of level g and adds
the n + 1 zeros of the polynomial G of degree n + 1 that is orthogonal, with
respect to the weight Q(x) = prod_j (x - x_j) over the existing nodes, to
every polynomial of degree <= n.  The resulting interpolatory rule is exact
for polynomials of degree 3n + 1 (3n + 2 by symmetry): 1, 5, 11, 23, 47, 95,
191 for 1, 3, 7, ..., 127 nodes.

Everything is computed with mpmath at 300 digits from these definitions:
  1. G's monomial coefficients from the n + 1 orthogonality conditions
     int_{-1}^{1} Q(x) G(x) x^k dx = 0, k = 0..n (moments 2/(m+1), m even);
  2. its zeros, one in each gap between consecutive existing nodes and in
     the two end gaps (the zeros interlace with the existing nodes), by
     bisection-safeguarded root finding;
  3. the weights of the interpolatory rule from the moment equations
     sum_j w_j x_j^k = int_{-1}^{1} x^k dx, k = 0..N-1.
The rules are mapped to [0, 1] (x -> (x+1)/2, w -> w/2) and rounded to
double once.  Run: python oracle/gen_gp_table.py (writes the header).
"""
import os
import sys

import mpmath as mp

LEVELS = 7  # 1, 3, 7, 15, 31, 63, 127 nodes
mp.mp.dps = 300


def moment(m):
    return mp.mpf(2) / (m + 1) if m % 2 == 0 else mp.mpf(0)


def poly_from_roots(roots):
    # monic, coefficients c[i] of x^i
    c = [mp.mpf(1)]
    for r in roots:
        nc = [mp.mpf(0)] * (len(c) + 1)
        for i, ci in enumerate(c):
            nc[i + 1] += ci
            nc[i] -= r * ci
        c = nc
    return c


def horner(c, x):
    v = mp.mpf(0)
    for ci in reversed(c):
        v = v * x + ci
    return v


def extend(nodes):
    n = len(nodes)
    q = poly_from_roots(nodes)
    # int Q x^m = sum_j q_j moment(j + m)
    def qm(m):
        return mp.fsum(q[j] * moment(j + m) for j in range(len(q)))
    A = mp.matrix(n + 1, n + 1)
    b = mp.matrix(n + 1, 1)
    for k in range(n + 1):
        for i in range(n + 1):
            A[k, i] = qm(i + k)
        b[k] = -qm(n + 1 + k)
    g = mp.lu_solve(A, b)
    gc = [g[i] for i in range(n + 1)] + [mp.mpf(1)]
    edges = [mp.mpf(-1)] + sorted(nodes) + [mp.mpf(1)]
    new = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        flo, fhi = horner(gc, lo), horner(gc, hi)
        if flo == 0:
            new.append(lo)
            continue
        if flo * fhi > 0:
            raise RuntimeError("no sign change in a gap: the zeros do not interlace")
        a, bb = lo, hi
        for _ in range(1200):  # bisection to the working precision
            mid = (a + bb) / 2
            fm = horner(gc, mid)
            if fm == 0:
                a = bb = mid
                break
            if (fm > 0) == (flo > 0):
                a, flo = mid, fm
            else:
                bb = mid
        new.append((a + bb) / 2)
    return sorted(list(nodes) + new)


def weights(nodes):
    N = len(nodes)
    V = mp.matrix(N, N)
    m = mp.matrix(N, 1)
    for k in range(N):
        for j in range(N):
            V[k, j] = nodes[j] ** k
        m[k] = moment(k)
    w = mp.lu_solve(V, m)
    return [w[j] for j in range(N)]


def build():
    rules = []
    nodes = [mp.mpf(0)]
    for g in range(1, LEVELS + 1):
        if g > 1:
            nodes = extend(nodes)
        w = weights(nodes)
        # symmetric by construction up to rounding at 300 digits; exactness check
        n = len(nodes)
        deg = 1 if g == 1 else 3 * ((n - 1) // 2) + 2
        for k in range(deg + 1):
            err = mp.fsum(wj * xj ** k for wj, xj in zip(w, nodes)) - moment(k)
            if abs(err) > mp.mpf(10) ** -250:
                raise RuntimeError("level %d not exact at degree %d" % (g, k))
        if min(w) <= 0:
            raise RuntimeError("non-positive weight at level %d" % g)
        rules.append(([(x + 1) / 2 for x in nodes], [wj / 2 for wj in w]))
    return rules


def main(path):
    rules = build()
    L = ["/* Gauss-Patterson rules on [0,1] for the oracle (test infrastructure).",
         " * Generated by oracle/gen_gp_table.py (Patterson extensions computed at",
         " * 300 digits with mpmath, rounded to double once); do not edit. */",
         "#define OR_GP_LEVELS %d" % LEVELS, ""]
    for g, (x, w) in enumerate(rules, start=1):
        n = len(x)
        L.append("static const double or_gp_x%d[%d] = {" % (g, n))
        L += ["    %s," % float(v).hex() for v in x]
        L.append("};")
        L.append("static const double or_gp_w%d[%d] = {" % (g, n))
        L += ["    %s," % float(v).hex() for v in w]
        L.append("};")
    L.append("static const double *const or_gp_x[OR_GP_LEVELS + 1] = {0, %s};"
             % ", ".join("or_gp_x%d" % g for g in range(1, LEVELS + 1)))
    L.append("static const double *const or_gp_w[OR_GP_LEVELS + 1] = {0, %s};"
             % ", ".join("or_gp_w%d" % g for g in range(1, LEVELS + 1)))
    with open(path, "w") as f:
        f.write("\n".join(L) + "\n")


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "sg_gp_table.h"))

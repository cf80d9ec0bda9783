"""Print the constant tables of toom.cu (needs sympy; run from anywhere).

Toom-K over F2[X] with x = X^32 evaluates at 0, inf and the 2K - 3 finite
nonzero points below; their pairwise differences factor into x, x + 1 and
x^2 + x + 1 only.  For each coefficient C_k (1 <= k <= 2K - 3) of the
product polynomial the Vandermonde system over F2(x) is solved in
common-denominator form: C_k = (sum_j P_kj(x) S_j) / (x^a (x+1)^b (x^2+x+1)^c)
with S_j = R(p_j) - C_0 - C_(2K-2) p_j^(2K-2).  Polynomials in x are printed
as lists of exponents (coefficients in F2)."""
import sympy as sp

x = sp.symbols("x")
POINTS = {
    4: [sp.Integer(1), x, x + 1, x**2, x**2 + 1],
    5: [sp.Integer(1), x, x + 1, x**2, x**2 + 1, x**2 + x, x**2 + x + 1],
}


def exps(e):
    p = sp.Poly(sp.expand(e), x, modulus=2)
    return sorted(int(m[0]) for m in p.monoms()) if not p.is_zero else []


def tables(K):
    pts = POINTS[K]
    nf = 2 * K - 3
    V = sp.Matrix([[p**k for k in range(1, nf + 1)] for p in pts])
    Vi = V.inv()
    interp = []
    for k in range(nf):
        nds = [sp.fraction(sp.together(sp.expand(Vi[k, j]))) for j in range(nf)]
        nds = [(sp.Poly(n, x, modulus=2), sp.Poly(d, x, modulus=2)) for n, d in nds]
        D = sp.Poly(1, x, modulus=2)
        for _, d in nds:
            D = sp.lcm(D, d)
        terms = []
        for n, d in nds:
            q, r = sp.div(D, d)
            assert r.is_zero
            terms.append(exps((n * q).as_expr()))
        fac = {str(f): int(e) for f, e in sp.factor_list(D.as_expr(), modulus=2)[1]}
        a, b, c = fac.pop("x", 0), fac.pop("x + 1", 0), fac.pop("x**2 + x + 1", 0)
        assert not fac, fac
        interp.append((a, b, c, terms))
    # p_j^i for the evaluation (points 0, finite nonzero ..., inf)
    pow_rows = [[[0]] + [[] for _ in range(K - 1)]]
    for p in pts:
        pow_rows.append([exps(p**i) for i in range(K)])
    pow_rows.append([[] for _ in range(K - 1)] + [[0]])
    top = [exps(p**(2 * K - 2)) for p in pts]
    return pow_rows, top, interp


def c_list(v):
    return "{" + ", ".join(str(e) for e in v) + "}"


def main():
    for K in (4, 5):
        pow_rows, top, interp = tables(K)
        print(f"// Toom-{K}")
        print(f"__constant__ ExpSet kPow{K}[{2 * K - 1}][{K}] = {{")
        for row in pow_rows:
            print("    {" + ", ".join(f"{{{len(s)}, {c_list(s or [0])}}}" for s in row) + "},")
        print("};")
        print(f"__constant__ ExpSet kTop{K}[{2 * K - 3}] = {{" + ", ".join(f"{{{len(s)}, {c_list(s)}}}" for s in top) + "};")
        print(f"__constant__ Interp kInterp{K}[{2 * K - 3}] = {{")
        for a, b, c, terms in interp:
            print(f"    {{{a}, {b}, {c}, {c_list([len(t) for t in terms])}, "
                  + "{" + ", ".join(c_list(t or [0]) for t in terms) + "}},")
        print("};")


if __name__ == "__main__":
    main()

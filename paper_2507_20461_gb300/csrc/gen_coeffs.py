"""Generate ``geno_coeffs.cuh``: the fixed linear maps of the GENO
reconstructions (compact and 1D non-compact), derived in exact rational arithmetic (sympy) and emitted as
straight-line device code.

Run ``python gen_coeffs.py`` after changing the stencils; the output is
committed so that building the library needs no sympy.

What is derived (cell units, reconstruction cell [-1/2, 1/2]^m):

1D (Sec. 4.2): the eighth-order polynomial p^7 on the four cells j-1..j+2
with their averages and averaged derivatives; its value and derivative at
the shared face x_{j+1/2} (identical for the left and the right state,
because the stencil is symmetric about the face).  The three sub-stencil
quadratics of each side are written by hand in the kernel (closed forms).

multi-D (Sec. 4.3 specialised to Cartesian cells): the cubic P = W0 +
sum_k c_k (mono_k - <mono_k>_0) fitted by least squares to the averages and
averaged gradients of the 2m face neighbours and the own averaged gradient;
the map data -> c, the quadratic forms of IS^H (|l| = 1..3) and IS^tau
(|l| = 3), and P - W0 and grad P at every face Gauss point.  In 3D the
monomial xi*eta*zeta is left out: it has zero average and zero averaged
gradient on all seven cells of the stencil.
"""
import itertools
import os

import sympy as sp
from sympy.printing.c import C99CodePrinter

HERE = os.path.dirname(os.path.abspath(__file__))
x, y, z = sp.symbols("x y z", real=True)
X = (x, y, z)
half = sp.Rational(1, 2)


def cell_avg(expr, off, m):
    r = expr
    for a in range(m):
        r = sp.integrate(r, (X[a], off[a] - half, off[a] + half))
    return sp.nsimplify(r)


def lit(v):
    v = sp.Rational(v)
    if v == 0:
        return "R(0)"
    return f"R({float(v)!r})"


def emit_assignments(lines, exprs, names, indent="    "):
    """cse + emit `name = expr;` with R-typed temporaries."""
    repl, red = sp.cse(exprs, symbols=sp.numbered_symbols("t"), optimizations="basic")
    out = []
    for s, e in repl:
        out.append(f"{indent}const R {s} = {ccode(e)};")
    for n, e in zip(names, red):
        out.append(f"{indent}{n} = {ccode(e)};")
    lines.extend(out)


def emit_linear(lines, exprs, names, syms, indent="    "):
    """Emit `name = sum_k K_k * syms[k];` for expressions linear in syms, each
    coefficient folded (exactly, surds included) into one literal, so that a
    term costs one fused multiply-add (a product of two literals would cost a
    multiply more: the compiler may not reassociate floating-point
    products)."""
    for n, e in zip(names, exprs):
        e = sp.expand(e)
        terms = []
        for k, sym in enumerate(syms):
            K = sp.nsimplify(e.coeff(sym))
            if K == 0:
                continue
            kv = float(K)
            v = f"{sym}"
            if kv == 1.0:
                t = v
            elif kv == -1.0:
                t = f"-{v}"
            else:
                t = f"R({kv!r})*{v}"
            terms.append(t)
        rest = sp.expand(e - sum(e.coeff(sym) * sym for sym in syms))
        assert rest == 0, "expression is not linear in the given symbols"
        body = " + ".join(terms).replace("+ -", "- ") if terms else "R(0)"
        lines.append(f"{indent}{n} = {body};")


class _Printer(C99CodePrinter):
    def _print_Rational(self, e):
        return lit(e)

    def _print_Integer(self, e):
        return lit(e)

    def _print_Float(self, e):
        return f"R({float(e)!r})"

    def _print_Pow(self, e):
        b, p = e.as_base_exp()
        if b.is_Number and p.is_Rational:
            return f"R({float(e)!r})"
        if p.is_Integer and 1 < p <= 4:
            s = self._print(b)
            return "(" + "*".join([f"({s})"] * int(p)) + ")"
        return super()._print_Pow(e)


_pr = _Printer()


def ccode(e):
    return _pr.doprint(e)


# --------------------------------------------------------------------- 1D
def gen_1d(lines):
    cs = sp.symbols("a0:8")
    p = sum(c * x**k for k, c in enumerate(cs))
    Wv = sp.symbols("w_m1 w_0 w_p1 w_p2")
    Dv = sp.symbols("d_m1 d_0 d_p1 d_p2")
    eqs = []
    for q, (wq, dq) in zip((-1, 0, 1, 2), zip(Wv, Dv)):
        eqs.append(sp.Eq(cell_avg(p, (q,), 1), wq))
        eqs.append(sp.Eq(cell_avg(sp.diff(p, x), (q,), 1), dq))
    sol = sp.solve(eqs, cs, dict=True)[0]
    P = p.subs(sol)
    val = sp.expand(P.subs(x, half))
    der = sp.expand(sp.diff(P, x).subs(x, half))
    lines.append("/* p^7 of the compact 1D stencil {j-1, j, j+1, j+2} (averages w_*, averaged")
    lines.append(" * derivatives in cell units d_*), at the face x_{j+1/2}: value and")
    lines.append(" * derivative (cell units of cell j).  Sec. 4.2, Eq. 8th-compact-HLP. */")
    lines.append("template <typename R>")
    lines.append("__host__ __device__ __forceinline__ void p7_face(R w_m1, R w_0, R w_p1, R w_p2, R d_m1, R d_0, R d_p1, R d_p2, R &val, R &der)")
    lines.append("{")
    # use the symmetric structure: emit directly
    lines.append(f"    val = {ccode(val)};")
    lines.append(f"    der = {ccode(der)};")
    lines.append("}")
    lines.append("")


# ------------------------------------------------- 1D non-compact (Sec. 4.1)
def _avg_poly(offsets, deg):
    """polynomial of degree deg (cell units, cell j = [-1/2, 1/2]) with the
    given cell averages u_o, o in offsets (deg + 1 of them)"""
    cs = sp.symbols(f"b0:{deg + 1}")
    p = sum(c * x**k for k, c in enumerate(cs))
    us = [sp.Symbol(f"u{o + 2}") for o in offsets]
    sol = sp.solve([sp.Eq(cell_avg(p, (o,), 1), u) for o, u in zip(offsets, us)], cs, dict=True)[0]
    return sp.expand(p.subs(sol))


def _js_indicator(P, deg):
    """sum_(l=1..deg) int_cell (d^l P / dxi^l)^2 (Jiang-Shu, cell units)"""
    r = sp.Integer(0)
    for l in range(1, deg + 1):
        r += sp.integrate(sp.expand(sp.diff(P, x, l) ** 2), (x, -half, half))
    return sp.expand(r)


def gen_noncompact(lines):
    """Left interface value at x_{j+1/2} of the non-compact GENO schemes:
    order 5: high-order p^4 on {j-2..j+2}, quadratics on {j-2,j-1,j},
    {j-1,j,j+1}, {j,j+1,j+2} (the 5th-order WENO stencils);
    order 6: p^5 on {j-2..j+3}, quadratics on {j-2,j-1,j}, {j-1,j,j+1},
    cubics on {j-1..j+2}, {j..j+3}.  Inputs u[i] = average at offset i - 2
    (minus any constant: every polynomial reproduces constants); the right
    value is the same map applied to the mirrored stencil."""
    for order, big, subs in (
        (5, list(range(-2, 3)), [((-2, -1, 0), 2), ((-1, 0, 1), 2), ((0, 1, 2), 2)]),
        (6, list(range(-2, 4)), [((-2, -1, 0), 2), ((-1, 0, 1), 2), ((-1, 0, 1, 2), 3), ((0, 1, 2, 3), 3)]),
    ):
        PH = _avg_poly(big, len(big) - 1)
        exprs = [PH.subs(x, half)]
        names = ["qH"]
        for k, (offs, deg) in enumerate(subs):
            Pk = _avg_poly(list(offs), deg)
            exprs.append(Pk.subs(x, half))
            names.append(f"p[{k}]")
        for k, (offs, deg) in enumerate(subs):
            Pk = _avg_poly(list(offs), deg)
            exprs.append(_js_indicator(Pk, deg))
            names.append(f"IS[{k}]")
        usyms = {sp.Symbol(f"u{i}"): sp.Symbol(f"u[{i}]") for i in range(len(big) + 1)}
        lines.append(f"/* {order}th-order non-compact GENO (Sec. 4.1): left value at x_(j+1/2) of the")
        lines.append(f" * high-order polynomial (qH) and of the {len(subs)} sub-stencil polynomials (p), and")
        lines.append(" * the sub-stencils' Jiang-Shu indicators sum_l int (d^l p)^2 (IS), from the")
        lines.append(" * averages u[i] at offsets i - 2 (cell units). */")
        lines.append("template <typename R>")
        lines.append(f"__host__ __device__ __forceinline__ void nc{order}_left(const R *__restrict__ u, R &qH, R *__restrict__ p, R *__restrict__ IS)")
        lines.append("{")
        emit_assignments(lines, [sp.expand(e).xreplace(usyms) for e in exprs], names)
        lines.append("}")
        lines.append("")


# --------------------------------------------------------------- multi-D
def monomials(m):
    out = []
    for t in range(1, 4):
        for e in itertools.product(range(4), repeat=m):
            if sum(e) == t:
                if m == 3 and e == (1, 1, 1):
                    continue
                out.append(e)
    return out


def mono_expr(e):
    r = sp.Integer(1)
    for a, k in enumerate(e):
        r *= X[a] ** k
    return r


def gen_md(lines, m):
    mons = monomials(m)
    nc = len(mons)
    zero = (0,) * m
    phi = [sp.expand(mono_expr(e) - cell_avg(mono_expr(e), zero, m)) for e in mons]
    # data layout: for q = 2e + (s > 0): dW_q, D_q[0..m-1]; then D_0[0..m-1]
    nd = 2 * m * (1 + m) + m
    A = []
    for e in range(m):
        for s in (-1, 1):
            off = [0] * m
            off[e] = s
            A.append([cell_avg(ph, off, m) for ph in phi])
            for a in range(m):
                A.append([cell_avg(sp.diff(ph, X[a]), off, m) for ph in phi])
    for a in range(m):
        A.append([cell_avg(sp.diff(ph, X[a]), zero, m) for ph in phi])
    A = sp.Matrix(A)
    assert A.shape == (nd, nc)
    N = A.T * A
    assert N.rank() == nc, "least-squares system is rank deficient"
    Minv = N.inv() * A.T  # nc x nd
    d = sp.symbols(f"d0:{nd}")
    c_exprs = [sp.expand(sum(Minv[k, j] * d[j] for j in range(nd))) for k in range(nc)]

    lines.append(f"/* {m}D compact cubic: c = M d, least squares (unit weights, cell units) with")
    lines.append(" * the own average exact.  d[q*(1+m)] = W_q - W_0 and d[q*(1+m)+1+a] = h dW/dx_a")
    lines.append(" * of face neighbour q = 2 e + (side > 0); d[2m(1+m)+a] = own h dW/dx_a.")
    lines.append(" * Monomials (coefficient order): " + ", ".join("x^%d y^%d z^%d" % (tuple(e) + (0,) * (3 - m)) for e in mons) + " */")
    lines.append("template <typename R>")
    lines.append(f"__host__ __device__ __forceinline__ void cubic{m}d_fit(const R *__restrict__ d, R *__restrict__ c)")
    lines.append("{")
    dsyms = {d[j]: sp.Symbol(f"d[{j}]") for j in range(nd)}
    emit_linear(lines, [ce.xreplace(dsyms) for ce in c_exprs], [f"c[{k}]" for k in range(nc)],
                [dsyms[d[j]] for j in range(nd)])
    lines.append("}")
    lines.append("")

    # smoothness indicators: quadratic forms in c
    cs = sp.symbols(f"c0:{nc}")
    P = sum(ck * ph for ck, ph in zip(cs, phi))
    ISH = sp.Integer(0)
    IStau = sp.Integer(0)
    for l in itertools.product(range(4), repeat=m):
        t = sum(l)
        if 1 <= t <= 3:
            dP = P
            for a in range(m):
                dP = sp.diff(dP, X[a], l[a]) if l[a] else dP
            v = cell_avg(sp.expand(dP * dP), zero, m)
            ISH += v
            if t == 3:
                IStau += v
    ISH = sp.expand(ISH)
    IStau = sp.expand(IStau)
    csyms = {cs[k]: sp.Symbol(f"c[{k}]") for k in range(nc)}
    lines.append(f"/* IS^H = sum_(1<=|l|<=3) int (D^l P)^2 and IS^tau = its |l| = 3 part (Eq. IS-highorder-1,")
    lines.append(" * Eq. IS-tau: IS^H minus the |l| <= 2 indicator), each multi-index once, cell units. */")
    lines.append("template <typename R>")
    lines.append(f"__host__ __device__ __forceinline__ void cubic{m}d_indicators(const R *__restrict__ c, R &ISH, R &IStau)")
    lines.append("{")
    emit_assignments(lines, [ISH.xreplace(csyms), IStau.xreplace(csyms)], ["ISH", "IStau"])
    lines.append("}")
    lines.append("")

    # Gauss points and evaluation
    g = sp.sqrt(3) / 6  # 1/(2 sqrt 3)
    ng = 2 if m == 2 else 4
    lines.append(f"/* P - W0 and the cell-unit gradient of P at Gauss point gp of the face on side s")
    lines.append(" * (0: minus, 1: plus) of axis d; tangential coordinates -/+ 1/(2 sqrt 3),")
    lines.append(" * gp = a + 2 b with a for the lower tangential axis.  out[0] value,")
    lines.append(" * out[1 + e] d/dxi_e. */")
    for dd in range(m):
        for s in (0, 1):
            tang = [a for a in range(m) if a != dd]
            for gp in range(ng):
                pt = {X[dd]: half if s else -half}
                for ti, a in enumerate(tang):
                    bit = (gp >> ti) & 1
                    pt[X[a]] = g if bit else -g
                exprs = [sp.expand(P.subs(pt))] + [sp.expand(sp.diff(P, X[e]).subs(pt)) for e in range(m)]
                names = [f"out[{k}]" for k in range(1 + m)]
                lines.append("template <typename R>")
                lines.append(f"__host__ __device__ __forceinline__ void cubic{m}d_eval_d{dd}_s{s}_g{gp}(const R *__restrict__ c, R *__restrict__ out)")
                lines.append("{")
                emit_linear(lines, [ex.xreplace(csyms) for ex in exprs], names, [csyms[cs[k]] for k in range(nc)])
                lines.append("}")
                lines.append("")
    if m == 2:
        lines.append("template <typename R, int M, int D, int S> struct CubicEval;")
    for dd in range(m):
        for s in (0, 1):
            cases = " ".join(f"case {gp}: cubic{m}d_eval_d{dd}_s{s}_g{gp}(c, o); break;" for gp in range(ng))
            lines.append(f"template <typename R> struct CubicEval<R, {m}, {dd}, {s}> {{")
            lines.append(f"    __host__ __device__ __forceinline__ static void run(int g, const R *c, R *o) {{ switch (g) {{ {cases} }} }}")
            lines.append("};")
    lines.append("")
    return nc, nd


def main():
    lines = [
        "/* Generated by gen_coeffs.py (exact rational arithmetic).  Do not edit. */",
        "#pragma once",
        "",
    ]
    gen_1d(lines)
    gen_noncompact(lines)
    info = {}
    for m in (2, 3):
        info[m] = gen_md(lines, m)
    lines.insert(3, f"#define GENO_NC2 {info[2][0]}\n#define GENO_ND2 {info[2][1]}\n#define GENO_NC3 {info[3][0]}\n#define GENO_ND3 {info[3][1]}\n")
    with open(os.path.join(HERE, "geno_coeffs.cuh"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

"""The FP32 stage kernel evaluates WENO5-JS (Sec. 2.2's reconstruction, Jiang & Shu 1996) in a rewritten
"triplet" form: every point triplet (L, C, R) gives s = L + R - 2C and u = sqrt(12/13) (L - R) / 2 once, the
three candidate values are C + 13/12 s -/+ 3/4 (L - R) and C + s/12 -/+ (L - R)/4, the smoothness indicators
are scaled by 12/13 (so that beta' = s^2 + (sqrt(12/13) s -/+ u)^2 or s^2 + u^2), the weights carry the linear
weights as 1, 6, 3, and the data are g = F +- alpha U = 2 f+- with epsilon scaled by 4. These CPU tests
restate those steps in exact arithmetic (sympy; the square roots cancel) and check that each face value is
exactly the textbook WENO5 of the split fluxes (times 2), for both upwind directions, for the level set's
one-sided derivatives, and that the branch-free flux (U + c_E p) v_n + c_A p is each flux kind of Eq.
euler2D. The FP32 adjoint's triplet form (per-role gradient shares of a face) is checked the same way against
the exact gradient of the textbook WENO5. FP32 results then differ from the definitions only by rounding."""
import random

import pytest

sp = pytest.importorskip("sympy")

KS = sp.sqrt(sp.Rational(12, 13))
KU = KS / 2
KQ = sp.sqrt(sp.Rational(13, 12)) / 2
EPS_SCALE = sp.Rational(12, 13)


def textbook_weno5(a, b, c, d, e, eps):
    q = [(2 * a - 7 * b + 11 * c) / 6, (-b + 5 * c + 2 * d) / 6, (2 * c + 5 * d - e) / 6]
    beta = [sp.Rational(13, 12) * (a - 2 * b + c) ** 2 + (a - 4 * b + 3 * c) ** 2 / 4,
            sp.Rational(13, 12) * (b - 2 * c + d) ** 2 + (b - d) ** 2 / 4,
            sp.Rational(13, 12) * (c - 2 * d + e) ** 2 + (3 * c - 4 * d + e) ** 2 / 4]
    alpha = [w / (eps + bk) ** 2 for w, bk in zip((sp.Rational(1, 10), sp.Rational(6, 10), sp.Rational(3, 10)), beta)]
    return sum(al * qk for al, qk in zip(alpha, q)) / sum(alpha)


def tri_data(L, C, R, eps_scaled):
    s = L + R - 2 * C
    u = KU * (L - R)
    bs = s * s + eps_scaled
    mm, pp = KS * s - u, KS * s + u
    Dm, Dt, Dp = mm * mm + bs, u * u + bs, pp * pp + bs
    return dict(s=s, u=u, base=C + s / 12, rm=1 / Dm ** 2, rt6=6 / Dt ** 2, rp=1 / Dp ** 2)


def tri_roles(d, left_to_right):
    lo, hi = d["base"] - KQ * d["u"], d["base"] + KQ * d["u"]
    bss = d["base"] + d["s"]
    if left_to_right:
        return dict(up=(bss - 3 * KQ * d["u"], d["rm"]), mid=(lo, d["rt6"]), down=(hi, 3 * d["rp"]))
    return dict(up=(bss + 3 * KQ * d["u"], d["rp"]), mid=(hi, d["rt6"]), down=(lo, 3 * d["rm"]))


def tri_face(a, b, c):
    return (a[1] * a[0] + b[1] * b[0] + c[1] * c[0]) / (a[1] + b[1] + c[1])


def _rationals(rnd, n, lo=-30, hi=30):
    return [sp.Rational(rnd.randint(lo * 64, hi * 64), rnd.randint(1, 64)) for _ in range(n)]


@pytest.mark.parametrize("seed", range(6))
def test_hydro_line_faces_are_the_textbook_weno5_of_the_split_fluxes(seed):
    rnd = random.Random(seed)
    K = 2
    U = _rationals(rnd, K + 6)
    F = _rationals(rnd, K + 6)
    alpha = sp.Rational(rnd.randint(1, 200), 7)
    eps = sp.Rational(1, 10 ** 6) if seed % 2 else sp.Rational(rnd.randint(1, 50), 3)  # a large eps too
    gp = [Fm + alpha * Um for Fm, Um in zip(F, U)]
    gm = [Fm - alpha * Um for Fm, Um in zip(F, U)]
    fp = [g / 2 for g in gp]
    fm = [g / 2 for g in gm]
    tp = {j: tri_roles(tri_data(gp[j - 1], gp[j], gp[j + 1], 4 * eps * EPS_SCALE), True) for j in range(1, K + 4)}
    tm = {j: tri_roles(tri_data(gm[j - 1], gm[j], gm[j + 1], 4 * eps * EPS_SCALE), False) for j in range(2, K + 5)}
    for f in range(K + 1):
        plus = tri_face(tp[f + 1]["up"], tp[f + 2]["mid"], tp[f + 3]["down"])
        minus = tri_face(tm[f + 4]["up"], tm[f + 3]["mid"], tm[f + 2]["down"])
        assert sp.simplify(plus - 2 * textbook_weno5(*fp[f:f + 5], eps)) == 0
        assert sp.simplify(minus - 2 * textbook_weno5(*fm[f + 1:f + 6][::-1], eps)) == 0


@pytest.mark.parametrize("seed", range(4))
def test_level_set_one_sided_derivatives(seed):
    rnd = random.Random(100 + seed)
    K = 2
    d = _rationals(rnd, K + 5)
    eps = sp.Rational(1, 10 ** 6)
    td = {j: tri_data(d[j - 1], d[j], d[j + 1], eps * EPS_SCALE) for j in range(1, K + 4)}
    tl = {j: tri_roles(t, True) for j, t in td.items()}
    tr = {j: tri_roles(t, False) for j, t in td.items()}
    for k in range(K):
        om = tri_face(tl[k + 1]["up"], tl[k + 2]["mid"], tl[k + 3]["down"])
        op = tri_face(tr[k + 4]["up"], tr[k + 3]["mid"], tr[k + 2]["down"])
        assert sp.simplify(om - textbook_weno5(*d[k:k + 5], eps)) == 0
        assert sp.simplify(op - textbook_weno5(*d[k + 1:k + 6][::-1], eps)) == 0


def test_branch_free_flux_is_each_flux_kind():
    rho, mn, mt, E, p, vn = sp.symbols("rho m_n m_t E p v_n")
    want = {0: rho * vn, 1: mn * vn + p, 2: mt * vn, 3: (E + p) * vn}
    conserved = {0: rho, 1: mn, 2: mt, 3: E}
    for kind, w in want.items():
        cE, cA = (1 if kind == 3 else 0), (1 if kind == 1 else 0)
        assert sp.expand((conserved[kind] + cE * p) * vn + cA * p - w) == 0


def test_candidate_values_and_scaled_indicators():
    """The closed forms the triplet form rests on, symbolically: the three candidates from (s, L - R) and
    12/13 of each indicator as s^2 plus a square of (sqrt(12/13) s -/+ u) or u."""
    a, b, c, d, e = sp.symbols("a b c d e")
    s0, t0 = a + c - 2 * b, a - c
    assert sp.expand(b + sp.Rational(13, 12) * s0 - sp.Rational(3, 4) * t0 - (2 * a - 7 * b + 11 * c) / 6) == 0
    s1, t1 = b + d - 2 * c, b - d
    assert sp.expand(c + s1 / 12 - t1 / 4 - (-b + 5 * c + 2 * d) / 6) == 0
    s2, t2 = c + e - 2 * d, c - e
    assert sp.expand(d + s2 / 12 + t2 / 4 - (2 * c + 5 * d - e) / 6) == 0
    for (L, C, R), beta, sign in (((a, b, c), sp.Rational(13, 12) * s0 ** 2 + (a - 4 * b + 3 * c) ** 2 / 4, -1),
                                  ((b, c, d), sp.Rational(13, 12) * s1 ** 2 + (b - d) ** 2 / 4, 0),
                                  ((c, d, e), sp.Rational(13, 12) * s2 ** 2 + (3 * c - 4 * d + e) ** 2 / 4, 1)):
        s, u = L + R - 2 * C, KU * (L - R)
        other = u if sign == 0 else KS * s + sign * u
        assert sp.expand(EPS_SCALE * beta - (s ** 2 + other ** 2)) == 0


# ---- the FP32 adjoint's triplet form: per role of a face, gbar dW/d(a', b', c') = WG dq_r + A (1, -2, 1) +
# B dt_r with WG = gbar a_r / sum a, cg = -2 gbar (q_r - W) (a_r / D_r) / sum a, A = 13/6 s cg, B = h_r cg
# (indicators unscaled, eps = 1e-6 on the split fluxes themselves), where q_r - W is formed from the
# triplets' second differences: w_r = a_r / sum a, D01 = (s_up - s_mid) / 3, D12 = (s_dn - s_mid) / 6,
# D02 = D01 + D12, q_up - W = w_mid D01 + w_dn D02, q_mid - W = w_dn D12 - w_up D01,
# q_dn - W = -(w_up D02 + w_mid D12).
ADJ_DQ = ((sp.Rational(2, 6), sp.Rational(-7, 6), sp.Rational(11, 6)),
          (sp.Rational(-1, 6), sp.Rational(5, 6), sp.Rational(2, 6)),
          (sp.Rational(2, 6), sp.Rational(5, 6), sp.Rational(-1, 6)))
ADJ_DT = ((1, -4, 3), (1, 0, -1), (3, -4, 1))
ADJ_EPS = sp.Rational(1, 10 ** 6)


def adj_tri(L, C, R, left_to_right):
    s, th = L + R - 2 * C, (L - R) / 2
    bs = sp.Rational(13, 12) * s * s + ADJ_EPS
    mm, pp = s - th, s + th
    rm, rt, rp = 1 / (mm * mm + bs), 1 / (th * th + bs), 1 / (pp * pp + bs)
    base = C + s / 12
    bss, lo, hi, at = base + s, base - th / 2, base + th / 2, 6 * rt * rt
    if left_to_right:
        roles = [(bss - 3 * th / 2, rm * rm, rm * rm * rm, mm), (lo, at, at * rt, th), (hi, 3 * rp * rp, 3 * rp ** 3, pp)]
    else:
        roles = [(bss + 3 * th / 2, rp * rp, rp ** 3, pp), (hi, at, at * rt, -th), (lo, 3 * rm * rm, 3 * rm ** 3, mm)]
    return roles, sp.Rational(13, 6) * s


def adj_face(roles, gbar):
    """roles: three (role tuple, s13, points in reconstruction order); returns {point: gradient share}, W."""
    sa = sum(r[1] for r, _, _ in roles)
    W = sum(r[1] * r[0] for r, _, _ in roles) / sa
    g, m2g = gbar / sa, -2 * gbar / sa
    w = [r[1] / sa for r, _, _ in roles]
    su13, sm13, sd13 = (s13 for _, s13, _ in roles)
    d01, d12 = (su13 - sm13) * sp.Rational(2, 13), (sd13 - sm13) * sp.Rational(1, 13)
    d02 = d01 + d12
    qmw = (w[1] * d01 + w[2] * d02, w[2] * d12 - w[0] * d01, -(w[0] * d02 + w[1] * d12))
    out = {}
    for k, ((q, a, nr, h), s13, pts) in enumerate(roles):
        assert sp.simplify(qmw[k] - (q - W)) == 0  # the candidate-difference identity
        WG, cg = a * g, qmw[k] * nr * m2g
        A, B = s13 * cg, h * cg
        for j, (pt, dq, dt, da) in enumerate(zip(pts, ADJ_DQ[k], ADJ_DT[k], (1, -2, 1))):
            out[pt] = out.get(pt, 0) + WG * dq + B * dt + A * da
    return out, W


@pytest.mark.parametrize("seed", range(4))
def test_adjoint_triplet_gradient_is_the_textbook_gradient(seed):
    rnd = random.Random(200 + seed)
    p = _rationals(rnd, 7, -8, 8)
    gbar = sp.Rational(rnd.randint(-99, 99), 13)
    x = sp.symbols("x0:5")
    Wsym = textbook_weno5(*x, ADJ_EPS)
    grad = [sp.diff(Wsym, xi) for xi in x]
    q = 3
    # left-biased face: triplets centred at q-2, q-1, q (roles up, mid, dn), stencil points q-3 .. q+1
    t = {j: adj_tri(p[j - 1], p[j], p[j + 1], True) for j in (q - 2, q - 1, q)}
    share, W = adj_face([(t[q - 2][0][0], t[q - 2][1], (q - 3, q - 2, q - 1)),
                         (t[q - 1][0][1], t[q - 1][1], (q - 2, q - 1, q)),
                         (t[q][0][2], t[q][1], (q - 1, q, q + 1))], gbar)
    pts = list(range(q - 3, q + 2))
    sub = dict(zip(x, [p[i] for i in pts]))
    assert sp.simplify(W - Wsym.subs(sub)) == 0
    for xi, i in zip(range(5), pts):
        assert sp.simplify(share[i] - gbar * grad[xi].subs(sub)) == 0
    # right-biased face: triplets centred at q+1, q, q-1, stencil q+2 .. q-2 in reconstruction order
    t = {j: adj_tri(p[j - 1], p[j], p[j + 1], False) for j in (q + 1, q, q - 1)}
    share, W = adj_face([(t[q + 1][0][0], t[q + 1][1], (q + 2, q + 1, q)),
                         (t[q][0][1], t[q][1], (q + 1, q, q - 1)),
                         (t[q - 1][0][2], t[q - 1][1], (q, q - 1, q - 2))], gbar)
    pts = list(range(q + 2, q - 3, -1))
    sub = dict(zip(x, [p[i] for i in pts]))
    assert sp.simplify(W - Wsym.subs(sub)) == 0
    for xi, i in zip(range(5), pts):
        assert sp.simplify(share[i] - gbar * grad[xi].subs(sub)) == 0

"""The fixed-point sums of the step kernels (csrc/fixsum.cuh: the density moments
of Eqs. Density and Momentum, the Shan-Chen stencil of Eq. ShanChenForce), built
for the host from the same source, against exact rational sums of the same
doubles (fractions.Fraction). The bound: within half an ulp of the result plus,
for each operand, 2^-7 of the largest operand's ulp (the bits a smaller operand
loses below the frame); sums of positive operands within 0.57 ulp; exact results
(representable sums, exact cancellation) reproduced exactly."""
import math
from fractions import Fraction

import numpy as np
import pytest


@pytest.fixture(scope="module")
def fx(fixsum_host):
    return fixsum_host


def density(lib, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((f.shape[0], 6))
    lib.fx_density(f.shape[0], f.ctypes.data, out.ctypes.data)
    return out


def stencil(lib, p):
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros((p.shape[0], 2))
    lib.fx_stencil(p.shape[0], p.ctypes.data, out.ctypes.data)
    return out


def ulp(x):
    return math.ulp(abs(float(x))) if x != 0 else math.ulp(0.0)


def check(res, exact, operands, nterms, what):
    """|res - exact| <= ulp(res)/2 + nterms 2^-7 ulp(max operand)."""
    big = max(abs(float(v)) for v in operands)
    bound = Fraction(ulp(res)) / 2 + nterms * Fraction(ulp(big)) / 128
    if exact != 0 and res != 0:
        # the rounding's half ulp is of the exact value's binade: take the larger
        bound = max(bound, Fraction(ulp(float(exact))) / 2 + nterms * Fraction(ulp(big)) / 128)
    err = abs(Fraction(float(res)) - exact)
    assert err <= bound, (what, float(res), float(exact), float(err / Fraction(ulp(big))))


def population_sets(rng, n, spread):
    """Nine populations per node: f_eq-like weights times a density in 10^[-6, 0] with
    relative perturbations up to `spread` (an interface node), or independent exponents."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    rho = 10.0 ** rng.uniform(-6, 0, size=(n, 1))
    f = w * rho * (1 + spread * rng.uniform(-1, 1, size=(n, 9)))
    return f


@pytest.mark.parametrize("spread", [0.0, 1e-12, 1e-3, 0.5, 0.99])
def test_density_moments_within_the_bound_of_the_exact_sums(fx, spread):
    rng = np.random.default_rng(20260 + int(spread * 1000))
    f = population_sets(rng, 3000, spread)
    out = density(fx, f)
    assert np.all(out[:, 5] == 1.0)
    for i in range(f.shape[0]):
        q = [Fraction(float(v)) for v in f[i]]
        rho = sum(q)
        jx = q[1] + q[5] + q[8] - q[3] - q[6] - q[7]
        jy = q[2] + q[5] + q[6] - q[4] - q[7] - q[8]
        m7 = (q[1] + q[3]) - (q[2] + q[4])
        m8 = (q[5] + q[7]) - (q[6] + q[8])
        # rho: a sum of positive operands, within 0.57 ulp of itself
        assert abs(Fraction(float(out[i, 0])) - rho) <= Fraction(ulp(out[i, 0])) * Fraction(57, 100), i
        check(out[i, 1], jx, f[i], 6, "jx")
        check(out[i, 2], jy, f[i], 6, "jy")
        check(out[i, 3], m7, f[i], 4, "m7")
        check(out[i, 4], m8, f[i], 4, "m8")


def test_density_moments_independent_exponents_and_exact_cases(fx):
    rng = np.random.default_rng(7)
    # independent magnitudes over 2^-60 .. 2^20: terms far below the largest vanish into
    # the frame's low bits, the bound still holds
    f = np.ldexp(1 + rng.random((4000, 9)), rng.integers(-60, 21, size=(4000, 9)))
    out = density(fx, f)
    for i in range(f.shape[0]):
        q = [Fraction(float(v)) for v in f[i]]
        check(out[i, 0], sum(q), f[i], 9, "rho")
        check(out[i, 1], q[1] + q[5] + q[8] - q[3] - q[6] - q[7], f[i], 6, "jx")
    # exactly representable sums come out exact; a state at rest has j = 0 exactly
    g = np.array([[4.0, 1.0, 1.0, 1.0, 1.0, 0.25, 0.25, 0.25, 0.25]]) * 2.0 ** -10
    o = density(fx, g)[0]
    assert o[0] == 9.0 * 2.0 ** -10 and o[1] == 0.0 and o[2] == 0.0 and o[3] == 0.0 and o[4] == 0.0
    assert not math.copysign(1.0, o[1]) < 0  # +0, as an IEEE x - x
    # mirror-symmetric populations (f1 = f3, f5 = f6, f8 = f7) cancel exactly in jx
    h = population_sets(np.random.default_rng(3), 200, 0.3)
    h[:, 3], h[:, 6], h[:, 7] = h[:, 1], h[:, 5], h[:, 8]
    assert np.all(density(fx, h)[:, 1] == 0.0)
    # ties: with the others multiples of 2^-40, + 2^-53 is exactly half an ulp and
    # rounds to even, + 3 2^-53 rounds up to the even neighbour
    t = np.full((2, 9), 2.0 ** -40)
    t[:, 0] = 1.0
    t[0, 1], t[1, 1] = 2.0 ** -53, 3 * 2.0 ** -53
    o = density(fx, t)
    assert o[0, 0] == 1.0 + 7 * 2.0 ** -40 and o[1, 0] == 1.0 + 7 * 2.0 ** -40 + 2.0 ** -51
    # an operand far below the others still counts as a sticky unit: above the tie
    t[0, 8] = 2.0 ** -300
    assert density(fx, t)[0, 0] == 1.0 + 6 * 2.0 ** -40 + 2.0 ** -52


def test_density_range_check_rejects_what_the_frame_cannot_hold(fx):
    base = np.full((1, 9), 0.1)
    for bad in (0.0, -0.1, 5e-324, 1e-310, 2.0 ** 1008, np.inf, np.nan):
        f = base.copy()
        f[0, 4] = bad
        assert density(fx, f)[0, 5] == 0.0, bad
    assert density(fx, base)[0, 5] == 1.0


@pytest.mark.parametrize("ratio", [1.0, 0.9, 1e-2, 1e-5])
def test_shan_chen_stencil_within_the_bound_of_the_exact_sums(fx, ratio):
    """psi over a 3 x 3 stencil: smooth fields, and interfaces where psi drops by
    `ratio` (liquid to vapour) across the stencil."""
    rng = np.random.default_rng(int(1 / ratio) % 100003)
    n = 4000
    psi_l = 10.0 ** rng.uniform(-3, 1, size=(n, 1))
    frac = rng.random((n, 8))
    p = psi_l * (ratio + (1 - ratio) * frac)
    out = stencil(fx, p)
    for i in range(n):
        q = [Fraction(float(v)) for v in p[i]]
        E_, W, N, S, NE, NW, SW, SE = q
        gx = 4 * (E_ - W) + (NE - SW) + (SE - NW)
        gy = 4 * (N - S) + (NE - SW) - (SE - NW)
        check(out[i, 0], gx, p[i], 12, "gx")
        check(out[i, 1], gy, p[i], 12, "gy")


def test_shan_chen_stencil_uniform_and_symmetric_fields_give_zero(fx):
    p = np.full((3, 8), 0.37)
    p[1] *= 1e-4
    p[2] = [0.5, 0.5, 0.2, 0.2, 0.3, 0.3, 0.3, 0.3]   # E = W, N = S, NE = NW = SW = SE
    out = stencil(fx, p)
    assert np.all(out == 0.0) and not np.any(np.signbit(out))
    # antisymmetry: swapping east and west (and the diagonals) negates gx exactly
    rng = np.random.default_rng(11)
    a = rng.uniform(0.01, 1.0, size=(500, 8))
    b = a[:, [1, 0, 2, 3, 5, 4, 7, 6]]   # E<->W, NE<->NW, SW<->SE
    oa, ob = stencil(fx, a), stencil(fx, b)
    assert np.array_equal(oa[:, 0], -ob[:, 0]) and np.array_equal(oa[:, 1], ob[:, 1])


def test_shan_chen_stencil_non_finite_or_negative_psi_gives_nan(fx):
    for bad in (np.inf, np.nan, -0.2):
        p = np.full((1, 8), 0.3)
        p[0, 5] = bad
        assert np.all(np.isnan(stencil(fx, p)))
    # a zero psi counts as (at most) one unit of the frame's last bit
    p = np.full((1, 8), 0.3)
    p[0, 1] = 0.0
    out = stencil(fx, p)[0]
    assert abs(out[0] - 4 * 0.3) <= 2 * math.ulp(1.2) and abs(out[1]) <= math.ulp(0.3)


def j_h(lib, a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros((a.shape[0], 4))
    lib.fx_j_h(a.shape[0], a.ctypes.data, out.ctypes.data)
    return out


def populations(lib, q, shear):
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros((q.shape[0], 9))
    lib.fx_populations(q.shape[0], 1 if shear else 0, q.ctypes.data, out.ctypes.data)
    return out


def frame_bound(res, exact, operands, coef_sum, headroom):
    """Half an ulp of the result plus half a frame unit per unit of coefficient (each
    operand is rounded to its nearest frame unit), plus one unit of slack; a frame unit
    is 2^-(11 - headroom) of the largest operand's ulp."""
    big = max(abs(float(v)) for v in operands)
    unit = Fraction(ulp(big)) / 2 ** (11 - headroom)
    half = Fraction(ulp(float(res))) / 2
    if exact != 0:
        half = max(half, Fraction(ulp(float(exact))) / 2)
    return half + (Fraction(coef_sum, 2) + 1) * unit


def test_j_h_combinations_within_the_bound(fx):
    rng = np.random.default_rng(5)
    n = 4000
    j = rng.normal(size=n) * 10.0 ** rng.uniform(-8, 0, size=n)
    h = rng.normal(size=n) * 10.0 ** rng.uniform(-8, 0, size=n)
    j[:50] = 0.0
    h[50:100] = -0.0
    out = j_h(fx, np.stack([j, h], axis=1))
    for i in range(n):
        J, H = Fraction(float(j[i])), Fraction(float(h[i]))
        for k, (ex, cs) in enumerate(((J + H, 2), (J + 2 * H, 3), (J + 3 * H, 4), (J - H, 2))):
            err = abs(Fraction(float(out[i, k])) - ex)
            assert err <= frame_bound(out[i, k], ex, (j[i], h[i]), cs, 4), (i, k)
    # exact cases: zero operands, and a state at rest
    assert np.array_equal(out[:50, 0], h[:50]) and np.array_equal(out[50:100, 0], j[50:100])
    assert np.array_equal(out[:50, 2], 3 * h[:50])


W = [Fraction(4, 9)] + [Fraction(1, 9)] * 4 + [Fraction(1, 36)] * 4
CX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
CY = [0, 0, 1, 0, -1, 1, 1, -1, -1]


def populations_by_definition(q, shear):
    """f*_i = w_i [rho + 3 c_i.P + 4.5 (c_i c_i - I/3) : Pi*] + zz (-8, 1, ..., 1), from the
    unscaled quantities rho = 36 r, P = 36 p, Pi = 36 (xx, yy, xy); with the rows 7, 8
    corrections Pi*_xx = Pi_xx + 18 p7 36 / 36, i.e. Pi*_xx - Pi*_yy = Pi_xx - Pi_yy + 36 p7
    and Pi*_xy = Pi_xy + 36 p8 (the trace relaxes with unit rate)."""
    r, xx, yy, xy, px, py, zz, p7, p8 = [Fraction(float(v)) for v in q]
    if not shear:
        p7 = p8 = Fraction(0)
    rho, Px, Py = 36 * r, 36 * px, 36 * py
    Pxx, Pyy, Pxy = 36 * xx + 18 * p7, 36 * yy - 18 * p7, 36 * (xy + p8)
    f = []
    for i in range(9):
        cx, cy = CX[i], CY[i]
        quad = (cx * cx - Fraction(1, 3)) * Pxx + (cy * cy - Fraction(1, 3)) * Pyy + 2 * cx * cy * Pxy
        z = -8 * zz if i == 0 else zz
        f.append(W[i] * (rho + 3 * (cx * Px + cy * Py) + Fraction(9, 2) * quad) + z)
    return f


COEF_SUM = [72, 44, 44, 44, 44, 32, 32, 32, 32]


@pytest.mark.parametrize("shear", [False, True])
@pytest.mark.parametrize("regime", ["bulk", "interface", "li_dominant"])
def test_reduced_populations_equal_the_collision_definition(fx, shear, regime):
    """The fixed-point output stage against the populations' definition (not against its
    own coefficient table): bulk nodes (second moments and forcing small against rho),
    interface nodes (all of similar size) and vapour nodes beside an interface where the
    Li term exceeds rho."""
    rng = np.random.default_rng({"bulk": 1, "interface": 2, "li_dominant": 3}[regime] + 10 * shear)
    n = 2500
    rho = 10.0 ** rng.uniform(-5, 0, size=n)
    scale = {"bulk": 1e-4, "interface": 0.3, "li_dominant": 1.0}[regime]
    q = np.empty((n, 9))
    q[:, 0] = rho / 36
    for k in range(1, 9):
        q[:, k] = rng.normal(size=n) * rho * scale / 36
    if regime == "li_dominant":
        q[:, 6] = rho * 10.0 ** rng.uniform(1, 4, size=n)
    out = populations(fx, q, shear)
    for i in range(n):
        ref = populations_by_definition(q[i], shear)
        ops = q[i] if shear else q[i, :7]
        for k in range(9):
            assert abs(Fraction(float(out[i, k])) - ref[k]) <= frame_bound(out[i, k], ref[k], ops, COEF_SUM[k], 7), \
                (i, k, float(out[i, k]), float(ref[k]))


def test_reduced_populations_conserve_mass_and_keep_rest_exact(fx):
    rng = np.random.default_rng(9)
    # a node at rest with no force: the equilibrium weights times rho, exactly
    r = 10.0 ** rng.uniform(-5, 0, size=200) / 36
    q = np.zeros((200, 9))
    q[:, 0] = r
    out = populations(fx, q, False)
    w = np.array([16, 4, 4, 4, 4, 1, 1, 1, 1], dtype=float)
    assert np.array_equal(out, w * r[:, None])
    # a mirror-symmetric node (P_x = 0, Pi_xy = 0) gives f1 = f3, f5 = f6, f7 = f8 exactly
    q = rng.normal(size=(300, 9)) * 1e-3
    q[:, 0] = np.abs(q[:, 0]) + 0.01
    q[:, 3] = q[:, 4] = q[:, 8] = 0.0
    out = populations(fx, q, True)
    assert np.array_equal(out[:, 1], out[:, 3]) and np.array_equal(out[:, 5], out[:, 6])
    assert np.array_equal(out[:, 7], out[:, 8])
    # the sum of the nine populations is rho = 36 r to within the nine roundings
    q = np.abs(rng.normal(size=(500, 9))) * 1e-2
    q[:, 0] = 0.1 + q[:, 0]
    out = populations(fx, q, True)
    for i in range(500):
        tot = sum(Fraction(float(v)) for v in out[i])
        assert abs(tot - 36 * Fraction(float(q[i, 0]))) <= 12 * Fraction(ulp(36 * q[i, 0]))


def test_reduced_populations_non_finite_input_gives_nan(fx):
    q = np.full((3, 9), 0.01)
    q[0, 6], q[1, 2], q[2, 8] = np.inf, np.nan, np.inf
    assert np.all(np.isnan(populations(fx, q, True)))


def populations_transpose(lib, mu, shear):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    out = np.zeros((mu.shape[0], 9))
    lib.fx_populations_transpose(mu.shape[0], 1 if shear else 0, mu.ctypes.data, out.ctypes.data)
    return out


def _unit(k):
    q = np.zeros(9)
    q[k] = 1.0
    return q


@pytest.mark.parametrize("shear", [False, True])
def test_populations_transpose_is_the_adjoint_of_the_definition(fx, shear):
    """The reverse-mode stage against the derivative of the populations' definition:
    out_k = sum_i mu_i df_i/dq_k, with df_i/dq_k = f_i(e_k) (f is linear in the
    scaled inputs), in exact rational arithmetic, within the frame's bound."""
    jac = [populations_by_definition(_unit(k), shear) for k in range(9)]  # jac[k][i]
    rng = np.random.default_rng(77 + shear)
    n = 2000
    mu = rng.normal(size=(n, 9)) * 10.0 ** rng.uniform(-6, 2, size=(n, 1))
    mu[:200] *= 10.0 ** rng.uniform(-3, 0, size=(200, 9))   # adjoints of unequal size
    mu[200:220, 4] = 0.0
    out = populations_transpose(fx, mu, shear)
    coef = [36, 72, 72, 36, 36, 36, 16, 36, 36]
    for i in range(n):
        m = [Fraction(float(v)) for v in mu[i]]
        for k in range(9 if shear else 7):
            ex = sum(m[j] * jac[k][j] for j in range(9))
            assert abs(Fraction(float(out[i, k])) - ex) <= frame_bound(out[i, k], ex, mu[i], coef[k], 8), (i, k)
    if not shear:
        assert np.all(out[:, 7:] == 0.0)


def test_populations_transpose_exact_cases(fx):
    # equal adjoints on every population: d(sum f)/d(rho/36) = 36, the rest cancels
    out = populations_transpose(fx, np.full((1, 9), 0.5), True)[0]
    assert out[0] == 18.0 and np.all(out[1:6] == [0.0, 0.0, 0.0, 0.0, 0.0]) and out[6] == 0.0
    assert out[7] == 0.0 and out[8] == 0.0
    q = np.full((2, 9), 0.1)
    q[1, 3] = np.nan
    assert np.all(np.isnan(populations_transpose(fx, q, True)[1]))


def test_j_h_transpose_within_the_bound(fx):
    rng = np.random.default_rng(31)
    n = 3000
    a = rng.normal(size=(n, 6)) * 10.0 ** rng.uniform(-8, 1, size=(n, 6))
    a[:100, 3] = 0.0
    a[100:200, 4] = 0.0
    out = np.zeros((n, 2))
    fx.fx_j_h_transpose(n, np.ascontiguousarray(a).ctypes.data, out.ctypes.data)
    for i in range(n):
        a1, a2, a3, a4, j0, h0 = [Fraction(float(v)) for v in a[i]]
        jb, hb = j0 + a1 + a2 + a3 + a4, h0 + a1 + 2 * a2 + 3 * a3 - a4
        assert abs(Fraction(float(out[i, 0])) - jb) <= frame_bound(out[i, 0], jb, a[i], 5, 5)
        assert abs(Fraction(float(out[i, 1])) - hb) <= frame_bound(out[i, 1], hb, a[i], 8, 5)


def test_psi_adjoint_gather_is_the_stencil_transpose(fx):
    """psi_bar(y) = own + sum_c W_c (c_x gx_bar(y - c) + c_y gy_bar(y - c)) with W = 4 on the
    axes and 1 on the diagonals: the value each neighbour y - c's stencil took from y,
    written out from the stencil's definition (gx = 4 (pE - pW) + ..., so node y enters
    the gx of its west neighbour with +4 and of its east neighbour with -4, etc.)."""
    rng = np.random.default_rng(41)
    n = 3000
    v = rng.normal(size=(n, 13)) * 10.0 ** rng.uniform(-6, 1, size=(n, 13))
    v[:50, 0] = 0.0
    out = np.zeros(n)
    fx.fx_psi_gather(n, np.ascontiguousarray(v).ctypes.data, out.ctypes.data)
    # neighbour offsets of the inputs (order: own, sxW, sxE, syS, syN, sxSW, sySW, sxNE,
    # syNE, sxNW, syNW, sxSE, sySE) and the stencil weight of node y in that neighbour's
    # g: for a neighbour at y - c the node sits at +c, with weight W_c c
    W = {(1, 0): 4, (-1, 0): 4, (0, 1): 4, (0, -1): 4, (1, 1): 1, (-1, -1): 1, (1, -1): 1, (-1, 1): 1}
    nb = [("x", (-1, 0)), ("x", (1, 0)), ("y", (0, -1)), ("y", (0, 1)), ("x", (-1, -1)), ("y", (-1, -1)),
          ("x", (1, 1)), ("y", (1, 1)), ("x", (-1, 1)), ("y", (-1, 1)), ("x", (1, -1)), ("y", (1, -1))]
    for i in range(n):
        q = [Fraction(float(t)) for t in v[i]]
        ex = q[0]
        for k, (comp, (dx, dy)) in enumerate(nb):
            cx, cy = -dx, -dy   # node y is at +c from the neighbour at y - c
            w = W[(cx, cy)] * (cx if comp == "x" else cy)
            ex += w * q[k + 1]
        assert abs(Fraction(float(out[i])) - ex) <= frame_bound(out[i], ex, v[i], 25, 6), i


@pytest.mark.parametrize("shear", [False, True])
def test_lambda_assembly_matches_the_moment_rows(fx, shear):
    """lambda_i = rho_bar + c_i . j_bar (+ M7_i m7_bar + M8_i m8_bar with rows 7, 8 of the
    MRT matrix restricted to the populations, (c_x^2 - c_y^2) and c_x c_y), exact."""
    rng = np.random.default_rng(43 + shear)
    n = 3000
    v = rng.normal(size=(n, 5)) * 10.0 ** rng.uniform(-6, 1, size=(n, 5))
    out = np.zeros((n, 9))
    fx.fx_lambda(n, 1 if shear else 0, np.ascontiguousarray(v).ctypes.data, out.ctypes.data)
    assert np.array_equal(out[:, 0], v[:, 0])
    for i in range(n):
        r, jx, jy, m7, m8 = [Fraction(float(t)) for t in v[i]]
        for k in range(1, 9):
            cx, cy = CX[k], CY[k]
            ex = r + cx * jx + cy * jy
            if shear:
                ex += (cx * cx - cy * cy) * m7 + cx * cy * m8
            ops = v[i] if shear else v[i, :3]
            assert abs(Fraction(float(out[i, k])) - ex) <= frame_bound(out[i, k], ex, ops, 4, 4), (i, k)


def test_operands_beyond_the_frame_range_give_nan(fx):
    """Every frame takes operands below 2^1008 (below it no rounded result can overflow
    the exponent); an operand at or above it gives NaN, as a non-finite one does."""
    big = 2.0 ** 1008
    assert np.all(np.isnan(j_h(fx, np.array([[1.0, big], [big, 0.5], [np.inf, 1.0]]))))
    assert np.all(np.isfinite(j_h(fx, np.array([[1.0, 2.0 ** 1007]]))))
    q = np.full((2, 9), 0.01)
    q[0, 6] = big
    out = populations(fx, q, True)
    assert np.all(np.isnan(out[0])) and np.all(np.isfinite(out[1]))
    p = np.full((1, 8), 0.3)
    p[0, 2] = big
    assert np.all(np.isnan(stencil(fx, p)))
    mu = np.full((1, 9), 0.2)
    mu[0, 5] = -big
    assert np.all(np.isnan(populations_transpose(fx, mu, True)[0, :9]))

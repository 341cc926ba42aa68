"""Pins of the oracle's drag laws as the push evaluates them (CPU only).

The table law (Sec. 2.2, Eq. contdrag and Eq. scatteringNdot tabulated over
(log10 gamma, s/L), read by bilinear interpolation) and the closed form for
radial photons (Eq. contdrag) each return F^, its derivative in u (the
Newton derivative of the implicit midpoint of Sec. 3) and ln N^.  These
tests tie that lookup to things other than its own formula:

* a table filled with a function that is bilinear in (log10 gamma, s/L) is
  reproduced exactly between nodes, for each sign row and either s end;
* at table nodes the lookup returns the stored quadrature value;
* between nodes of a table of the radial closed form, the lookup is within
  the bilinear interpolation bound (from the table's second differences) of
  the closed form at the same point;
* the derivatives equal central differences of F, and the table's is zero
  where gamma is clamped at the top of the table.

A swapped sign row, an s index off by a row (s/L mapped onto ns instead of
ns - 1 intervals), transposed table axes or a wrong d(log10 gamma)/du each
fail one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_17661_b300 import workloads as W

NG, NS, GMAX = 16, 8, 8.0


def _u_of(log10g, sign):
    g = 10.0 ** log10g
    return sign * math.sqrt(max(g * g - 1.0, 0.0))


def _k_code(S):
    """drag_scale / R_cells: F^ per R_star -> du per cell-crossing time."""
    return S.cfg["drag_scale"] / S.scalars()["R_cells"]


def _coeffs():
    # F = a + b lg + c sf + d lg sf per sign row (lg = log10 gamma, sf = s/L);
    # distinct rows, so that a swapped sign row or transposed axes show
    return {0: (0.7, -0.31, 2.3, 0.45), 1: (-1.9, 0.62, -0.8, 1.7)}, {0: (-3.0, 0.5, 1.1, -0.2),
                                                                        1: (-2.0, -0.3, 0.4, 0.9)}


def _bilinear_table(cF, cN):
    """Table of the oracle's layout [sign][s row][gamma node][F, lnN] whose
    entries are a function bilinear in (log10 gamma, s/L) at the nodes:
    gamma nodes at log10 gamma = GMAX i/(NG-1), s rows at s/L = j/(NS-1)."""
    T = np.zeros((2, NS, NG, 2))
    lg = GMAX * np.arange(NG) / (NG - 1)
    sf = np.arange(NS) / (NS - 1)
    for sg in (0, 1):
        a, b, c, d = cF[sg]
        T[sg, :, :, 0] = a + b * lg[None, :] + c * sf[:, None] + d * lg[None, :] * sf[:, None]
        a, b, c, d = cN[sg]
        T[sg, :, :, 1] = a + b * lg[None, :] + c * sf[:, None] + d * lg[None, :] * sf[:, None]
    return T


def _table_sim(T, **over):
    cfg = W.config("C1", table_n_gamma=NG, table_n_s=NS, table_log10g_max=GMAX, **over)
    return cfg, O.Sim(cfg, table=T.reshape(-1))


def test_table_lookup_reproduces_a_bilinear_function_between_nodes():
    cF, cN = _coeffs()
    cfg, S = _table_sim(_bilinear_table(cF, cN))
    k = _k_code(S)
    N = cfg["n_cells"]
    rng = np.random.default_rng(5)
    for _ in range(400):
        lg = rng.uniform(0.0, GMAX)
        sg = int(rng.integers(0, 2))
        s = rng.uniform(0.0, N)
        u = _u_of(lg, 1.0 if sg == 0 else -1.0)
        if sg == 1 and u == 0.0:
            continue
        lg_exact = math.log10(math.sqrt(1.0 + u * u))
        sf = s / N
        a, b, c, d = cF[sg]
        F_want = k * (a + b * lg_exact + c * sf + d * lg_exact * sf)
        a, b, c, d = cN[sg]
        lnN_want = a + b * lg_exact + c * sf + d * lg_exact * sf
        F, dF, rate = S.drag(u, s)
        assert F == pytest.approx(F_want, rel=1e-11, abs=1e-11 * k)
        assert math.log(rate / k) == pytest.approx(lnN_want, rel=1e-11, abs=1e-11)


def test_table_lookup_at_both_line_ends_and_beyond_the_table():
    cF, cN = _coeffs()
    cfg, S = _table_sim(_bilinear_table(cF, cN))
    k = _k_code(S)
    N = cfg["n_cells"]
    for s, sf in ((0.0, 0.0), (float(N), 1.0)):
        for sg, sign in ((0, 1.0), (1, -1.0)):
            for lg in (0.5, 3.3, 7.9):
                u = _u_of(lg, sign)
                a, b, c, d = cF[sg]
                F, _, _ = S.drag(u, s)
                assert F == pytest.approx(k * (a + b * lg + c * sf + d * lg * sf), rel=1e-11)
            # above the table's top the lookup holds the top node's value
            a, b, c, d = cF[sg]
            F, dF, _ = S.drag(_u_of(GMAX + 1.5, sign), s)
            assert F == pytest.approx(k * (a + b * GMAX + c * sf + d * GMAX * sf), rel=1e-11)
            assert dF == 0.0


def test_table_derivative_is_the_slope_of_the_interpolant():
    cF, cN = _coeffs()
    cfg, S = _table_sim(_bilinear_table(cF, cN))
    k = _k_code(S)
    N = cfg["n_cells"]
    rng = np.random.default_rng(8)
    for _ in range(300):
        lg = rng.uniform(0.05, GMAX - 0.05)
        sign = float(rng.choice([-1.0, 1.0]))
        s = rng.uniform(0.0, N)
        u = _u_of(lg, sign)
        node = lg / (GMAX / (NG - 1))
        if abs(u) < 1e-2 or abs(node - round(node)) < 1e-3:
            continue
        # stay inside one gamma cell of the table: a relative step of 1e-5 in u
        h = 1e-5 * abs(u)
        Fp, _, _ = S.drag(u + h, s)
        Fm, _, _ = S.drag(u - h, s)
        _, dF, _ = S.drag(u, s)
        fd = (Fp - Fm) / (2.0 * h)
        sg = 0 if sign > 0 else 1
        a, b, c, d = cF[sg]
        # analytic slope of the generating function: dF/du = k (b + d s/L) dlog10g/du
        gam2 = 1.0 + u * u
        want = k * (b + d * s / N) * u / (gam2 * math.log(10.0))
        assert dF == pytest.approx(fd, rel=1e-8)
        assert dF == pytest.approx(want, rel=1e-10)


def test_table_nodes_return_the_stored_quadrature_value():
    cfg = W.config("C1", table_n_gamma=NG, table_n_s=NS, table_log10g_max=GMAX, quad_n_mu=16, quad_n_phi=16)
    T = O.build_table(cfg).reshape(2, NS, NG, 2)
    S = O.Sim(cfg, table=T.reshape(-1))
    k = _k_code(S)
    N = cfg["n_cells"]
    for sg, sign in ((0, 1.0), (1, -1.0)):
        for j in (0, 3, NS - 1):
            for i in (1, 6, NG - 1):
                u = _u_of(GMAX * i / (NG - 1), sign)
                s = N * j / (NS - 1)
                F, _, rate = S.drag(u, s)
                scale = np.max(np.abs(T[sg, j, :, 0]))
                assert F == pytest.approx(k * T[sg, j, i, 0], rel=1e-9, abs=1e-9 * k * scale)
                if T[sg, j, i, 1] > -600:
                    assert math.log(rate / k) == pytest.approx(T[sg, j, i, 1], rel=1e-9, abs=1e-9)


def test_table_off_node_within_bilinear_bound_of_the_radial_closed_form():
    """RADIAL table (entries are Eq. contdrag at the nodes): between nodes the
    lookup differs from the closed form at the same (gamma, s) by no more than
    the bilinear interpolation bound a(1-a)/2 |D_tt| + c(1-c)/2 |D_ss| (in
    node units), with the second differences taken from the table around the
    cell.  An s index off by part of a row makes a first-order error that
    exceeds it."""
    ng, ns = 64, 64
    cfg = W.config("C1", table_n_gamma=ng, table_n_s=ns, table_log10g_max=GMAX, photon_model=O.PHOTON_RADIAL)
    T = O.build_table(cfg).reshape(2, ns, ng, 2)
    S = O.Sim(cfg, table=T.reshape(-1))
    C = O.Sim(dict(cfg, drag_law=O.DRAG_CLOSED))
    N = cfg["n_cells"]
    rng = np.random.default_rng(13)
    checked = 0
    for _ in range(600):
        i = int(rng.integers(1, ng - 3))
        j = int(rng.integers(1, ns - 3))
        a = rng.uniform(0.05, 0.95)
        c = rng.uniform(0.05, 0.95)
        sg = int(rng.integers(0, 2))
        sign = 1.0 if sg == 0 else -1.0
        lg = GMAX * (i + a) / (ng - 1)
        s = N * (j + c) / (ns - 1)
        u = _u_of(lg, sign)
        Ft, _, _ = S.drag(u, s)
        Fc, _, _ = C.drag(u, s)
        F = T[sg, :, :, 0]
        dtt = max(abs(F[jj, ii + 1] - 2 * F[jj, ii] + F[jj, ii - 1])
                  for jj in (j, j + 1) for ii in (i, i + 1))
        dss = max(abs(F[jj + 1, ii] - 2 * F[jj, ii] + F[jj - 1, ii])
                  for jj in (j, j + 1) for ii in (i, i + 1))
        bound = _k_code(S) * (a * (1 - a) / 2 * dtt + c * (1 - c) / 2 * dss)
        # a factor 2 covers the variation of the second differences over the cell
        assert abs(Ft - Fc) <= 2.0 * bound + 1e-12 * abs(Fc), (i, j, a, c, sg, Ft, Fc, bound)
        checked += 1
    assert checked == 600


@pytest.mark.parametrize("s_frac", [0.02, 0.2, 0.5, 0.83])
def test_closed_form_derivative_matches_central_differences(s_frac):
    """The closed form's dF/du (Eq. contdrag differentiated: the factor
    gamma (mu - beta), the resonance variable y and g(y)) against central
    differences of F, over u in +-[1e-3, 1e6], at points of the line with
    different (x, b, mu)."""
    cfg = W.config("C1", drag_law=O.DRAG_CLOSED, photon_model=O.PHOTON_RADIAL)
    S = O.Sim(cfg)
    s = s_frac * cfg["n_cells"]
    n_ok = 0
    for sign in (1.0, -1.0):
        for lu in np.linspace(-3.0, 6.0, 37):
            u = sign * 10.0 ** lu
            # Richardson-extrapolated central difference: where the Wien
            # factor makes F ~ exp(-y) with y in the hundreds, the plain
            # difference's h^2 term alone would exceed the tolerance
            h = 1e-5 * abs(u)
            F, dF, _ = S.drag(u, s)
            d1 = (S.drag(u + h, s)[0] - S.drag(u - h, s)[0]) / (2.0 * h)
            d2 = (S.drag(u + h / 2, s)[0] - S.drag(u - h / 2, s)[0]) / h
            fd = (4.0 * d2 - d1) / 3.0
            scale = abs(dF) + abs(F) / abs(u)
            if scale == 0.0:
                continue
            assert abs(dF - fd) <= 1e-6 * scale, (u, s, F, dF, fd)
            n_ok += 1
    assert n_ok >= 20

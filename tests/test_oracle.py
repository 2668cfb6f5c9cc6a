"""Pins for the FP64 oracle: every check here comes from something other than
the oracle itself (hand-derived closed forms, exact rational arithmetic,
library routines on tiny inputs, invariants of Eq. 1).  CPU only."""
import glob
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import gwas_synth
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _study(n, p, k, h, sigma2=1.0, seed=7, m=23):
    s = gwas_synth.study(n, p, k, h, sigma2, seed=seed)
    X = gwas_synth.dosages(n, 0, m, seed=seed).astype(np.float64)
    return s, X


def _bruteforce_eq1(Phi, XL, y, XR, h, sigma2):
    """Eq. 1 with numpy's explicit inverse (library routine), per SNP."""
    n = Phi.shape[0]
    Mi = np.linalg.inv(sigma2 * (h * Phi + (1 - h) * np.eye(n)))
    rs, ses = [], []
    for i in range(XR.shape[1]):
        Xi = np.column_stack([XL, XR[:, i]])
        S = Xi.T @ Mi @ Xi
        rs.append(np.linalg.solve(S, Xi.T @ Mi @ y))
        ses.append(np.sqrt(np.diag(np.linalg.inv(S))))
    return np.array(rs).T, np.array(ses).T


# --- hand-derived closed forms ------------------------------------------------

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
def test_golden_closed_forms(path):
    d = json.load(open(path))
    n = d["n"]
    XL = np.array(d["XL"], dtype=float).reshape(n, d["p"] - 1)
    r, se, chi2, st = oracle.gls_from_phi(np.array(d["Phi"], float), XL, np.array(d["y"], float),
                                          np.array(d["XR"], float), d["h"], d["sigma2"])
    assert st.tolist() == [0] * len(d["chi2"])
    np.testing.assert_allclose(r, np.array(d["r"]), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(se, np.array(d["se"]), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(chi2, np.array(d["chi2"]), rtol=1e-13, atol=1e-14)


# --- exact rational brute force ------------------------------------------------

def _frac_solve(A, b):
    """Gauss-Jordan elimination in exact rationals."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * b2 for a, b2 in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def test_exact_rational_eq1():
    rng = np.random.default_rng(3)
    n, q = 6, 2
    B = rng.integers(-2, 3, size=(n, n))
    Phi = [[Fraction(int(v)) for v in row] for row in (B @ B.T + n * np.eye(n, dtype=int))]
    h, sigma2 = Fraction(3, 5), Fraction(5, 2)
    M = [[sigma2 * (h * Phi[i][j] + ((1 - h) if i == j else 0)) for j in range(n)] for i in range(n)]
    XL = np.column_stack([np.ones(n, dtype=int), rng.integers(-3, 4, size=(n, q - 1))])
    XR = rng.integers(0, 3, size=(n, 4))
    y = rng.integers(-5, 6, size=n)
    r_o, se_o, _, st = oracle.gls_from_phi(np.array(Phi, dtype=float), XL, y, XR, float(h), float(sigma2))
    assert not st.any()
    for i in range(XR.shape[1]):
        X = [[Fraction(int(v)) for v in row] for row in np.column_stack([XL, XR[:, i]])]
        p = len(X[0])
        MiX = [_frac_solve(M, [X[r][c] for r in range(n)]) for c in range(p)]  # columns of M^-1 X
        Miy = _frac_solve(M, [Fraction(int(v)) for v in y])
        S = [[sum(X[r][a] * MiX[b][r] for r in range(n)) for b in range(p)] for a in range(p)]
        rhs = [sum(X[r][a] * Miy[r] for r in range(n)) for a in range(p)]
        r_exact = _frac_solve(S, rhs)
        Sinv_diag = [_frac_solve(S, [Fraction(int(j == c)) for j in range(p)])[c] for c in range(p)]
        np.testing.assert_allclose(r_o[:, i], [float(v) for v in r_exact], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(se_o[:, i] ** 2, [float(v) for v in Sinv_diag], rtol=1e-13)


# --- library routines on tiny inputs ------------------------------------------------

@pytest.mark.parametrize("n,p,h,sigma2", [(40, 4, 0.6, 1.0), (64, 2, 0.3, 2.5), (33, 6, 0.9, 0.7), (17, 1, 0.5, 1.0)])
def test_bruteforce_numpy_inverse(n, p, h, sigma2):
    s, X = _study(n, p, 2 * n, h, sigma2, m=37)
    r, se, chi2, st = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, h, sigma2)
    r_b, se_b = _bruteforce_eq1(s["Phi"], s["XL"], s["y"], X, h, sigma2)
    assert not st.any()
    np.testing.assert_allclose(r, r_b, rtol=1e-10, atol=1e-12 * np.abs(r_b).max())
    np.testing.assert_allclose(se, se_b, rtol=1e-11)
    np.testing.assert_allclose(chi2, (r[-1] / se[-1]) ** 2, rtol=1e-12)


def test_potrf_reconstructs_and_is_lower():
    s, _ = _study(50, 4, 100, 0.6)
    M = oracle.form_m(s["Phi"], 0.6, 1.3)
    L = oracle.potrf(M)
    assert np.allclose(np.triu(L, 1), 0.0)
    assert (np.diag(L) > 0).all()
    np.testing.assert_allclose(L @ L.T, M, rtol=0, atol=1e-13 * np.abs(M).max())
    np.testing.assert_allclose(L, np.linalg.cholesky(M), rtol=1e-12, atol=1e-14)


def test_potrf_reports_first_bad_pivot():
    A = np.eye(6)
    A[3, 3] = -1.0
    with pytest.raises(oracle.NotSPD) as e:
        oracle.potrf(A)
    assert e.value.index == 3
    B = np.ones((4, 4)) + np.eye(4) * 0.0  # rank one: pivot 1 is exactly zero
    with pytest.raises(oracle.NotSPD) as e:
        oracle.potrf(B)
    assert e.value.index == 1


def test_trsm_lower_solves():
    s, X = _study(70, 4, 140, 0.6, m=19)
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.6, 1.0))
    Xt = oracle.trsm_lower(L, X)
    np.testing.assert_allclose(L @ Xt, X, rtol=0, atol=1e-12)
    from scipy.linalg import solve_triangular
    np.testing.assert_allclose(Xt, solve_triangular(L, X, lower=True), rtol=1e-12, atol=1e-13)


# --- invariants and special cases of Eq. 1 ------------------------------------------------

def test_h0_reduces_to_ols():
    s, X = _study(80, 4, 160, 0.0, sigma2=1.7, m=21)
    r, se, _, _ = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.0, 1.7)
    for i in range(X.shape[1]):
        Xi = np.column_stack([s["XL"], X[:, i]])
        b, *_ = np.linalg.lstsq(Xi, s["y"], rcond=None)
        np.testing.assert_allclose(r[:, i], b, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(se[:, i], np.sqrt(1.7 * np.diag(np.linalg.inv(Xi.T @ Xi))), rtol=1e-11)


@pytest.mark.parametrize("h", [0.2, 0.8, 1.0])
def test_identity_phi_is_ols_for_any_h(h):
    s, X = _study(60, 3, 120, h, m=9)
    r, _, _, _ = oracle.gls_from_phi(np.eye(60), s["XL"], s["y"], X, h, 1.0)
    for i in range(X.shape[1]):
        b, *_ = np.linalg.lstsq(np.column_stack([s["XL"], X[:, i]]), s["y"], rcond=None)
        np.testing.assert_allclose(r[:, i], b, rtol=1e-10, atol=1e-12)


def test_sigma2_invariance():
    s, X = _study(90, 4, 180, 0.6, m=17)
    out = {sg: oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.6, sg) for sg in (0.1, 1.0, 7.0)}
    for sg in (0.1, 7.0):
        np.testing.assert_allclose(out[sg][0], out[1.0][0], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(out[sg][1], out[1.0][1] * np.sqrt(sg), rtol=1e-12)


def test_exact_recovery():
    s, X = _study(75, 4, 150, 0.5, m=11)
    beta = np.array([0.7, -1.2, 0.4, 2.5])
    for i in range(X.shape[1]):
        y = np.column_stack([s["XL"], X[:, i]]) @ beta
        r, _, _, _ = oracle.gls_from_phi(s["Phi"], s["XL"], y, X[:, i:i + 1], 0.5, 1.0)
        np.testing.assert_allclose(r[:, 0], beta, rtol=1e-11, atol=1e-12)


def test_permutation_permutes_results():
    s, X = _study(64, 4, 128, 0.6, m=40)
    r, se, chi2, _ = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.6, 1.0)
    perm = np.random.default_rng(1).permutation(X.shape[1])
    r2, se2, chi22, _ = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X[:, perm], 0.6, 1.0)
    np.testing.assert_array_equal(r2, r[:, perm])
    np.testing.assert_array_equal(se2, se[:, perm])
    np.testing.assert_array_equal(chi22, chi2[perm])


def test_choice_of_factor():
    """Any F with F F^T = M gives the same r (Eq. 2 does not depend on the factor)."""
    s, X = _study(48, 4, 96, 0.7, m=13)
    M = 0.7 * s["Phi"] + 0.3 * np.eye(48)
    w, V = np.linalg.eigh(M)
    F = V @ np.diag(np.sqrt(w)) @ V.T  # symmetric square root
    r, _, _, _ = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.7, 1.0)
    yt = np.linalg.solve(F, s["y"])
    for i in range(X.shape[1]):
        Xt = np.linalg.solve(F, np.column_stack([s["XL"], X[:, i]]))
        b, *_ = np.linalg.lstsq(Xt, yt, rcond=None)
        np.testing.assert_allclose(r[:, i], b, rtol=1e-10, atol=1e-12)


def test_column_scaling_and_y_shift():
    s, X = _study(55, 4, 110, 0.6, m=7)
    r, _, _, _ = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.6, 1.0)
    r2, _, _, _ = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], 3.0 * X, 0.6, 1.0)
    np.testing.assert_allclose(r2[-1], r[-1] / 3.0, rtol=1e-11)
    np.testing.assert_allclose(r2[:-1], r[:-1], rtol=1e-11, atol=1e-13)
    r3, _, _, _ = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"] + 2.5 * s["XL"][:, 1], X, 0.6, 1.0)
    expect = r.copy()
    expect[1] += 2.5
    np.testing.assert_allclose(r3, expect, rtol=1e-11, atol=1e-12)


def test_singular_snp_status():
    s, X = _study(60, 4, 120, 0.6, m=4)
    X[:, 1] = 2.0          # monomorphic: collinear with the intercept
    X[:, 2] = 2.0
    X[7, 2] = 1.0          # one sample differs: still a valid design
    r, se, chi2, st = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.6, 1.0)
    assert st.tolist() == [0, 1, 0, 0]
    assert np.isnan(r[:, 1]).all() and np.isnan(se[:, 1]).all() and np.isnan(chi2[1])
    assert np.isfinite(r[:, [0, 2, 3]]).all()


def test_group_tail_and_empty():
    s, X = _study(30, 4, 60, 0.6, m=33)  # 33 = 2 groups of 16 + a tail of 1
    r, _, _, _ = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.6, 1.0)
    r_b, _ = _bruteforce_eq1(s["Phi"], s["XL"], s["y"], X, 0.6, 1.0)
    np.testing.assert_allclose(r, r_b, rtol=1e-10, atol=1e-12)
    r0, se0, c0, st0 = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X[:, :0], 0.6, 1.0)
    assert r0.shape == (4, 0) and st0.shape == (0,)


def test_generator_columns_regenerate_independently():
    full = gwas_synth.dosages(100, 0, 700, seed=5)
    np.testing.assert_array_equal(gwas_synth.dosages(100, 250, 530, seed=5), full[:, 250:530])
    assert set(np.unique(full)) <= {0, 1, 2}
    Phi = gwas_synth.kinship(gwas_synth.kinship_genotypes(80, 40, seed=5))
    np.testing.assert_allclose(Phi, Phi.T, rtol=0, atol=0)
    assert np.linalg.eigvalsh(Phi).min() >= gwas_synth.KINSHIP_RIDGE * 0.999


# --- gradients and REML (the differentiation form) ---------------------------------

def test_grad_matches_central_differences():
    s, X = _study(70, 4, 140, 0.6, sigma2=1.3, m=6)
    L = oracle.potrf(oracle.form_m(s["Phi"], 0.6, 1.3))
    chi2, dh, dy = oracle.gls_grad(L, s["Phi"], 0.6, 1.3, s["XL"], s["y"], X)
    c_ref = oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.6, 1.3)[2]
    np.testing.assert_allclose(chi2, c_ref, rtol=1e-12)
    d = 1e-6
    fd_h = (oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.6 + d, 1.3)[2]
            - oracle.gls_from_phi(s["Phi"], s["XL"], s["y"], X, 0.6 - d, 1.3)[2]) / (2 * d)
    np.testing.assert_allclose(dh, fd_h, rtol=1e-6, atol=1e-8)
    for j in (0, 13, 69):
        yp, ym = s["y"].copy(), s["y"].copy()
        yp[j] += d
        ym[j] -= d
        fd = (oracle.gls_from_phi(s["Phi"], s["XL"], yp, X, 0.6, 1.3)[2].sum()
              - oracle.gls_from_phi(s["Phi"], s["XL"], ym, X, 0.6, 1.3)[2].sum()) / (2 * d)
        assert abs(dy[j] - fd) <= 1e-6 * max(1.0, abs(fd)), (j, dy[j], fd)


def test_grad_special_cases():
    s, X = _study(50, 3, 100, 0.4, m=5)
    # Phi = I: M = sigma2 I for every h, so chi2 does not depend on h
    L = oracle.potrf(oracle.form_m(np.eye(50), 0.4, 1.0))
    _, dh, _ = oracle.gls_grad(L, np.eye(50), 0.4, 1.0, s["XL"], s["y"], X)
    np.testing.assert_array_equal(dh, 0.0)
    # b does not depend on sigma2 and (S^-1)_pp scales with it, so chi2 and its gradients scale 1/sigma2
    L2 = oracle.potrf(oracle.form_m(s["Phi"], 0.4, 2.0))
    L1 = oracle.potrf(oracle.form_m(s["Phi"], 0.4, 1.0))
    c2, dh2, dy2 = oracle.gls_grad(L2, s["Phi"], 0.4, 2.0, s["XL"], s["y"], X)
    c1, dh1, dy1 = oracle.gls_grad(L1, s["Phi"], 0.4, 1.0, s["XL"], s["y"], X)
    np.testing.assert_allclose(c2, c1 / 2.0, rtol=1e-11)
    np.testing.assert_allclose(dh2, dh1 / 2.0, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(dy2, dy1 / 2.0, rtol=1e-9, atol=1e-12)


def test_reml_gradient_and_closed_forms():
    s, _ = _study(80, 3, 160, 0.5)
    XL, y, Phi = s["XL"], s["y"], s["Phi"]
    l, dl, s2 = oracle.reml(Phi, XL, y, 0.5)
    d = 1e-6
    fd = (oracle.reml(Phi, XL, y, 0.5 + d, grad=False)[0] - oracle.reml(Phi, XL, y, 0.5 - d, grad=False)[0]) / (2 * d)
    assert abs(dl - fd) <= 1e-6 * max(1.0, abs(fd))
    # h = 0: V = I, the REML likelihood of ordinary least squares
    n, q = XL.shape
    beta, *_ = np.linalg.lstsq(XL, y, rcond=None)
    rss = float(np.sum((y - XL @ beta) ** 2))
    l0 = -0.5 * ((n - q) * np.log(rss / (n - q)) + np.linalg.slogdet(XL.T @ XL)[1])
    assert abs(oracle.reml(Phi, XL, y, 0.0, grad=False)[0] - l0) <= 1e-9 * abs(l0)
    # Phi = I: the likelihood does not depend on h
    g = oracle.reml(np.eye(n), XL, y, 0.3)[1]
    assert abs(g) <= 1e-10


def test_reml_argmax_is_a_stationary_maximum():
    s = gwas_synth.study(120, 3, 240, 0.5, seed=9)
    h_hat = oracle.reml_argmax(s["Phi"], s["XL"], s["y"])
    assert 0.0 < h_hat < 1.0
    l, dl, _ = oracle.reml(s["Phi"], s["XL"], s["y"], h_hat)
    assert abs(dl) <= 1e-4
    for dh in (-1e-3, 1e-3):
        assert oracle.reml(s["Phi"], s["XL"], s["y"], h_hat + dh, grad=False)[0] <= l

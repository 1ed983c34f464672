"""Comparison helpers shared by the GPU parity tests."""
import numpy as np

import oracle

# the covariance bar: relative Frobenius error against the binary64 oracle
COV_RTOL = 1e-5


def frob(a):
    return np.sqrt((np.asarray(a, np.float64) ** 2).sum(-1))


def full_frob(c6):
    """Frobenius norm of packed symmetric matrices (off-diagonals twice)."""
    c6 = np.asarray(c6, np.float64)
    w = np.array([1, 2, 2, 1, 2, 1], np.float64)
    return np.sqrt((c6 ** 2 * w).sum(-1))


def check_raw_cov(gpu6, ref6, rtol=COV_RTOL):
    """||C_gpu - C_64||_F <= rtol ||C_64||_F row by row (absolute 1e-30 floor
    for all-duplicate neighbourhoods)."""
    err = full_frob(np.asarray(gpu6, np.float64) - ref6)
    bound = rtol * full_frob(ref6) + 1e-30
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"{bad.size} rows over tolerance, e.g. row {bad[:5]} err {err[bad[:5]]} bound {bound[bad[:5]]}"


def check_regularised_cov(gpu6, ref6, raw_ref6, raw_gpu6, eps, rtol=COV_RTOL):
    """Regularised C' = I - (1-eps) n n^T.

    Bar: ||C'_gpu - C'_64||_F <= rtol ||C'_64||_F.  The normal is an
    eigenvector, so its error grows as 1/gap (Davis-Kahan: sin(theta) <=
    ||dC|| / (lambda2 - lambda3)); where the binary32 covariance error dC
    (measured, raw_gpu6 vs raw_ref6) over the eigen-gap allows more, the
    bound becomes rtol ||C'|| + 4 (||dC||_F + 1e-6 ||C||_F) / gap, the 1e-6
    covering the binary32 eigen-solve itself (~16u).  Rows with
    a repeated smallest eigenvalue (gap ~ 0) accept any unit normal from its
    eigenspace: C'_gpu must have eigenvalues {eps, 1, 1} and n^T C n within
    1e-6 tr(C) of lambda_min.  Returns the fraction of rows held to the plain
    rtol bound."""
    gpu6 = np.asarray(gpu6, np.float64)
    C = oracle.unpack6(raw_ref6)
    w, V = np.linalg.eigh(C)
    tr = np.maximum(w.sum(-1), 1e-300)
    gap = w[:, 1] - w[:, 0]
    dC = full_frob(np.asarray(raw_gpu6, np.float64) - raw_ref6)
    cnorm = full_frob(raw_ref6)
    err = full_frob(gpu6 - ref6)
    base = rtol * full_frob(ref6)
    dk = 4.0 * (dC + 1e-6 * cnorm) / np.maximum(gap, 1e-300)
    plain = err <= base
    degenerate = gap <= 1e-6 * tr
    ok = plain | ((~degenerate) & (err <= base + dk))
    for i in np.nonzero(~ok & degenerate)[0]:
        G = oracle.unpack6(gpu6[i])
        gw, gv = np.linalg.eigh(G)
        assert np.allclose(gw, [eps, 1.0, 1.0], atol=1e-5), (i, gw)
        n = gv[:, 0]
        assert n @ C[i] @ n <= w[i, 0] + 1e-6 * tr[i], i
        ok[i] = True
    bad = np.nonzero(~ok)[0]
    assert bad.size == 0, f"{bad.size} rows over tolerance, e.g. {bad[:5]} err {err[bad[:5]]} gap/tr {(gap / tr)[bad[:5]]}"
    return float(plain.mean())


U32 = 2.0 ** -24


def gicp_tolerance(eps_reg: float) -> float:
    """Relative bound for the GPU's GICP sums against the binary64 oracle.

    Per pair the GPU works in binary32.  For plane-regularised covariances
    (eigenvalues {1, 1, eps}) the combined S = C_q + R C_p R^T has
    eigenvalues in [2 eps, 2] with the middle one >= 1, and the adjugate
    inverse with the rounding of S gives an Omega whose error, measured in
    Omega's own metric (|x^T dOmega y| <= g sqrt(x^T Omega x  y^T Omega y)),
    is below about 20 u / eps; the residual, the Jacobian products and the
    32-lane binary32 sum add a few u more.  Summed over pairs,
    Cauchy-Schwarz turns this into |dH_rc| <= tau sqrt(H_rr H_cc),
    |db_r| <= tau sqrt(H_rr E) and |dE| <= tau E with tau below."""
    return 32.0 * U32 / eps_reg + 16.0 * U32


def check_gicp(got: dict, want: dict, tau: float) -> dict:
    """Asserts the bound of gicp_tolerance; returns the worst ratios."""
    assert got["pairs"] == want["pairs"]
    Hd = np.diag(want["H"]).copy()
    scaleH = np.sqrt(np.outer(Hd, Hd))
    scaleb = np.sqrt(Hd * want["error"])
    rh = np.abs(got["H"] - want["H"]) / np.maximum(scaleH, 1e-300)
    rb = np.abs(got["b"] - want["b"]) / np.maximum(scaleb, 1e-300)
    re = abs(got["error"] - want["error"]) / max(want["error"], 1e-300)
    worst = {"H": float(rh.max()), "b": float(rb.max()), "E": float(re)}
    assert worst["H"] <= tau and worst["b"] <= tau and worst["E"] <= tau, (worst, tau)
    return worst

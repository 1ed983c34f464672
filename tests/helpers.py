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


# eigen-gap bands of the regularised-covariance bar, as gap / tr(C) with
# gap = lambda2 - lambda3 of the binary64 covariance
WELL_GAP = 1e-2
DEGENERATE_GAP = 1e-6


def check_regularised_cov(gpu6, ref6, raw_ref6, raw_gpu6, eps, rtol=COV_RTOL, label=""):
    """Regularised C' = I - (1-eps) n n^T, held to a per-row rule by eigen-gap
    band (gap = lambda2 - lambda3 of the binary64 C, tr = tr C):

    * gap/tr >= 1e-2 (a well-defined normal): ||C'_gpu - C'_64||_F <= rtol
      ||C'_64||_F, no exceptions.
    * 1e-6 < gap/tr < 1e-2: the normal is an eigenvector, so its error grows
      as 1/gap (Davis-Kahan: sin(theta) <= ||E|| / gap for a perturbation
      E).  E is the measured binary32 covariance error dC (raw_gpu6 against
      raw_ref6) plus the backward error of a binary32 eigen-solve, taken as
      16u ||C||_F ~ 1e-6 ||C||_F; the row passes at rtol ||C'|| +
      4 (||dC||_F + 1e-6 ||C||_F) / gap.
    * gap/tr <= 1e-6 (repeated smallest eigenvalue): any unit normal from
      its eigenspace is correct, so C'_gpu must have eigenvalues {eps, 1, 1}
      and n^T C n within 1e-6 tr(C) of lambda_min.

    Prints and returns the row count of each band with its worst relative
    error."""
    gpu6 = np.asarray(gpu6, np.float64)
    C = oracle.unpack6(raw_ref6)
    w, _ = np.linalg.eigh(C)
    tr = np.maximum(w.sum(-1), 1e-300)
    gap = w[:, 1] - w[:, 0]
    g = gap / tr
    dC = full_frob(np.asarray(raw_gpu6, np.float64) - raw_ref6)
    cnorm = full_frob(raw_ref6)
    err = full_frob(gpu6 - ref6)
    base = rtol * full_frob(ref6)
    rel = err / np.maximum(full_frob(ref6), 1e-300)
    well = g >= WELL_GAP
    degenerate = g <= DEGENERATE_GAP
    mid = ~well & ~degenerate
    bad_well = np.nonzero(well & (err > base))[0]
    assert bad_well.size == 0, (
        f"{label} {bad_well.size} rows with gap/tr >= {WELL_GAP} over {rtol}: rows {bad_well[:5]} "
        f"rel err {rel[bad_well[:5]]} gap/tr {g[bad_well[:5]]}")
    dk = 4.0 * (dC + 1e-6 * cnorm) / np.maximum(gap, 1e-300)
    bad_mid = np.nonzero(mid & (err > base + dk))[0]
    assert bad_mid.size == 0, (
        f"{label} {bad_mid.size} rows with {DEGENERATE_GAP} < gap/tr < {WELL_GAP} over the Davis-Kahan bound: "
        f"rows {bad_mid[:5]} rel err {rel[bad_mid[:5]]} gap/tr {g[bad_mid[:5]]}")
    for i in np.nonzero(degenerate & (err > base))[0]:
        G = oracle.unpack6(gpu6[i])
        gw, gv = np.linalg.eigh(G)
        assert np.allclose(gw, [eps, 1.0, 1.0], atol=1e-5), (label, i, gw)
        n = gv[:, 0]
        assert n @ C[i] @ n <= w[i, 0] + 1e-6 * tr[i], (label, i)

    def band(m):
        return {"rows": int(m.sum()), "max_rel_err": float(rel[m].max()) if m.any() else 0.0,
                "over_rtol": int((m & (err > base)).sum())}

    bands = {"well": band(well), "mid": band(mid), "degenerate": band(degenerate)}
    print(f"regularised cov bands {label}: {bands}")
    return bands


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

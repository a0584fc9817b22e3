"""Per-entry rounding-error bound of the RAS/ILU(k) preconditioner apply
(Sections 2.5-2.6), for the parity tests.

For one block, the L solve computes y_i = r_i - sum_j l_ij y_j and the U
solve z_i = (y_i - sum_j u_ij z_j) / u_ii.  Evaluating row i in floating
point with unit roundoff u adds a local error of at most
gamma_i * (|r_i| + sum_j |l_ij| |y_j|), gamma_i = (w_i + extra) u / (1 - ...)
with w_i the row's entry count (first order: (w_i + extra) u).  Errors of
earlier rows reach row i through the same recurrence, so the accumulated
error e obeys |e_i| <= d_i + sum_j |l_ij| |e_j|: the solve with the
comparison matrix (unit diagonal, off-diagonal -|l_ij|) of the local errors
bounds it entry by entry.  The U solve adds its own local errors
(gamma_i (|y_i| + sum_j |u_ij| |z_j|) + 2u |u_ii z_i| for the reciprocal
diagonal and the product) to the error carried in from y and divides by
|u_ii|.  RAS writes every block's z on its owned rows, so the bound of a
row of z is the owning block's.

Everything here is computed from the oracle's factors and solves, in FP64:
a bound for a computation in FP64 (u = 2^-53) or in FP32 (u = 2^-24, with
the factors, r and z rounded to FP32: two more roundings per row).
"""
import numpy as np


def _abs_parts(F):
    """Row of every entry, masks of the strict L and U entries, |diag U|."""
    rows = np.repeat(np.arange(F.n), np.diff(F.row_ptr))
    lo, up, dg = F.col < rows, F.col > rows, F.col == rows
    diag = np.zeros(F.n)
    diag[rows[dg]] = np.abs(F.val[dg])
    return rows, lo, up, diag


def _matvec_abs(F, rows, mask, x):
    """sum_j |f_ij| |x_j| over the entries in mask, per row."""
    w = np.abs(F.val[mask]) * np.abs(x[F.col[mask]])
    return np.bincount(rows[mask], weights=w, minlength=F.n)


def _comparison(F, lo, up, orc):
    """A factor whose unit-lower solve computes x_i = d_i + sum |l_ij| x_j and
    whose upper solve computes x_i = (d_i + sum |u_ij| x_j) / |u_ii|."""
    val = np.abs(F.val)
    val[lo | up] *= -1.0
    return orc.Factor(F.n, F.row_ptr, F.col, val, F.lev)


def apply_bounds(orc, R, r, which):
    """Entry-wise bounds on |z_computed - z_exact| for z = M^{-1} r with M the
    oracle's RAS object R, one per entry of which (False: computed in FP64;
    True: in FP32 from FP32 factors)."""
    r = np.asarray(r, np.float64)
    out = [np.zeros(R.n) for _ in which]
    for b in range(R.nblocks):
        V, own_lo, own_hi, F = R.block(b)
        rows, lo, up, diag = _abs_parts(F)
        wL = np.bincount(rows[lo], minlength=F.n)
        wU = np.bincount(rows[up], minlength=F.n)
        rb = r[V]
        y = orc.lsolve_unit(F, rb)
        z = orc.usolve(F, y)
        G = _comparison(F, lo, up, orc)
        magL = np.abs(rb) + _matvec_abs(F, rows, lo, y)
        magU = np.abs(y) + _matvec_abs(F, rows, up, z)
        own = (V >= own_lo) & (V < own_hi)
        for E, fp32 in zip(out, which):
            u = 2.0 ** -24 if fp32 else 2.0 ** -53
            extra = 3 if fp32 else 1
            eL = orc.lsolve_unit(G, (wL + extra) * u * magL)
            eU = orc.usolve(G, eL + (wU + extra) * u * magU + 2 * u * diag * np.abs(z))
            if fp32:
                eU = eU + u * np.abs(z)  # the FP32 result itself
            E[V[own]] = eU[own]
    return out


def apply_bound(orc, R, r, fp32=False):
    return apply_bounds(orc, R, r, [fp32])[0]


def check_apply(orc, R, r, got, fp32=False, what="", ref=None):
    """Assert |got - ref| <= bound(device) + bound(oracle) entry by entry;
    returns the worst ratio |got - ref| / (bound(device) + bound(oracle))."""
    if ref is None:
        ref = R.apply(r)
    e_dev, e_orc = apply_bounds(orc, R, r, [fp32, False])
    bound = e_dev + e_orc
    got = np.asarray(got, np.float64)
    assert np.all(np.isfinite(got)), ("a row was not written", what)
    diff = np.abs(got - ref)
    bad = diff > bound
    assert not np.any(bad), (what, int(np.argmax(diff - bound)), float(np.max(diff - bound)))
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(bound > 0, diff / bound, 0.0)
    worst = float(np.max(ratio)) if ratio.size else 0.0
    print("apply parity %s: worst |z - z_ref| / bound = %.3g" % (what, worst))
    return worst

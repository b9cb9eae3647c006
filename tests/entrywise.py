"""Entry-by-entry parity bounds for operator and filter results (helper, not a test file).

A relative Frobenius-norm bound over a whole block hides an error confined to a few rows: a
periodic seam plane or a tile face that is wrong by 100x the rounding error still passes.
The checks here bound every entry on its own.

* Operator results Y = Ht X: each entry is a sum of products, and the forward-error bound of
  a floating-point sum of products is |fl(y) - y| <= gamma_n sum_i |a_i| |b_i|, so an entry
  is compared against tol * (|Ht| |X|)_Iv, the sum of the magnitudes of the terms that form
  it (computed with the oracle's assembled matrix, or row by row from the cell definition
  for the full-size slabs).
* Filter results p(Ht) X: the magnitude recurrence of the three-term filter grows
  exponentially while the filtered block does not, so there the bound is tol times the
  largest entry of the same column of the reference (a column-wise max-abs bound).
"""
import numpy as np


def _report(err, bound, what):
    ratio = err / np.maximum(bound, np.finfo(float).tiny)
    i, j = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    return (f"{what}: entry ({i}, {j}) error {err[i, j]:.3e} > bound {bound[i, j]:.3e} "
            f"(worst ratio {ratio[i, j]:.2f}; {int(np.sum(ratio > 1))} entries over)")


def assert_operator_entries(got, ref, mag, tol, what="H X"):
    """|got - ref| <= tol * mag entry by entry; mag = (|Ht| |X|) for the same entries."""
    got, ref, mag = (np.asarray(a, dtype=np.float64) for a in (got, ref, mag))
    assert got.shape == ref.shape == mag.shape
    err = np.abs(got - ref)
    bound = tol * mag
    assert np.all(err <= bound), _report(err, bound, what)
    return float(np.max(err / np.maximum(mag, np.finfo(float).tiny)))


def assert_column_maxabs(got, ref, tol, what="filter"):
    """|got - ref|_Iv <= tol * max_J |ref_Jv| for every entry."""
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape
    err = np.abs(got - ref)
    bound = tol * np.broadcast_to(np.max(np.abs(ref), axis=0, keepdims=True), ref.shape)
    assert np.all(err <= bound), _report(err, bound, what)
    return float(np.max(err / np.maximum(bound / tol, np.finfo(float).tiny)))


def magnitude(H, X):
    """(|Ht| |X|) with the oracle's assembled (sparse) Ht."""
    return abs(H) @ np.abs(np.asarray(X, dtype=np.float64))

"""Parity bars shared by the GPU tests.

Every field comparison with the oracle (or with the library's own FP64 path,
where a test says so) checks two things:

* the relative L2 error ``||got - ref|| / ||ref||`` against the bar ``tol``
  (the bar the method's accuracy is stated in: 1e-12 in FP64, 1e-5 .. 1e-6 in
  FP32);
* the largest element error against ``K_ELEM * tol * max|ref|``.

The second bar catches an error confined to a few cells (one wall plane, one
tile edge, one ragged tail), which the L2 norm of a large field averages away:
on the 256 x 256 x 128 shear drop a single wrong cell of size 5e-4 still
passes a 1e-6 relative-L2 bar, but fails the element bar (1e-5) by 50x.
K_ELEM = 10 leaves room for the ratio of a spread error's maximum to its RMS
(every test prints both errors) while staying far below the sqrt(N) by which
the L2 bar lets a concentrated error through.
"""
import numpy as np

K_ELEM = 10.0


def rel_l2(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def max_rel(a, b):
    """max |a - b| / max |b|."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def assert_parity(got, ref, tol, what="", k=K_ELEM):
    """Assert rel-L2 <= tol and max|got - ref| <= k tol max|ref|; returns both errors."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite values"
    l2 = rel_l2(got, ref)
    em = max_rel(got, ref)
    print(f"{what}: rel L2 {l2:.3e} (bar {tol:.0e}), max elem {em:.3e} (bar {k * tol:.0e})")
    assert l2 <= tol, f"{what}: rel L2 {l2:.3e} > {tol:.1e}"
    assert em <= k * tol, f"{what}: max element error {em:.3e} of max|ref| > {k * tol:.1e}"
    return l2, em

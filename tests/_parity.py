"""Comparison of a CUDA image with the FP64 oracle's on the same seeded
inputs: relative L2 over all pixels x bins x Stokes components, and, so that a
small cluster of wrong elements cannot hide in a large image, the largest
per-element difference relative to the image's largest magnitude."""
import numpy as np

TOL = 1e-3        # relative L2 (the FP32-vs-FP64 tolerance of the method's images)
ELEM_TOL = 1e-3   # max |gpu - oracle| over elements / max |oracle|


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def elem_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def assert_parity(img, ref, tol=TOL, elem_tol=ELEM_TOL, label=None):
    r, e = rel_l2(img, ref), elem_err(img, ref)
    assert r <= tol, ("rel-L2", r, label)
    assert e <= elem_tol, ("max element error / max |oracle|", e, label)
    return r, e

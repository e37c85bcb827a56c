"""Gradient comparison of the CUDA path against the FP64 oracle: per variable class and element by
element.

One norm over the whole gradient hides a class whose entries are small next to the others: the
reserve block r of rt617 is five orders of magnitude below the voltage block, so it could be wholly
wrong while ||g - g_ref|| / ||g_ref|| stays under 1e-4.  Every parity test therefore checks

* each variable class c (v, theta, p, q, r, tau, phi, u) against its own norm,
      ||g_c - r_c||_2 <= tol ||r_c||_2,
* and every element against its own magnitude plus a floor tied to its class,
      |g_i - r_i| <= tol_e (|r_i| + FLOOR ||r_c||_inf),   FLOOR = 0.1,
  with tol_e = tol on the FP64 path and 10 tol on the mixed path.

Why a floor: an element's rounding error does not scale with the element itself where large terms
cancel in it (the v and theta entries sum branch-end adjoints of opposite sign) or where its penalty
sits at a kink of the soft-abs / soft-ReLU, whose derivative moves by 1/eps per unit of error in its
argument.  In the mixed path that argument (a bus balance from FP32 flows, a post-contingency flow)
carries FP32 rounding, so an element near a kink can be off by c/eps times it.  Measured worst
cases over all parity cases, relative to |r_i| + 0.1 ||r_c||_inf: 3e-11 on the FP64 path, 1e-4 on
the mixed path.  With tol_e = 10 tol on the mixed path a wrong sign or a dropped term in an element
still fails unless the element is below 5e-5 of its class's largest entry.
"""
import numpy as np

FLOOR = 0.1
TOL64 = 1e-10
TOL32 = 1e-4


def class_slices(case):
    """(name, slice) of each non-empty variable class of one instance, in the layout of x."""
    T, n, G = case.T, case.n_bus, case.n_gen
    X = int(getattr(case, "n_xf", 0))
    U = G if getattr(case, "commit", False) else 0
    out = []
    o = 0
    for name, size in (("v", T * n), ("theta", T * n), ("p", T * G), ("q", T * G), ("r", T * G),
                       ("tau", T * X), ("phi", T * X), ("u", T * U)):
        if size:
            out.append((name, slice(o, o + size)))
        o += size
    assert o == case.n_x
    return out


def grad_errors(g, ref, case=None, classes=None):
    """{class: (normwise relative error, worst element ratio |g_i - r_i| / (|r_i| + FLOOR max|r_c|))}
    over the variable classes of `case`, or over `classes` ((name, index array or slice) pairs)."""
    g = np.asarray(g, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    out = {}
    for name, sl in (class_slices(case) if classes is None else classes):
        gc, rc = g[sl], ref[sl]
        nr = np.linalg.norm(rc)
        mx = np.abs(rc).max()
        d = np.abs(gc - rc)
        if nr == 0.0:  # a class with no gradient at all: compare against the whole vector's scale
            scale = max(np.abs(ref).max(), 1e-300)
            out[name] = (float(np.linalg.norm(gc) / scale), float(d.max() / scale))
        else:
            out[name] = (float(np.linalg.norm(gc - rc) / nr), float((d / (np.abs(rc) + FLOOR * mx)).max()))
    return out


def check_grad(g, ref, case, tol, elem_tol=None, label="", classes=None):
    """Assert the per-class and element-wise bounds above (elem_tol defaults to tol)."""
    elem_tol = tol if elem_tol is None else elem_tol
    assert np.all(np.isfinite(g)), f"{label}: non-finite gradient"
    for name, (nrel, erel) in grad_errors(g, ref, case, classes).items():
        assert nrel <= tol, f"{label} class {name}: ||g - g_ref|| / ||g_ref|| = {nrel:.3e} > {tol:.1e}"
        assert erel <= elem_tol, f"{label} class {name}: element error {erel:.3e} > {elem_tol:.1e}"


def check64(g, ref, case, label=""):
    check_grad(g, ref, case, TOL64, TOL64, label)


def check32(g, ref, case, label=""):
    check_grad(g, ref, case, TOL32, 10 * TOL32, label)


def check_prec(g, ref, case, precision, label=""):
    """precision: 0 (FP64 path) or 1 (mixed path), the QG_FP64 / QG_MIXED values."""
    (check64 if precision == 0 else check32)(g, ref, case, label)


def check_at(g, ref, case, tol, label="", classes=None):
    """check_grad at a stated class tolerance: FP64-path tolerances (<= 1e-9) check elements at the
    same tolerance, mixed-path ones at 10 times it."""
    check_grad(g, ref, case, tol, tol if tol <= 1e-9 else 10 * tol, label, classes)

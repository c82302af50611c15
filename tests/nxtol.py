"""Tolerances shared by the GPU parity tests (FP32 on the GPU vs the FP64 oracle).

PageRank family: L1 over the vector <= 1e-6 and per-vertex relative error
<= 1e-4 over vertices with a non-zero reference. Gradients of the weighted-
PageRank adjoint: the same two numbers, with L1 taken relative to the
reference's L1 norm (ranks sum to one, so for ranks the two agree).

dL/dw_uv = a r_u / W_u (lambda_v - y_u), y_u = sum_v' w^_uv' lambda_v', is a
difference of two positive terms. FP32 carries lambda and y to a relative
error eps of about 1e-7..1e-6, so an entry's error is about
eps * a r_u / W_u (|lambda_v| + |y_u|) however small the difference is. An
entry counts as cancelling when |dL/dw| < 1e-2 of that operand scale
S_e = a r_u / W_u (|lambda_v| + |y_u|); it must then be within 1e-6 S_e (the
error the 1e-4 relative bound allows at the boundary). Every other entry must
be within 1e-4 relative.
"""
import numpy as np

L1_TOL = 1e-6
REL_TOL = 1e-4
CANCEL = 1e-2


def pr_err(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.float64)
    l1 = float(np.abs(gpu - ref).sum())
    nz = ref != 0
    rel = float((np.abs(gpu - ref)[nz] / np.abs(ref[nz])).max()) if nz.any() else 0.0
    return l1, rel


def assert_pr_close(gpu, ref, what=""):
    l1, rel = pr_err(gpu, ref)
    print(f"{what}: L1={l1:.3e} max_rel={rel:.3e}")
    assert l1 <= L1_TOL, (what, l1, rel)
    assert rel <= REL_TOL, (what, l1, rel)
    return l1, rel


def assert_grad_t_close(got, ref, what="dL/dt"):
    """dL/dt = (1 - a) lambda: a sum of non-negative terms, no cancellation."""
    got = np.asarray(got, dtype=np.float64)
    rl1 = np.abs(got - ref).sum() / max(np.abs(ref).sum(), 1e-300)
    nz = ref != 0
    rel = float((np.abs(got - ref)[nz] / np.abs(ref[nz])).max()) if nz.any() else 0.0
    print(f"{what}: rel_L1={rl1:.3e} max_rel={rel:.3e}")
    assert rl1 <= L1_TOL and rel <= REL_TOL, (what, rl1, rel)
    assert (got[~nz] == 0).all(), (what, "entries the reference holds at zero")
    return rl1, rel


def assert_grad_w_close(got, ref, s, d, w, alpha=0.85, what="dL/dw"):
    """dL/dw against the oracle's adjoint (`ref`: its dict with r, lam, dw)."""
    got = np.asarray(got, dtype=np.float64)
    want = ref["dw"]
    s = np.asarray(s, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    n = len(ref["r"])
    W = np.bincount(s, weights=w, minlength=n)
    lam = ref["lam"]
    y = np.bincount(s, weights=w / W[s] * lam[d], minlength=n)
    scale = alpha * ref["r"][s] / W[s] * (np.abs(lam[d]) + np.abs(y[s]))
    err = np.abs(got - want)
    rl1 = err.sum() / max(np.abs(want).sum(), 1e-300)
    cancel = np.abs(want) < CANCEL * scale
    keep = ~cancel & (want != 0)
    rel = float((err[keep] / np.abs(want[keep])).max()) if keep.any() else 0.0
    floor = float((err[cancel] / scale[cancel]).max()) if cancel.any() else 0.0
    print(f"{what}: rel_L1={rl1:.3e} max_rel={rel:.3e} over {int(keep.sum())} entries; "
          f"{int(cancel.sum())} cancelling entries within {floor:.3e} of their operand scale")
    assert rl1 <= L1_TOL, (what, rl1)
    assert rel <= REL_TOL, (what, rel)
    assert floor <= REL_TOL * CANCEL, (what, floor)
    return rl1, rel

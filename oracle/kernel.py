"""Cubic-spline softening kernel and the overlap integral g_ij (oracle, FP64).

Parity: pinned.  tests/test_oracle_kernel.py checks
  * int W d^3x = 1 (Sec. 2.4: "This kernel integrates to 1"),
  * int g(d) d^3d = 1 for any (h_i, h_j) (g is the convolution of two unit kernels),
  * g against a direct 2D quadrature of the unsubstituted (r, cos theta) form of
    App. D with the roles of i and j swapped (so the substitution used below and
    the h_i >= h_j ordering are checked independently),
  * g(d; h_i, h_j) -> W(d, h_i) as h_j/h_i -> 0, and g = 0 for d >= h_i + h_j.
"""
import numpy as np

_INV_PI8 = 8.0 / np.pi

# Gauss-Legendre nodes/weights on [-1, 1].
_GL3_X, _GL3_W = np.polynomial.legendre.leggauss(3)
_GL5_X, _GL5_W = np.polynomial.legendre.leggauss(5)


def w_unit(u):
    """Dimensionless kernel w(u) with W(r, h) = w(r/h) / h^3 (Sec. 2.4 cubic spline)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    inner = (u >= 0.0) & (u <= 0.5)
    outer = (u > 0.5) & (u <= 1.0)
    out[inner] = 1.0 - 6.0 * u[inner] ** 2 + 6.0 * u[inner] ** 3
    out[outer] = 2.0 * (1.0 - u[outer]) ** 3
    return _INV_PI8 * out


def W(r, h):
    """Cubic-spline kernel W(r, h) (Sec. 2.4); zero for r > h."""
    r = np.asarray(r, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    return w_unit(r / h) / h ** 3


def _int_u_w(lo, hi):
    """int_lo^hi u w(u) du for 0 <= lo <= hi, exact.

    u w(u) is a polynomial of degree 4 on [0, 1/2] and on [1/2, 1] and zero
    beyond 1, so 3-point Gauss-Legendre on each piece is exact.  The integrand
    is non-negative, so the result has no cancellation even when hi - lo is tiny.
    """
    total = 0.0
    for a, b in ((0.0, 0.5), (0.5, 1.0)):
        l = max(lo, a)
        r = min(hi, b)
        if r <= l:
            continue
        mid = 0.5 * (l + r)
        half = 0.5 * (r - l)
        u = mid + half * _GL3_X
        total += half * float(np.dot(_GL3_W, u * w_unit(u)))
    return total


def overlap_g(d, h_i, h_j):
    """Overlap integral g_ij = int d^3x W(|x - x_i|, h_i) W(|x - x_j|, h_j).

    Defined in Eq. dm-update-prob; evaluated as in App. D.  g is symmetric, so
    the pair is ordered with h_a = max(h_i, h_j) >= h_b = min (App. D) and
        g = (2 pi / h_b^3) int_0^1 ds s^2 w(s) int_{-1}^{1} dc w(sqrt(s^2 + delta^2 - 2 delta s c) / q)
    with delta = d / h_a and q = h_b / h_a.  The inner c-integral is done exactly
    by the substitution t^2 = s^2 + delta^2 - 2 delta s c:
        int dc w(t/q) = (q^2 / (delta s)) int_{|s-delta|/q}^{(s+delta)/q} u w(u) du ,
    and the remaining s-integrand is a piecewise polynomial of degree <= 9, so
    5-point Gauss-Legendre between its breakpoints is exact.  delta = 0 uses the
    limit int dc w(t/q) = 2 w(s/q).
    """
    d = float(d)
    h_a = float(max(h_i, h_j))
    h_b = float(min(h_i, h_j))
    if d >= h_a + h_b:
        return 0.0
    delta = d / h_a
    q = h_b / h_a
    if delta == 0.0:
        brk = {0.0, 0.5, 1.0, 0.5 * q, q}
    else:
        brk = {0.0, 0.5, 1.0}
        for c in (0.5 * q - delta, q - delta, delta, delta - 0.5 * q, delta + 0.5 * q,
                  delta - q, delta + q):
            if 0.0 < c < 1.0:
                brk.add(c)
    pts = sorted(b for b in brk if 0.0 <= b <= 1.0)
    total = 0.0
    for l, r in zip(pts[:-1], pts[1:]):
        if r <= l:
            continue
        mid = 0.5 * (l + r)
        half = 0.5 * (r - l)
        for xk, wk in zip(_GL5_X, _GL5_W):
            s = mid + half * xk
            ws = float(w_unit(np.array([s]))[0])
            if ws == 0.0:
                continue
            if delta == 0.0:
                inner = 2.0 * float(w_unit(np.array([s / q]))[0])
            else:
                inner = (q * q / (delta * s)) * _int_u_w(abs(s - delta) / q, (s + delta) / q)
            total += wk * half * s * s * ws * inner
    return 2.0 * np.pi / h_b ** 3 * total


def overlap_g_many(d, h_i, h_j):
    """Vectorised wrapper over overlap_g (a Python loop; oracle speed is not a goal)."""
    d = np.asarray(d, dtype=np.float64).ravel()
    h_i = np.broadcast_to(np.asarray(h_i, dtype=np.float64), d.shape).ravel()
    h_j = np.broadcast_to(np.asarray(h_j, dtype=np.float64), d.shape).ravel()
    out = np.empty_like(d)
    for k in range(d.size):
        out[k] = overlap_g(d[k], h_i[k], h_j[k])
    return out


def _int_u_w_vec(lo, hi):
    """Vectorised _int_u_w: int_lo^hi u w(u) du elementwise (exact 3-point GL per piece)."""
    total = np.zeros(np.broadcast(lo, hi).shape)
    for a, b in ((0.0, 0.5), (0.5, 1.0)):
        l = np.maximum(lo, a)
        r = np.minimum(hi, b)
        span = np.maximum(r - l, 0.0)
        mid = 0.5 * (l + r)
        half = 0.5 * span
        acc = np.zeros_like(total)
        for xk, wk in zip(_GL3_X, _GL3_W):
            u = mid + half * xk
            acc += wk * u * w_unit(u)
        total += half * acc
    return total


def overlap_g_vec(d, h_i, h_j):
    """overlap_g for arrays of pairs; the same breakpoints and exact rules, vectorised.

    For every pair all ten candidate breakpoints {0, 1/2, 1, q/2-delta, q-delta,
    delta, delta +- q/2, delta +- q} are clipped to [0, 1] and sorted, giving up
    to eleven sub-intervals (empty ones contribute zero).
    """
    d = np.asarray(d, dtype=np.float64).ravel()
    h_i = np.broadcast_to(np.asarray(h_i, dtype=np.float64), d.shape).ravel()
    h_j = np.broadcast_to(np.asarray(h_j, dtype=np.float64), d.shape).ravel()
    h_a = np.maximum(h_i, h_j)
    h_b = np.minimum(h_i, h_j)
    delta = d / h_a
    q = h_b / h_a
    live = d < h_a + h_b
    cand = np.stack([np.zeros_like(d), np.full_like(d, 0.5), np.ones_like(d),
                     0.5 * q - delta, q - delta, delta, delta - 0.5 * q, delta + 0.5 * q,
                     delta - q, delta + q, 0.5 * q, q], axis=1)
    cand = np.sort(np.clip(cand, 0.0, 1.0), axis=1)
    total = np.zeros_like(d)
    zero_delta = delta == 0.0
    safe_delta = np.where(zero_delta, 1.0, delta)
    for k in range(cand.shape[1] - 1):
        l = cand[:, k]
        r = cand[:, k + 1]
        mid = 0.5 * (l + r)
        half = 0.5 * (r - l)
        for xk, wk in zip(_GL5_X, _GL5_W):
            s = mid + half * xk
            ws = w_unit(s)
            safe_s = np.where(s > 0.0, s, 1.0)
            inner = (q * q / (safe_delta * safe_s)) * _int_u_w_vec(np.abs(s - delta) / q, (s + delta) / q)
            inner = np.where(zero_delta, 2.0 * w_unit(s / q), inner)
            total += wk * half * s * s * ws * inner
    return np.where(live, 2.0 * np.pi / h_b ** 3 * total, 0.0)

"""Explicit Runge-Kutta pairs and step-size control, written from Section 2.2 and Appendix A of
arXiv:1810.10197.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Tableaus: exact fractions as printed in Appendix A (BS5 with the b-hat error estimator
  that Section 2.2 names, DP5) and the classical RK4 of Kutta.
* One attempt: stage inputs Y_i = u + h sum_{j<i} a_ij k_j, stage derivatives k_i = f(Y_i),
  the main solution u_new = u + h sum_j b_j k_j and the embedded difference
  e = u_new - v_new = h sum_j (b_j - bhat_j) k_j.  For a first-same-as-last pair the last
  row of A equals b, so u_new is the last stage input, and its derivative is the next
  step's k_1.
* Error norm (Section 2.2.1): sc = atol + rtol * max(|u_old|, |u_new|) per component and
  mode (complex modulus); err_j = sqrt( sum_k |e|^2 / sc^2 / n_modes ), err = max_j err_j,
  with n_modes = nx ny (nz/2+1), the number of stored frequencies.
* Controller (Section 2.2.1): h_new = h * min(dmax, max(dmin, delta * err^(-1/(q+1))))
  with delta = 0.8, dmax = 2, dmin = 0.01, q = 4 the embedded order.  err <= 1 accepts;
  otherwise the step is redone with h_new.  dmax = 1 for the step that follows a rejection.
  Readings (listed in the design notes): the last step is clipped to end exactly at t_end
  and h is the clipped step (a step h >= (t_end - t)(1 - 1e-10) counts as the last one, so
  fixed steps that divide the interval end on t_end despite rounding of t); a non-finite err
  rejects with factor dmin; err = 0 takes dmax.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction as Fr
from typing import Callable, List, Optional

import numpy as np


@dataclass(frozen=True)
class Tableau:
    name: str
    c: tuple
    A: tuple          # lower-triangular rows, A[i] has i entries
    b: tuple
    bhat: Optional[tuple]
    order: int
    embedded_order: Optional[int]
    fsal: bool

    @property
    def stages(self) -> int:
        return len(self.c)


def _row(*xs):
    return tuple(Fr(x) for x in xs)


# Classical fourth-order method of Kutta (1901).
RK4 = Tableau(
    name="RK4",
    c=_row(0, Fr(1, 2), Fr(1, 2), 1),
    A=(_row(), _row(Fr(1, 2)), _row(0, Fr(1, 2)), _row(0, 0, 1)),
    b=_row(Fr(1, 6), Fr(1, 3), Fr(1, 3), Fr(1, 6)),
    bhat=None, order=4, embedded_order=None, fsal=False,
)

# Bogacki-Shampine 5(4) pair, Appendix A (b-hat estimator).
BS5 = Tableau(
    name="BS5",
    c=_row(0, Fr(1, 6), Fr(2, 9), Fr(3, 7), Fr(2, 3), Fr(3, 4), 1, 1),
    A=(
        _row(),
        _row(Fr(1, 6)),
        _row(Fr(2, 27), Fr(4, 27)),
        _row(Fr(183, 1372), Fr(-162, 343), Fr(1053, 1372)),
        _row(Fr(68, 297), Fr(-4, 11), Fr(42, 143), Fr(1960, 3861)),
        _row(Fr(597, 22528), Fr(81, 352), Fr(63099, 585728), Fr(58653, 366080), Fr(4617, 20480)),
        _row(Fr(174197, 959244), Fr(-30942, 79937), Fr(8152137, 19744439), Fr(666106, 1039181),
             Fr(-29421, 29068), Fr(482048, 414219)),
        _row(Fr(587, 8064), 0, Fr(4440339, 15491840), Fr(24353, 124800), Fr(387, 44800),
             Fr(2152, 5985), Fr(7267, 94080)),
    ),
    b=_row(Fr(587, 8064), 0, Fr(4440339, 15491840), Fr(24353, 124800), Fr(387, 44800),
           Fr(2152, 5985), Fr(7267, 94080), 0),
    bhat=_row(Fr(2479, 34992), 0, Fr(123, 416), Fr(612941, 3411720), Fr(43, 1440), Fr(2272, 6561),
              Fr(79937, 1113912), Fr(3293, 556956)),
    order=5, embedded_order=4, fsal=True,
)

# Dormand-Prince 5(4) pair, Appendix A.
DP5 = Tableau(
    name="DP5",
    c=_row(0, Fr(1, 5), Fr(3, 10), Fr(4, 5), Fr(8, 9), 1, 1),
    A=(
        _row(),
        _row(Fr(1, 5)),
        _row(Fr(3, 40), Fr(9, 40)),
        _row(Fr(44, 45), Fr(-56, 15), Fr(32, 9)),
        _row(Fr(19372, 6561), Fr(-25360, 2187), Fr(64448, 6561), Fr(-212, 729)),
        _row(Fr(9017, 3168), Fr(-355, 33), Fr(46732, 5247), Fr(49, 176), Fr(-5103, 18656)),
        _row(Fr(35, 384), 0, Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84)),
    ),
    b=_row(Fr(35, 384), 0, Fr(500, 1113), Fr(125, 192), Fr(-2187, 6784), Fr(11, 84), 0),
    bhat=_row(Fr(5179, 57600), 0, Fr(7571, 16695), Fr(393, 640), Fr(-92097, 339200),
              Fr(187, 2100), Fr(1, 40)),
    order=5, embedded_order=4, fsal=True,
)

TABLEAUS = {"RK4": RK4, "BS5": BS5, "DP5": DP5}

# Controller constants of Section 2.2.1.
DELTA = 0.8
DELTA_MAX = 2.0
DELTA_MIN = 0.01


def rk_attempt(f: Callable, u: np.ndarray, h: float, tab: Tableau, k1: Optional[np.ndarray] = None):
    """One Runge-Kutta attempt from u with step h.

    Returns (u_new, e, ks) where e = h sum_j (b_j - bhat_j) k_j (None without an embedded
    pair) and ks the stage derivatives.  k1 = f(u) may be passed in (first same as last).
    For an FSAL pair u_new is the last stage input Y_s (its row of A equals b).
    """
    s = tab.stages
    ks: List[np.ndarray] = []
    Y = u
    for i in range(s):
        if i == 0:
            Y = u
            ks.append(f(u) if k1 is None else k1)
            continue
        acc = None
        for j, a in enumerate(tab.A[i]):
            if a != 0:
                term = float(a) * ks[j]
                acc = term if acc is None else acc + term
        Y = u + h * acc if acc is not None else u
        ks.append(f(Y))
    if tab.fsal:
        u_new = Y
    else:
        acc = None
        for j, bj in enumerate(tab.b):
            if bj != 0:
                term = float(bj) * ks[j]
                acc = term if acc is None else acc + term
        u_new = u + h * acc
    e = None
    if tab.bhat is not None:
        acc = None
        for j, (bj, bh) in enumerate(zip(tab.b, tab.bhat)):
            d = bj - bh
            if d != 0:
                term = float(d) * ks[j]
                acc = term if acc is None else acc + term
        e = h * acc
    return u_new, e, ks


def error_norm(u_old: np.ndarray, u_new: np.ndarray, e: np.ndarray, atol: float, rtol: float,
               nmodes: int) -> float:
    """err = max_j sqrt( (1/nmodes) sum_k (|e_jk| / sc_jk)^2 ), sc = atol + rtol max(|u_old|,|u_new|).

    Axis 0 indexes the components j; the sum runs over every other axis.  A mode whose
    embedded error is exactly zero contributes zero, whatever its scale: with a purely
    relative tolerance (atol = 0) a mode that is zero in both solutions has sc = 0, and the
    quotient 0/0 is read as 0 (Section 2.2.1 scales the error; it does not define 0/0).  A
    nonzero error over sc = 0 stays infinite.
    """
    sc = atol + rtol * np.maximum(np.abs(u_old), np.abs(u_new))
    ae = np.abs(e)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(ae == 0.0, 0.0, ae / sc)
    ncomp = e.shape[0]
    errs = [math.sqrt(float(np.sum(r[j] ** 2)) / nmodes) for j in range(ncomp)]
    return max(errs)


def controller_factor(err: float, after_reject: bool) -> float:
    """min(dmax, max(dmin, 0.8 err^(-1/5))); dmax = 1 right after a rejection."""
    dmax = 1.0 if after_reject else DELTA_MAX
    if not math.isfinite(err):
        return DELTA_MIN
    if err == 0.0:
        return dmax
    return min(dmax, max(DELTA_MIN, DELTA * err ** (-1.0 / (BS5.embedded_order + 1))))


# PI controller (Gustafsson; Hairer & Wanner II, Sec. IV.2): the paper names it as future work
# (Section 4).  Exponents alpha = 0.7/(q+1), beta = 0.4/(q+1), q = 4.
PI_ALPHA = 0.7 / 5.0
PI_BETA = 0.4 / 5.0


def pi_factor(err: float, err_prev: float, after_reject: bool) -> float:
    """min(dmax, max(dmin, 0.8 err^(-alpha) err_prev^beta)) for an accepted step."""
    dmax = 1.0 if after_reject else DELTA_MAX
    if err == 0.0:
        return dmax
    return min(dmax, max(DELTA_MIN, DELTA * err ** (-PI_ALPHA) * err_prev ** PI_BETA))


@dataclass
class Result:
    u: np.ndarray
    t: float
    h_next: float
    n_rhs: int = 0
    n_acc: int = 0
    n_rej: int = 0
    status: str = "ok"
    history: list = field(default_factory=list)   # (t_start, h, err, accepted)


def integrate(f: Callable, u0: np.ndarray, t0: float, t_end: float, method: str, h0: float,
              rtol: float = 1e-6, atol: float = 1e-6, nmodes: Optional[int] = None,
              max_rejects: int = 30, max_steps: int = 10 ** 7,
              on_accept: Optional[Callable] = None, controller="I",
              post_step: Optional[Callable] = None) -> Result:
    """Integrate u' = f(u) from t0 to t_end.

    method: "RK4" (fixed h0), "BS5_FIXED" (fixed h0, error logged), "BS5_ADAPTIVE",
    "DP5_FIXED", "DP5_ADAPTIVE".  The last step is clipped to land on t_end.
    controller (adaptive methods): "I" (Section 2.2.1), "PI", or ("MLP", params): after an
    accepted step the PI factor, or the network's bounded correction of it, replaces the
    Section 2.2.1 factor; the MLP controller falls back to the PI factor for its first 3
    accepted steps and when the network's output is not finite; a rejected attempt always
    takes the Section 2.2.1 factor.
    post_step(u_old, u_new) -> u, if given, replaces the state after every accepted step (the
    band rescale forcing of Section 3.3.1); when it returns a new array the derivative carried
    over by a first-same-as-last pair no longer belongs to the state and k_1 is evaluated afresh.
    """
    from . import mlp as _mlp
    tabname, _, mode = method.partition("_")
    tab = TABLEAUS[tabname]
    adaptive = mode == "ADAPTIVE"
    if nmodes is None:
        nmodes = int(np.prod(u0.shape[1:]))
    res = Result(u=u0.copy(), t=float(t0), h_next=float(h0))
    u = res.u
    t = res.t
    h = float(h0)
    k1 = None
    after_reject = False
    rejects_in_row = 0
    steps = 0
    err_prev = 1.0
    hist = []            # accepted (err, h, rejections before it), newest first
    rej_since = 0
    while t < t_end and steps < max_steps:
        steps += 1
        # last step: land exactly on t_end (also when h falls short of it by rounding only)
        clipped = h >= (t_end - t) * (1.0 - 1e-10)
        h_step = t_end - t if clipped else h
        if h_step < 1e-12 * max(1.0, abs(t)):
            res.status = "step_underflow"
            break
        u_new, e, ks = rk_attempt(f, u, h_step, tab, k1)
        res.n_rhs += tab.stages - (1 if k1 is not None else 0)
        err = error_norm(u, u_new, e, atol, rtol, nmodes) if e is not None else 0.0
        if adaptive:
            accepted = math.isfinite(err) and err <= 1.0
            fac = controller_factor(err, after_reject)
            is_mlp = isinstance(controller, tuple) and controller[0] == "MLP"
            if accepted and (controller == "PI" or is_mlp):
                fac = pi_factor(err, err_prev, after_reject)
            if accepted and is_mlp:
                hist = [(err, h_step, rej_since)] + hist[:4]
                if len(hist) >= 4:
                    prop = _mlp.propose_factor(controller[1], hist, err_prev)
                    if prop is not None:
                        fac = min(1.0, prop) if after_reject else prop
            h_new = h_step * fac
        else:
            accepted = True
            h_new = h
        res.history.append((t, h_step, err, accepted))
        if accepted:
            t = t_end if clipped else t + h_step
            k1 = ks[-1] if tab.fsal else None
            if post_step is not None:
                u_post = post_step(u, u_new)
                if u_post is not u_new:      # a changed state needs a fresh k_1
                    k1 = None
                u_new = u_post
            u = u_new
            after_reject = False
            rejects_in_row = 0
            rej_since = 0
            if err > 0:
                err_prev = err
            res.n_acc += 1
            if on_accept is not None:
                on_accept(t, u, ks[-1] if tab.fsal else None)
        else:
            after_reject = True
            k1 = ks[0] if tab.fsal else None
            rejects_in_row += 1
            rej_since += 1
            res.n_rej += 1
            if rejects_in_row > max_rejects:
                res.status = "max_rejects"
                break
        h = h_new
    res.u, res.t, res.h_next = u, t, h
    return res

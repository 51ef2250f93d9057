"""Fourier-lattice helpers of the oracle: k-mode sets, the RBE normaliser H,
the sampling distribution h(k), the RBE k-sampler and the diagonal constants.

ORACLE: test infrastructure (see oracle/__init__.py). Plain numpy, FP64.

Paper references (Gan, Gao, Liang, Xu, arXiv 2403.01521):
  * lattice K^2 = 2pi/Lx Z x 2pi/Ly Z and the k cutoff |k| <= k_c
    (proof of Prop. 2.2; Section 2.3);
  * h(k) = e^{-k^2/(4 alpha^2)}/H, H = sum_{k != 0} e^{-k^2/(4 alpha^2)}
    (Eq. 4.5) and its Poisson-summation form (Eq. 4.6, read with alpha^2:
    H = (alpha^2 Lx Ly/pi) sum_n e^{-alpha^2 (n_x^2 Lx^2 + n_y^2 Ly^2)} - 1);
  * the RBE estimator U* = (H/P) sum_eta phi~^RB(k_eta) with
    phi~^RB(k) = e^{k^2/(4 alpha^2)} phi~(k) (Eqs. 4.7-4.9).

The k-sampler draws i.i.d. lattice vectors from h. Because h factorises into
two one-dimensional discrete Gaussians p(m) ~ e^{-pi^2 m^2/(alpha L)^2}, each
component is drawn by inversion of its cumulative table and the origin is
rejected. The paper's own sampler, the independence Metropolis chain of
App. G (rounded-normal proposals, optional downsampling), is
metropolis_modes. Random words come from the counter-based generator Philox4x64-10
(Salmon, Moraes, Dror, Shaw, SC'11), written here from its definition.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, erfc

PI = math.pi

# ---------------------------------------------------------------- k modes


def kcut_for_tail(alpha: float, tail: float) -> float:
    """k_c with e^{-k_c^2/(4 alpha^2)} = tail, i.e. k_c = 2 alpha sqrt(ln(1/tail))."""
    return 2.0 * alpha * math.sqrt(math.log(1.0 / tail))


def full_modes(Lx: float, Ly: float, kc: float):
    """All lattice vectors k != 0 with |k|^2 <= k_c^2 (both k and -k).

    Returns integer arrays (mx, my). |k|^2 is evaluated as
    (2 pi mx/Lx)^2 + (2 pi my/Ly)^2 in FP64.
    """
    mxm = int(math.floor(kc * Lx / (2 * PI))) + 1
    mym = int(math.floor(kc * Ly / (2 * PI))) + 1
    mx, my = np.meshgrid(np.arange(-mxm, mxm + 1), np.arange(-mym, mym + 1),
                         indexing="ij")
    mx = mx.ravel()
    my = my.ravel()
    kx = 2 * PI * mx / Lx
    ky = 2 * PI * my / Ly
    keep = (kx * kx + ky * ky <= kc * kc) & ~((mx == 0) & (my == 0))
    return mx[keep].astype(np.int64), my[keep].astype(np.int64)


def kvec(mx, my, Lx, Ly):
    kx = 2 * PI * np.asarray(mx, float) / Lx
    ky = 2 * PI * np.asarray(my, float) / Ly
    return kx, ky, np.sqrt(kx * kx + ky * ky)


# ---------------------------------------------------------------- H


def H_direct(alpha: float, Lx: float, Ly: float) -> float:
    """H = sum_{k != 0} e^{-k^2/(4 alpha^2)} by direct lattice summation."""
    def axis(L):
        # terms e^{-pi^2 m^2/(alpha L)^2}; stop once they underflow 1e-40
        m = np.arange(0, int(10 * alpha * L / PI) + 10)
        t = np.exp(-(PI * m / (alpha * L)) ** 2)
        return t[0] + 2.0 * t[1:].sum()
    return float(axis(Lx) * axis(Ly) - 1.0)


def H_poisson(alpha: float, Lx: float, Ly: float, alpha_power: int = 2) -> float:
    """Poisson-summation form of H (Eq. 4.6).

    alpha_power=2 is the reading this project uses; alpha_power=1 reproduces
    the form as printed (kept only so a test can show it disagrees with the
    direct sum).
    """
    a = alpha ** alpha_power

    def axis(L):
        n = np.arange(1, 20)
        return 1.0 + 2.0 * np.exp(-a * (n * L) ** 2).sum()
    return float(a * Lx * Ly / PI * axis(Lx) * axis(Ly) - 1.0)


# ---------------------------------------------------------------- constants


def diag_kspace(alpha, Lx, Ly, mx, my):
    """sum over the given modes of (pi/(Lx Ly)) erfc(k/(2 alpha))/k.

    This is the j = i part of U_l^k per unit Q = sum q_i^2 (Eq. 3.20). The
    potential gets twice this times q_i.
    """
    from scipy.special import erfc
    _, _, k = kvec(mx, my, Lx, Ly)
    return float((PI / (Lx * Ly) * erfc(k / (2 * alpha)) / k).sum())


def diag_kspace_all(alpha, Lx, Ly, rel: float = 1e-18):
    """The same diagonal sum over the whole lattice (k != 0), used by the
    random-batch estimator, whose sample covers every k."""
    from scipy.special import erfc
    # erfc(x) < 1e-18 beyond x ~ 6.1, so |k| <= 14 alpha is ample
    kc = 14.0 * alpha
    mx, my = full_modes(Lx, Ly, kc)
    return diag_kspace(alpha, Lx, Ly, mx, my)


def diag_kzero(alpha, Lx, Ly):
    """j = i part of U_l^0 per unit Q: -(pi/(Lx Ly)) g0(0), g0(0)=1/(alpha sqrt(pi)).

    Eq. 3.25 prints the constant as -pi Q/(alpha Lx Ly); taking the j = i term
    of Eq. 2.16 gives -sqrt(pi) Q/(alpha Lx Ly), which is what is used.
    """
    return -(PI / (Lx * Ly)) / (alpha * math.sqrt(PI))


def self_energy_coef(alpha):
    """U_self per unit Q: (1/2) sum_i q_i phi_self^i / q_i^2 = alpha/sqrt(pi) (Eq. 2.12)."""
    return alpha / math.sqrt(PI)


# ---------------------------------------------------------------- Philox4x64-10

_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B
_MASK32 = np.uint64(0xFFFFFFFF)


def _mulhilo64(a: np.ndarray, b: int):
    """Full 64x64 -> 128-bit product of uint64 arrays a and constant b."""
    a = np.asarray(a, np.uint64)
    b0 = np.uint64(b & 0xFFFFFFFF)
    b1 = np.uint64(b >> 32)
    a0 = a & _MASK32
    a1 = a >> np.uint64(32)
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> np.uint64(32)) + (p01 & _MASK32) + (p10 & _MASK32)
    lo = (p00 & _MASK32) | ((mid & _MASK32) << np.uint64(32))
    hi = p11 + (p01 >> np.uint64(32)) + (p10 >> np.uint64(32)) + (mid >> np.uint64(32))
    return hi, lo


def philox4x64_10(ctr, key):
    """Philox4x64 with 10 rounds. ctr: (..., 4) uint64, key: (..., 2) uint64."""
    with np.errstate(over="ignore"):
        c = [np.asarray(ctr[..., i], np.uint64).copy() for i in range(4)]
        k0 = np.asarray(key[..., 0], np.uint64).copy()
        k1 = np.asarray(key[..., 1], np.uint64).copy()
        for _ in range(10):
            hi0, lo0 = _mulhilo64(c[0], _M0)
            hi1, lo1 = _mulhilo64(c[2], _M1)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            k0 = k0 + np.uint64(_W0)
            k1 = k1 + np.uint64(_W1)
    return np.stack(c, axis=-1)


# ---------------------------------------------------------------- k sampler

SAMPLER_TAG = 0x52424531          # fourth counter word of every draw
TAIL_SQRT = 6.4380                # components with pi^2 m^2/(alpha L)^2 > 41.4 are dropped


def axis_mmax(alpha: float, L: float) -> int:
    return int(math.floor(TAIL_SQRT * alpha * L / PI)) + 1


def axis_cdf(alpha: float, L: float):
    """Cumulative table of p(m) ~ e^{-pi^2 m^2/(alpha L)^2}, m = -mmax..mmax."""
    mmax = axis_mmax(alpha, L)
    m = np.arange(-mmax, mmax + 1)
    wgt = np.exp(-(PI * m / (alpha * L)) ** 2)
    c = np.cumsum(wgt)
    return c / c[-1], mmax


def uniform53(word: np.ndarray) -> np.ndarray:
    """Top 53 bits of a 64-bit word as a double in [0, 1)."""
    return (np.asarray(word, np.uint64) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def sample_modes(P: int, seed: int, call: int, alpha: float, Lx: float, Ly: float,
                 stream: int = 0):
    """P i.i.d. lattice vectors from h(k) (origin excluded).

    Sample eta, attempt a uses Philox4x64-10 with counter
    (eta, a, call, TAG + stream * 2^32) and key (seed, 0); `stream` separates
    independent systems drawn in the same call (one per slab of a batch).
    Words 0,1 give (mx, my); if that is the origin, words 2,3 are tried; if
    that is the origin too, the next attempt is used.
    """
    cx, mxm = axis_cdf(alpha, Lx)
    cy, mym = axis_cdf(alpha, Ly)
    out_x = np.zeros(P, np.int64)
    out_y = np.zeros(P, np.int64)
    todo = np.arange(P)
    attempt = 0
    while todo.size:
        ctr = np.zeros((todo.size, 4), np.uint64)
        ctr[:, 0] = todo
        ctr[:, 1] = attempt
        ctr[:, 2] = np.uint64(call)
        ctr[:, 3] = np.uint64(SAMPLER_TAG + (int(stream) << 32))
        key = np.zeros((todo.size, 2), np.uint64)
        key[:, 0] = np.uint64(seed)
        wds = philox4x64_10(ctr, key)
        done = np.zeros(todo.size, bool)
        for pair in ((0, 1), (2, 3)):
            ix = np.searchsorted(cx, uniform53(wds[:, pair[0]]), side="right")
            iy = np.searchsorted(cy, uniform53(wds[:, pair[1]]), side="right")
            mx = ix - mxm
            my = iy - mym
            ok = ~done & ~((mx == 0) & (my == 0))
            out_x[todo[ok]] = mx[ok]
            out_y[todo[ok]] = my[ok]
            done |= ok
        todo = todo[~done]
        attempt += 1
    return out_x, out_y


MH_TAG = 0x4D484731               # fourth counter word of the Metropolis draws


def round_half_away(x):
    """Nearest integer, halves away from zero (C's round())."""
    x = np.asarray(x, float)
    return (np.sign(x) * np.floor(np.abs(x) + 0.5)).astype(np.int64)


def proposal_pmf(m, alpha: float, L: float):
    """q(m) of App. G: the probability that a normal of mean 0 and variance
    (alpha L)^2/(2 pi^2) rounds to the integer m; erf(pi/(2 alpha L)) at
    m = 0, else half the difference of erf at pi(2|m| +- 1)/(2 alpha L),
    written with erfc so that the far tail keeps its relative accuracy."""
    a = PI / (2.0 * alpha * L)
    m = np.abs(np.asarray(m, float))
    return np.where(m == 0, erf(a), 0.5 * (erfc(a * (2 * m - 1)) - erfc(a * (2 * m + 1))))


def mh_log_weight(mx, my, alpha: float, Lx: float, Ly: float):
    """log[H(m)/q(m)] up to a constant (H(m) = h(k) of Eq. 4.5 unnormalised):
    the acceptance ratio of App. G is exp of the difference of two of these.
    Both factorise over the axes: the x part plus the y part."""
    def axis(m, L):
        return -(PI * np.asarray(m, float) / (alpha * L)) ** 2 - np.log(proposal_pmf(m, alpha, L))
    return axis(mx, Lx) + axis(my, Ly)


def mh_proposal(w0, w1, alpha: float, Lx: float, Ly: float):
    """Proposals of App. G from pairs of 64-bit words (arrays): a pair of
    normals by the Box-Muller transform (u1 = 1 - uniform53(w0) in (0, 1],
    u2 = uniform53(w1)), scaled to the standard deviations
    alpha L/(sqrt(2) pi), rounded to the nearest integers."""
    u1 = 1.0 - uniform53(w0)
    u2 = uniform53(w1)
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * PI * u2
    sx = alpha * Lx / (math.sqrt(2.0) * PI)
    sy = alpha * Ly / (math.sqrt(2.0) * PI)
    return round_half_away(sx * r * np.cos(th)), round_half_away(sy * r * np.sin(th))


def _mh_words(i0, i1, call, seed, stream):
    i0 = np.atleast_1d(np.asarray(i0, np.uint64))
    ctr = np.zeros((i0.size, 4), np.uint64)
    ctr[:, 0] = i0
    ctr[:, 1] = np.uint64(i1)
    ctr[:, 2] = np.uint64(call)
    ctr[:, 3] = np.uint64(MH_TAG + (int(stream) << 32))
    key = np.zeros((i0.size, 2), np.uint64)
    key[:, 0] = np.uint64(seed)
    return philox4x64_10(ctr, key)


def metropolis_modes(P: int, seed: int, call: int, alpha: float, Lx: float, Ly: float,
                     stream: int = 0, thin: int = 1, return_rate: bool = False):
    """P lattice vectors from h(k) by the independence Metropolis chain of
    App. G, keeping every thin-th state (the downsampling rate).

    Start: attempt a = 0, 1, ... (Philox counter (a, 1, call, MH_TAG +
    stream 2^32), key (seed, 0)) gives two proposals, from words (0, 1) and
    (2, 3); the first that is not the origin is the initial state; after 64
    attempts the state is (1, 0). Step eta = 1 .. P thin uses counter
    (eta - 1, 0, call, MH_TAG + stream 2^32): words 0, 1 give the proposal,
    word 2 the uniform u; the origin is rejected (h = 0 there), any other
    proposal is accepted when u < H(new) q(old) / (H(old) q(new)), tested
    as d >= 0 or log u < d with d the log of that ratio. The sample after
    step j thin is the j-th output. The proposals do not depend on the state
    (App. G), so they are drawn for all steps first; the chain itself runs
    step by step."""
    state = (1, 0)
    w = _mh_words(np.arange(64), 1, call, seed, stream)
    ax, ay = mh_proposal(w[:, 0], w[:, 1], alpha, Lx, Ly)
    bx, by = mh_proposal(w[:, 2], w[:, 3], alpha, Lx, Ly)
    for a in range(64):
        if ax[a] != 0 or ay[a] != 0:
            state = (int(ax[a]), int(ay[a]))
            break
        if bx[a] != 0 or by[a] != 0:
            state = (int(bx[a]), int(by[a]))
            break
    n = P * thin
    w = _mh_words(np.arange(n), 0, call, seed, stream)
    px, py = mh_proposal(w[:, 0], w[:, 1], alpha, Lx, Ly)
    with np.errstate(divide="ignore"):
        logu = np.log(uniform53(w[:, 2]))          # -inf for u = 0
    origin = (px == 0) & (py == 0)
    lwp = mh_log_weight(px, py, alpha, Lx, Ly)    # not used at the origin
    lw = float(mh_log_weight(state[0], state[1], alpha, Lx, Ly))
    out_x = np.zeros(P, np.int64)
    out_y = np.zeros(P, np.int64)
    accepted = 0
    for eta in range(1, n + 1):
        t = eta - 1
        if not origin[t]:
            d = float(lwp[t]) - lw
            if d >= 0.0 or float(logu[t]) < d:
                state, lw = (int(px[t]), int(py[t])), float(lwp[t])
                accepted += 1
        if eta % thin == 0:
            out_x[eta // thin - 1], out_y[eta // thin - 1] = state
    if return_rate:
        return out_x, out_y, accepted / n
    return out_x, out_y


def h_pmf(alpha, Lx, Ly, mx, my):
    """h at lattice points, normalised by H (exact, Eq. 4.5)."""
    H = H_direct(alpha, Lx, Ly)
    _, _, k = kvec(mx, my, Lx, Ly)
    return np.exp(-k * k / (4 * alpha * alpha)) / H

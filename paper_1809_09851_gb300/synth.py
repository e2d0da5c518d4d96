"""Seeded synthetic inputs for the Euler building blocks.

This module draws random numbers and nothing else: it holds none of the
building blocks' arithmetic (no EOS, no conversion between variable sets),
so that the CUDA path and the FP64 CPU oracle can both be fed from it without
sharing any of the method's code.  Fields are returned in primitive form
V = (rho, v_1..v_D, p) (paper section 2.2, Fig. 9); each side converts them to
conservative form with its own cons-from-prim implementation.

Streams are counter-based (numpy Philox keyed by (seed, plane)), so the first
n values of a plane do not depend on how many are drawn: a small case is a
prefix of the full-size case.

Workloads (sizes and distributions of the paper's mini-app, section 3, and of
the benchmark configurations):
  * ``euler1d``   : D=1, rho ~ U[0.5, 2], u ~ N(0, 1), p ~ U[0.5, 2]
  * ``euler3d``   : D=3, rho ~ U[0.1, 10], v_i ~ N(0, sd=2), p ~ U[0.1, 10];
                    W ~ N(0, 1) (5 planes) for the characteristic transform
  * ``precision`` : ``euler3d`` with 5% of points near vacuum
                    (rho, p ~ U[1e-4, 1e-3]) and 5% at Mach M ~ U[10, 50]
                    given as a Mach number and a unit direction per point
  * ``cotangent`` : G ~ N(0, 1), nv planes (upstream gradients of a VJP)
  * ``euler_eos`` : D=1..3 under a general EOS: rho ~ U[0.2, 4], v_i ~ N(0, 1),
                    p ~ U[0.1, 10], with the nondimensional EOS parameter sets
                    ``EOS_NASG`` and ``EOS_VDW`` (1 - b rho >= 0.6 and c^2 > 0
                    on the whole range)
  * ``serving``   : request stream and smooth periodic initial data for the
                    finite-volume serving loop
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED = 1809
SEED_W = 9851


def _rng(seed: int, plane: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, plane])))


def uniform(n: int, lo: float, hi: float, seed: int, plane: int) -> np.ndarray:
    return _rng(seed, plane).uniform(lo, hi, size=n)


def normal(n: int, sd: float, seed: int, plane: int) -> np.ndarray:
    return _rng(seed, plane).normal(0.0, sd, size=n)


def euler_primitive(n: int, D: int, rho_rng, v_sd: float, p_rng, seed: int = SEED):
    """Primitive planes [rho, v_1..v_D, p] with independent per-plane streams."""
    rho = uniform(n, rho_rng[0], rho_rng[1], seed, 0)
    vs = [normal(n, v_sd, seed, 1 + k) for k in range(D)]
    p = uniform(n, p_rng[0], p_rng[1], seed, 10)
    return [rho, *vs, p]


def euler1d(n: int, seed: int = SEED):
    """1D Euler: rho ~ U[0.5,2], u ~ N(0,1), p ~ U[0.5,2]."""
    return euler_primitive(n, 1, (0.5, 2.0), 1.0, (0.5, 2.0), seed)


def euler3d(n: int, seed: int = SEED, D: int = 3):
    """3D (or 2D) Euler: rho ~ U[0.1,10], v_i ~ N(0, sd 2), p ~ U[0.1,10]."""
    return euler_primitive(n, D, (0.1, 10.0), 2.0, (0.1, 10.0), seed)


# Nondimensional parameter sets of the general-EOS workload (section 2.2,
# "Equations of state"): a Noble-Abel stiffened gas and a van der Waals gas.
EOS_NASG = {"kind": "nasg", "gamma": 1.6, "p_inf": 1.0, "b": 0.1, "q": -0.3, "cv": 2.0}
EOS_VDW = {"kind": "vdw", "gamma": 1.4, "a": 0.05, "b": 0.1, "cv": 2.5}


def euler_eos(n: int, D: int = 3, seed: int = SEED):
    """General-EOS states: rho ~ U[0.2, 4], v_i ~ N(0, 1), p ~ U[0.1, 10]."""
    return euler_primitive(n, D, (0.2, 4.0), 1.0, (0.1, 10.0), seed)


def char_weights(n: int, nv: int = 5, seed: int = SEED_W):
    """W ~ N(0,1), nv planes (input of the characteristic transform)."""
    return [normal(n, 1.0, seed, 20 + k) for k in range(nv)]


def cotangent(n: int, nv: int = 5, seed: int = SEED_W + 1):
    """G ~ N(0,1), nv planes (upstream gradient of the flux VJP)."""
    return [normal(n, 1.0, seed, 40 + k) for k in range(nv)]


@dataclass
class PrecisionCase:
    V: list            # primitive planes; velocity is 0 at the high-Mach points
    vacuum: np.ndarray  # bool mask of the near-vacuum points
    mach: np.ndarray   # Mach number at the high-Mach points, 0 elsewhere
    direction: list    # unit direction (3 planes) of the high-Mach velocity


def precision(n: int, seed: int = SEED, frac_vacuum: float = 0.05, frac_mach: float = 0.05):
    """euler3d fields with 5% near-vacuum and 5% high-Mach points.

    The high-Mach velocity is v = M c n with c the local sound speed; that
    product is formed by the caller with its own EOS, so this module only
    returns M and the unit vector n.
    """
    V = euler3d(n, seed)
    sel = uniform(n, 0.0, 1.0, seed, 50)
    vacuum = sel < frac_vacuum
    fast = (sel >= frac_vacuum) & (sel < frac_vacuum + frac_mach)
    nvac = int(vacuum.sum())
    V[0][vacuum] = uniform(nvac, 1e-4, 1e-3, seed, 51)
    V[4][vacuum] = uniform(nvac, 1e-4, 1e-3, seed, 52)
    mach = np.zeros(n)
    nf = int(fast.sum())
    mach[fast] = uniform(nf, 10.0, 50.0, seed, 53)
    g = [normal(nf, 1.0, seed, 54 + k) for k in range(3)]
    norm = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    direction = [np.zeros(n) for _ in range(3)]
    for k in range(3):
        direction[k][fast] = g[k] / norm
        V[1 + k][fast] = 0.0
    return PrecisionCase(V=V, vacuum=vacuum, mach=mach, direction=direction)


# ---------------------------------------------------------------------------
# Serving workload
# ---------------------------------------------------------------------------

@dataclass
class Request:
    rid: int
    arrival: float  # seconds from the start of the stream
    n: int          # cells per side of the periodic n^3 grid
    steps: int      # explicit time steps to run
    seed: int


def request_stream(count: int, rate: float = 2000.0, n_lo: int = 16, n_hi: int = 192,
                   steps_lo: int = 10, steps_hi: int = 200, seed: int = SEED):
    """Poisson arrivals (mean `rate` per second), n log-uniform in [n_lo, n_hi]
    (rounded), steps uniform in {steps_lo..steps_hi}."""
    gaps = _rng(seed, 60).exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    ln = _rng(seed, 61).uniform(math.log(n_lo), math.log(n_hi), size=count)
    ns = np.clip(np.rint(np.exp(ln)).astype(np.int64), n_lo, n_hi)
    steps = _rng(seed, 62).integers(steps_lo, steps_hi + 1, size=count)
    return [Request(i, float(t[i]), int(ns[i]), int(steps[i]), seed * 7919 + i)
            for i in range(count)]


def smooth_params(seed: int):
    """Wave vectors k (3x3 ints in 1..3), phases and amplitudes of the three
    sinusoids of the rho (plane 0) and p (plane 1) perturbations."""
    out = []
    for plane in (0, 1):
        r = _rng(seed, 70 + plane)
        k = r.integers(1, 4, size=(3, 3))
        ph = r.uniform(0.0, 2.0 * math.pi, size=3)
        a = r.uniform(0.5, 1.0, size=3)
        out.append((k, ph, a))
    return out


def smooth_perturbation(n: int, seed: int, amplitude: float = 0.1):
    """rho and p planes for one periodic n^3 grid: 1 + amplitude * g(x) with g a
    sum of 3 seeded low-wavenumber sinusoids scaled to max |g| = 1; v = 0.

    Returns [rho, v_x, v_y, v_z, p] (primitive, x fastest).
    """
    x = (np.arange(n) + 0.5) / n
    X = x[None, None, :]
    Y = x[None, :, None]
    Z = x[:, None, None]
    out = []
    for k, ph, a in smooth_params(seed):
        g = np.zeros((n, n, n))
        for m in range(3):
            g = g + a[m] * np.sin(2 * math.pi * (k[m, 0] * X + k[m, 1] * Y + k[m, 2] * Z) + ph[m])
        g = g / np.abs(g).max()
        out.append((1.0 + amplitude * g).reshape(-1))
    zero = np.zeros(n ** 3)
    return [out[0], zero, zero.copy(), zero.copy(), out[1]]

"""Seeded synthetic inputs for the L-HWENO hot path.

This module holds only problem set-up: grids, initial data (with their exact
derivatives), boundary-condition names and the seeded draws of the batched
Riemann workload. It contains none of the scheme's arithmetic, imports neither
the CUDA library nor the oracle, and is the one module both sides share.

Boundary conditions are named by strings ("periodic", "outflow",
"reflective", "inflow", "dmr_bottom", "dmr_top"); each side maps them to its
own codes.

Random draws use splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds; a double in [0, 1) is the top 53 bits
times 2^-53.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator (see module docstring)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def choice(self, items):
        return items[self.next_u64() % len(items)]


@dataclass
class Workload:
    """A problem instance (or a ragged batch of 1D instances).

    Arrays are FP64 and laid out [instance][component][j][i] with i
    contiguous: U, V (= U_x) and, in 2D, W (= U_y). For a batch, instance k
    occupies m * nx[k] consecutive values starting at m * offsets[k].
    """
    name: str
    equation: str                 # "burgers", "euler" or "buckley" (1D)
    dim: int
    nx: List[int]                 # points per instance (1D) or [nx] (2D)
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    t_end: float
    bc: Tuple[str, str, str, str]  # x-low, x-high, y-low, y-high
    U: np.ndarray
    V: np.ndarray
    W: Optional[np.ndarray] = None
    gas_gamma: float = 1.4
    inflow: Tuple[float, ...] = (0.0, 0.0, 0.0, 0.0)   # conserved imposed state
    pre: Tuple[float, ...] = (0.0, 0.0, 0.0, 0.0)      # DMR pre-shock state
    dmr_x0: float = 1.0 / 6.0
    dmr_speed: float = 10.0
    dmr_angle: float = math.pi / 3.0
    dt_mode: str = "cfl"          # "cfl" (dt ~ dx) or "accuracy" (dt ~ dx^{5/3})
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return (3 if self.dim == 1 else 4) if self.equation == "euler" else 1

    @property
    def batch(self) -> int:
        return len(self.nx) if self.dim == 1 else 1

    @property
    def points(self) -> int:
        return int(sum(self.nx)) if self.dim == 1 else self.nx[0] * self.ny

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.nx)[:-1]]).astype(np.int64)

    def instance(self, k: int):
        """Views (U, V) of instance k of a 1D batch, shape (m, nx[k])."""
        m, n, o = self.m, self.nx[k], int(self.offsets[k])
        return (self.U[m * o:m * (o + n)].reshape(m, n),
                self.V[m * o:m * (o + n)].reshape(m, n))


def centers(lo: float, hi: float, n: int) -> np.ndarray:
    """Cell centres x_i = lo + (i + 1/2) dx of a uniform grid of n points."""
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * ((hi - lo) / n)


def euler_conserved(rho, u, p, gamma, v=None):
    """Conserved (rho, rho u[, rho v], E) from primitives, E = p/(g-1) + rho|u|^2/2."""
    rho, u, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, p))
    if v is None:
        return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])
    v = np.asarray(v, dtype=np.float64)
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


# ---------------------------------------------------------------------------
# 1D scalar: Burgers u_t + (u^2/2)_x = 0 on [0, 2], periodic, u0 = 0.5 + sin(pi x)
# (Examples 3.1 and 3.3).
# ---------------------------------------------------------------------------
def burgers1d_sine(n: int = 400, t_end: float = 1.5 / math.pi, dt_mode: str = "cfl") -> Workload:
    x = centers(0.0, 2.0, n)
    U = (0.5 + np.sin(np.pi * x)).reshape(1, n)
    V = (np.pi * np.cos(np.pi * x)).reshape(1, n)
    return Workload("burgers1d_sine", "burgers", 1, [n], 1, 0.0, 2.0, 0.0, 1.0, t_end,
                    ("periodic", "periodic", "periodic", "periodic"),
                    U.ravel().copy(), V.ravel().copy(), dt_mode=dt_mode)


# 1D Euler smooth density wave (Example 3.2): rho = 1 + 0.2 sin(pi x), u = p = 1.
def euler1d_smooth(n: int, t_end: float = 2.0, gamma: float = 1.4,
                   dt_mode: str = "accuracy") -> Workload:
    x = centers(0.0, 2.0, n)
    rho = 1.0 + 0.2 * np.sin(np.pi * x)
    drho = 0.2 * np.pi * np.cos(np.pi * x)
    one = np.ones(n)
    U = euler_conserved(rho, one, one, gamma)
    V = np.stack([drho, drho * 1.0, 0.5 * drho * 1.0])
    return Workload("euler1d_smooth", "euler", 1, [n], 1, 0.0, 2.0, 0.0, 1.0, t_end,
                    ("periodic",) * 4, U.ravel().copy(), V.ravel().copy(),
                    gas_gamma=gamma, dt_mode=dt_mode)


# 1D Euler Riemann problem on [0, 1] with the jump at x = 0.5, outflow.
def riemann1d(n: int, left, right, t_end: float = 0.15, gamma: float = 1.4) -> Workload:
    x = centers(0.0, 1.0, n)
    lo = x < 0.5
    rho = np.where(lo, left[0], right[0])
    u = np.where(lo, left[1], right[1])
    p = np.where(lo, left[2], right[2])
    U = euler_conserved(rho, u, p, gamma)
    V = np.zeros_like(U)
    return Workload("riemann1d", "euler", 1, [n], 1, 0.0, 1.0, 0.0, 1.0, t_end,
                    ("outflow", "outflow", "periodic", "periodic"),
                    U.ravel().copy(), V.ravel().copy(), gas_gamma=gamma,
                    meta=dict(left=tuple(left), right=tuple(right)))


RIEMANN_SIZES = (200, 400, 800, 1600, 3200)


def riemann_batch(count: int = 2048, seed: int = 20220711, sizes=RIEMANN_SIZES,
                  t_end: float = 0.15, gamma: float = 1.4) -> Workload:
    """Ragged batch of 1D Euler Riemann problems: per instance N uniform over
    `sizes`; left/right rho ~ U[0.1, 1], u ~ U[-0.5, 0.5], p ~ U[0.1, 1]
    (draw order per instance: N, rhoL, uL, pL, rhoR, uR, pR); jump at
    x = 0.5 on [0, 1]; outflow; V = 0."""
    rng = SplitMix64(seed)
    nx, states, Us, Vs = [], [], [], []
    for _ in range(count):
        n = rng.choice(sizes)
        left = (rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0))
        right = (rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0))
        w = riemann1d(n, left, right, t_end, gamma)
        nx.append(n)
        states.append((left, right))
        Us.append(w.U)
        Vs.append(w.V)
    return Workload("riemann_batch", "euler", 1, nx, 1, 0.0, 1.0, 0.0, 1.0, t_end,
                    ("outflow", "outflow", "periodic", "periodic"),
                    np.concatenate(Us), np.concatenate(Vs), gas_gamma=gamma,
                    meta=dict(states=states, seed=seed))


# ---------------------------------------------------------------------------
# 2D
# ---------------------------------------------------------------------------
def burgers2d_sine(n: int, t_end: float = 0.5 / math.pi, dt_mode: str = "accuracy") -> Workload:
    """2D Burgers on [0, 4]^2, u0 = 0.5 + sin(pi (x + y)/2), periodic (Examples 3.8, 3.10)."""
    x = centers(0.0, 4.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")   # [j][i]
    s = np.pi * (X + Y) / 2.0
    U = (0.5 + np.sin(s)).reshape(1, n, n)
    D = (0.5 * np.pi * np.cos(s)).reshape(1, n, n)
    return Workload("burgers2d_sine", "burgers", 2, [n], n, 0.0, 4.0, 0.0, 4.0, t_end,
                    ("periodic",) * 4, U.ravel().copy(), D.ravel().copy(),
                    D.ravel().copy(), dt_mode=dt_mode)


def euler2d_smooth(n: int, ny: Optional[int] = None, u: float = 0.7, v: float = 0.3,
                   t_end: float = 2.0, gamma: float = 1.4,
                   dt_mode: str = "accuracy") -> Workload:
    """2D Euler density wave on [0, 2]^2: rho = 1 + 0.2 sin(pi (x + y)),
    constant velocity (u, v) and p = 1, periodic; U, U_x, U_y exact."""
    ny = n if ny is None else ny
    x, y = centers(0.0, 2.0, n), centers(0.0, 2.0, ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    rho = 1.0 + 0.2 * np.sin(np.pi * (X + Y))
    drho = 0.2 * np.pi * np.cos(np.pi * (X + Y))
    U = euler_conserved(rho, np.full_like(rho, u), np.ones_like(rho), gamma,
                        v=np.full_like(rho, v))
    D = np.stack([drho, drho * u, drho * v, 0.5 * drho * (u * u + v * v)])
    return Workload("euler2d_smooth", "euler", 2, [n], ny, 0.0, 2.0, 0.0, 2.0, t_end,
                    ("periodic",) * 4, U.ravel().copy(), D.ravel().copy(), D.ravel().copy(),
                    gas_gamma=gamma, dt_mode=dt_mode, meta=dict(u=u, v=v))


# Double Mach reflection (Example 3.11; Woodward-Colella set-up): a Mach 10
# shock at 60 degrees to the x axis meets the wall y = 0 at x = 1/6 at t = 0.
# Pre-shock gas (rho, p) = (1.4, 1) at rest; post-shock rho = 8, p = 116.5,
# speed 8.25 along (cos 30deg, -sin 30deg).
DMR_PRE = (1.4, 0.0, 0.0, 1.0)
DMR_POST = (8.0, 8.25 * math.cos(math.pi / 6.0), -8.25 * math.sin(math.pi / 6.0), 116.5)


def double_mach(nx: int = 1920, ny: int = 480, t_end: float = 0.2, gamma: float = 1.4) -> Workload:
    x, y = centers(0.0, 4.0, nx), centers(0.0, 1.0, ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    x0, ang = 1.0 / 6.0, math.pi / 3.0
    post = X < x0 + Y / math.tan(ang)
    rho = np.where(post, DMR_POST[0], DMR_PRE[0])
    u = np.where(post, DMR_POST[1], DMR_PRE[1])
    v = np.where(post, DMR_POST[2], DMR_PRE[2])
    p = np.where(post, DMR_POST[3], DMR_PRE[3])
    U = euler_conserved(rho, u, p, gamma, v=v)
    Z = np.zeros_like(U)
    post_c = tuple(float(a) for a in euler_conserved(DMR_POST[0], DMR_POST[1], DMR_POST[3], gamma,
                                                     v=DMR_POST[2]))
    pre_c = tuple(float(a) for a in euler_conserved(DMR_PRE[0], DMR_PRE[1], DMR_PRE[3], gamma,
                                                    v=DMR_PRE[2]))
    return Workload("double_mach", "euler", 2, [nx], ny, 0.0, 4.0, 0.0, 1.0, t_end,
                    ("inflow", "outflow", "dmr_bottom", "dmr_top"),
                    U.ravel().copy(), Z.ravel().copy(), Z.ravel().copy(), gas_gamma=gamma,
                    inflow=post_c, pre=pre_c, dmr_x0=x0, dmr_speed=10.0, dmr_angle=ang)


def _euler1d_piecewise(name, n, x0, x1, pieces, bc, t_end, gamma=1.4):
    """1D Euler with piecewise-constant primitive data: pieces is a list of
    (x_right_edge, (rho, u, p)); V = 0 (no derivative of a jump)."""
    x = centers(x0, x1, n)
    rho, u, p = np.empty(n), np.empty(n), np.empty(n)
    left = x0
    for edge, (r, uu, pp) in pieces:
        sel = (x >= left) & (x < edge)
        rho[sel], u[sel], p[sel] = r, uu, pp
        left = edge
    U = euler_conserved(rho, u, p, gamma)
    return Workload(name, "euler", 1, [n], 1, x0, x1, 0.0, 1.0, t_end,
                    (bc, bc, "periodic", "periodic"), U.ravel().copy(),
                    np.zeros_like(U).ravel(), gas_gamma=gamma)


def lax(n: int = 200, t_end: float = 0.16) -> Workload:
    """Lax problem (Example 3.5): (0.445, 0.698, 3.528) | (0.5, 0, 0.571),
    jump at x = 0 on [-0.5, 0.5], outflow."""
    return _euler1d_piecewise("lax", n, -0.5, 0.5,
                              [(0.0, (0.445, 0.698, 3.528)), (np.inf, (0.5, 0.0, 0.571))],
                              "outflow", t_end)


def shu_osher(n: int = 400, t_end: float = 1.8) -> Workload:
    """Shu-Osher problem (Example 3.6) on [-5, 5], outflow: a Mach 3 shock at
    x = -4 running into rho = 1 + 0.2 sin(5x). The smooth part carries its
    exact derivative."""
    x = centers(-5.0, 5.0, n)
    post = x < -4.0
    rho = np.where(post, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
    u = np.where(post, 2.629369, 0.0)
    p = np.where(post, 10.333333, 1.0)
    U = euler_conserved(rho, u, p, 1.4)
    drho = np.where(post, 0.0, np.cos(5.0 * x))
    V = np.stack([drho, np.zeros(n), np.zeros(n)])
    return Workload("shu_osher", "euler", 1, [n], 1, -5.0, 5.0, 0.0, 1.0, t_end,
                    ("outflow", "outflow", "periodic", "periodic"), U.ravel().copy(),
                    V.ravel().copy())


def blast_waves(n: int = 800, t_end: float = 0.038) -> Workload:
    """Interaction of two blast waves (Example 3.7) on [0, 1], reflective
    walls: p = 1000 | 0.01 | 100 split at x = 0.1 and 0.9, rho = 1, u = 0."""
    return _euler1d_piecewise("blast_waves", n, 0.0, 1.0,
                              [(0.1, (1.0, 0.0, 1000.0)), (0.9, (1.0, 0.0, 0.01)),
                               (np.inf, (1.0, 0.0, 100.0))], "reflective", t_end)


# Linear-weight sets of the study in Example 3.7 (reconstruction G, limiter D).
WEIGHT_SETS = {"G1": (0.99, 0.005, 0.005), "G2": (1 / 3, 1 / 3, 1 / 3), "G3": (0.01, 0.495, 0.495),
               "D1": (0.99, 0.005, 0.005), "D2": (1 / 3, 1 / 3, 1 / 3), "D3": (0.01, 0.495, 0.495)}


def burgers_adjoint_batch(count: int = 256, n: int = 800, seed: int = 5, amplitude: float = 0.05,
                          t_end: float = 0.5 / math.pi) -> Workload:
    """Batch of 1D Burgers problems for gradient checks: u0 = 0.5 + sin(pi x)
    plus a seeded smooth perturbation of up to 4 Fourier modes with total
    amplitude <= `amplitude`, periodic on [0, 2], smooth up to t_end, with
    the exact derivative as V."""
    rng = SplitMix64(seed)
    x = centers(0.0, 2.0, n)
    Us, Vs = [], []
    for _ in range(count):
        u = 0.5 + np.sin(np.pi * x)
        v = np.pi * np.cos(np.pi * x)
        for mode in range(1, 5):
            a = amplitude / 4.0 * rng.uniform(-1.0, 1.0)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            u = u + a * np.sin(mode * np.pi * x + ph)
            v = v + a * mode * np.pi * np.cos(mode * np.pi * x + ph)
        Us.append(u)
        Vs.append(v)
    return Workload("burgers_adjoint_batch", "burgers", 1, [n] * count, 1, 0.0, 2.0, 0.0, 1.0,
                    t_end, ("periodic",) * 4, np.concatenate(Us), np.concatenate(Vs),
                    meta=dict(seed=seed))


def fourier_2d(rng: SplitMix64, n: int, ny: int, lo: float, hi: float, amplitude: float,
               modes: int = 4):
    """Seeded smooth periodic field on [lo, hi]^2 (a sum of `modes` Fourier
    modes with wave numbers 1..2 in each direction, total amplitude <=
    `amplitude`) and its exact x and y derivatives, on cell centres."""
    L = hi - lo
    x, y = centers(lo, hi, n), centers(lo, hi, ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    f = np.zeros_like(X)
    fx = np.zeros_like(X)
    fy = np.zeros_like(X)
    for _ in range(modes):
        a = amplitude / modes * rng.uniform(-1.0, 1.0)
        kx = 2.0 * math.pi / L * int(rng.uniform(0.0, 3.0))
        ky = 2.0 * math.pi / L * (1 + int(rng.uniform(0.0, 2.0)))
        ph = rng.uniform(0.0, 2.0 * math.pi)
        s = np.sin(kx * X + ky * Y + ph)
        c = np.cos(kx * X + ky * Y + ph)
        f += a * s
        fx += a * kx * c
        fy += a * ky * c
    return f, fx, fy


def euler2d_adjoint(n: int = 512, seed: int = 7, steps: int = 400, t_end: float = 0.25,
                    gamma: float = 1.4) -> Workload:
    """2D Euler gradient workload on [0, 2]^2, periodic: the density wave of
    euler2d_smooth plus a seeded smooth perturbation of up to 4 Fourier modes
    (amplitude 0.05) in rho, u = 0.7, v = 0.3, p = 1, exact U_x, U_y; a fixed
    time step t_end / steps (CFL about 0.54 at n = 512)."""
    rng = SplitMix64(seed)
    x = centers(0.0, 2.0, n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    f, fx, fy = fourier_2d(rng, n, n, 0.0, 2.0, 0.05)
    u, v = 0.7, 0.3
    rho = 1.0 + 0.2 * np.sin(np.pi * (X + Y)) + f
    rx = 0.2 * np.pi * np.cos(np.pi * (X + Y)) + fx
    ry = 0.2 * np.pi * np.cos(np.pi * (X + Y)) + fy
    U = euler_conserved(rho, np.full_like(rho, u), np.ones_like(rho), gamma, v=np.full_like(rho, v))
    Vx = np.stack([rx, rx * u, rx * v, 0.5 * rx * (u * u + v * v)])
    Wy = np.stack([ry, ry * u, ry * v, 0.5 * ry * (u * u + v * v)])
    return Workload("euler2d_adjoint", "euler", 2, [n], n, 0.0, 2.0, 0.0, 2.0, t_end,
                    ("periodic",) * 4, U.ravel().copy(), Vx.ravel().copy(), Wy.ravel().copy(),
                    gas_gamma=gamma, meta=dict(seed=seed, steps=steps, dt=t_end / steps))


def buckley_leverett(n: int = 80, t_end: float = 0.4) -> Workload:
    """Example 3.4: u_t + (4u^2 / (4u^2 + (1 - u)^2))_x = 0 on [-1, 1], u0 = 1
    on [-1/2, 0] and 0 elsewhere, V = 0 (discontinuous data); outflow
    boundaries (the paper states none; no wave reaches them before T)."""
    x = centers(-1.0, 1.0, n)
    U = np.where((x >= -0.5) & (x <= 0.0), 1.0, 0.0)
    return Workload("buckley_leverett", "buckley", 1, [n], 1, -1.0, 1.0, 0.0, 1.0, t_end,
                    ("outflow", "outflow", "periodic", "periodic"), U.copy(), np.zeros(n))


def buckley_batch(count: int = 2048, seed: int = 20220712, sizes=RIEMANN_SIZES,
                  t_end: float = 0.4) -> Workload:
    """Ragged batch of Example 3.4 problems (u0 = 1 on [-1/2, 0], else 0, on
    [-1, 1], outflow): per instance N uniform over `sizes`."""
    rng = SplitMix64(seed)
    nx = [sizes[min(len(sizes) - 1, int(rng.uniform(0.0, len(sizes))))] for _ in range(count)]
    Us = [buckley_leverett(n, t_end).U for n in nx]
    return Workload("buckley_batch", "buckley", 1, nx, 1, -1.0, 1.0, 0.0, 1.0, t_end,
                    ("outflow", "outflow", "periodic", "periodic"), np.concatenate(Us),
                    np.zeros(sum(nx)))

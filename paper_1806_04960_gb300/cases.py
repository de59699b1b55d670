"""Seeded synthetic initial states for the solver and for the FP64 oracle.

This module only builds inputs: grids, solid masks and initial conserved states
Q = (alpha*rho, alpha*rho*u, alpha*rho*v, alpha) as four SoA planes of shape
(ny, nx), x index fastest.  It holds none of the scheme's arithmetic; both the
CUDA path and the oracle receive the same arrays from here.

Physical set-ups follow the paper's test problems (Section 5):
  * liquid at rest in hydrostatic balance, rho = rho0 exp(-g rho0 (y - y0) / k0)
    (Eq. BNs_eq3 and the dam-break initial density, Section 5.5);
  * gas at p = 0, rho = rho0, u = 0 with volume fraction eps (Section 5 preamble);
  * obstacles are cells removed from the domain (Sections 5.1 and 5.5);
  * k0 from the Mach-0.3 rule k0 = rho0 (2 sqrt(g H) / 0.3)^2, which reproduces
    the paper's 6.54e5 (H = 1.5), 6.37e5 (H = 1.4618) and 2.62e5 (H = 0.6).

Random numbers come from numpy's PCG64 with the seeds stated per workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

RHO0 = 1000.0
GRAV = 9.81
EPS_GAS = 1.0e-3

BC_WALL = 0
BC_TRANSMISSIVE = 1


def mach03_k0(height: float, rho0: float = RHO0, g: float = GRAV) -> float:
    """Tait constant giving Mach 0.3 for the reference speed 2 sqrt(g H)."""
    vref = 2.0 * math.sqrt(g * height)
    return rho0 * (vref / 0.3) ** 2


@dataclass
class Case:
    """One solver input: grid, equation of state, boundaries and initial state."""
    name: str
    nx: int
    ny: int
    x0: float
    y0: float
    dx: float
    dy: float
    rho0: float = RHO0
    k0: float = 4.36e5
    gamma: float = 1.0
    g: float = GRAV
    eps: float = EPS_GAS
    sides: tuple = (BC_WALL, BC_WALL, BC_WALL, BC_WALL)   # W, E, S, N
    solid: np.ndarray = None     # uint8 (ny, nx), 1 = removed cell
    q: np.ndarray = None         # float64 (4, ny, nx)
    cfl: float = 0.9
    steps: int = 200
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def xc(self) -> np.ndarray:
        return self.x0 + (np.arange(self.nx) + 0.5) * self.dx

    def yc(self) -> np.ndarray:
        return self.y0 + (np.arange(self.ny) + 0.5) * self.dy

    def with_state(self, q: np.ndarray) -> "Case":
        return replace(self, q=np.ascontiguousarray(q, dtype=np.float64))


def _rect_mask(xc, yc, rects):
    """Cells whose centre lies inside any rectangle (x_left, x_right, y_bottom, y_top)."""
    X, Y = np.meshgrid(xc, yc)
    m = np.zeros(X.shape, dtype=bool)
    for (xl, xr, yb, yt) in rects:
        m |= (X >= xl) & (X <= xr) & (Y >= yb) & (Y <= yt)
    return m


def dambreak(nx: int, ny: int, *, lx: float = 4.0, ly: float = 2.0, x0: float = 0.0,
             x_col: float = 1.0, h_col: float = 1.0, rects=(), k0: float | None = None,
             lake_level: float | None = None, g: float = GRAV, eps: float = EPS_GAS,
             name: str = "dambreak", steps: int = 200, cfl: float = 0.9,
             sides=(BC_WALL, BC_WALL, BC_WALL, BC_WALL)) -> Case:
    """Water column [0, x_col] x [0, h_col] in hydrostatic balance, gas elsewhere.

    With ``lake_level`` set, the whole fluid domain is instead a lake at rest with
    its free surface at that height: alpha = 1 below, eps above, and the density
    follows the same exponential profile in both layers (an exact rest state of
    the model, the gas continuing the liquid's profile).
    """
    if k0 is None:
        k0 = mach03_k0(h_col)
    dx, dy = lx / nx, ly / ny
    c = Case(name=name, nx=nx, ny=ny, x0=x0, y0=0.0, dx=dx, dy=dy, k0=k0, g=g, eps=eps,
             steps=steps, cfl=cfl, sides=tuple(sides))
    xc, yc = c.xc(), c.yc()
    X, Y = np.meshgrid(xc, yc)
    solid = _rect_mask(xc, yc, rects)
    kappa = g * RHO0 / k0
    if lake_level is None:
        liquid = (X < x_col) & (Y < h_col)
        rho = np.where(liquid, RHO0 * np.exp(-kappa * (Y - h_col)), RHO0)
    else:
        liquid = Y < lake_level
        rho = RHO0 * np.exp(-kappa * (Y - lake_level))
    alpha = np.where(liquid, 1.0, eps)
    q = np.zeros((4, ny, nx))
    q[0] = alpha * rho
    q[3] = alpha
    q[:, solid] = 0.0
    c.solid = solid.astype(np.uint8)
    c.q = q
    c.meta = dict(x_col=x_col, h_col=h_col, rects=list(rects), lake_level=lake_level)
    return c


def lake_box(n: int = 100, *, obstacle: bool = True, k0: float = 2.78e5) -> Case:
    """Water at rest of Section 5.1: [-0.5,0.5] x [0,1] all liquid (alpha = 1),
    free surface at y = 1, optionally with the block [-0.25,0.25] x [0,0.33]
    removed from the domain."""
    rects = [(-0.25, 0.25, 0.0, 0.33)] if obstacle else []
    return dambreak(n, n, lx=1.0, ly=1.0, x0=-0.5, rects=rects, k0=k0, lake_level=1.0,
                    name=f"lake_box_{n}{'_obst' if obstacle else ''}")


def c2_rects(seed: int = 1806, count: int = 8):
    """Eight random bed obstacles: height U(0.05,0.4), width U(0.05,0.3),
    left edge U(1.2, 3.7 - width); overlaps allowed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rects = []
    for _ in range(count):
        h = rng.uniform(0.05, 0.4)
        w = rng.uniform(0.05, 0.3)
        xl = rng.uniform(1.2, 3.7 - w)
        rects.append((xl, xl + w, 0.0, h))
    return rects


C1_RECT = (2.5, 2.7, 0.0, 0.3)


def c1(nx: int = 128, ny: int = 64) -> Case:
    """FP64 dam break over one 0.2 x 0.3 obstacle at x = 2.5, 200 steps at CFL 0.9."""
    return dambreak(nx, ny, rects=[C1_RECT], name=f"dambreak_{nx}x{ny}", steps=200)


def c1_lake(nx: int = 128, ny: int = 64) -> Case:
    """Lake at rest at y0 = 1.0 (with air above) on the dam-break grid and obstacle."""
    return dambreak(nx, ny, rects=[C1_RECT], lake_level=1.0, name=f"lake_{nx}x{ny}", steps=200)


C5_TARGET_RECT = (2.5, 2.7, 0.0, 0.25)


def c5(nx: int = 512, ny: int = 256, steps: int = 2000, cfl: float = 0.45) -> Case:
    """Gradient workload: the dam break of c1 (k0 = 4.36e5) at nx x ny."""
    return dambreak(nx, ny, rects=[C1_RECT], k0=4.36e5, cfl=cfl, name=f"adjoint_{nx}x{ny}",
                    steps=steps)


def c5_target(nx: int = 512, ny: int = 256, seed: int = 5, cfl: float = 0.45) -> Case:
    """Initial state whose gauge record is the loss's target: column height
    0.95, obstacle height 0.25, density and velocity perturbed (seed 5)."""
    c = dambreak(nx, ny, h_col=0.95, rects=[C5_TARGET_RECT], k0=4.36e5, cfl=cfl,
                 name=f"adjoint_target_{nx}x{ny}")
    return perturbed(c, seed)


def c5_gauges(c: Case, count: int = 16, seed: int = 5, region=(0.0, 2.0, 0.0, 1.2)):
    """``count`` distinct flat cell indices j*nx + i drawn (PCG64, seed) from the
    fluid cells whose centre lies in region = (x_left, x_right, y_bottom, y_top),
    where the dam-break wave passes; sorted."""
    xl, xr, yb, yt = region
    X, Y = np.meshgrid(c.xc(), c.yc())
    ok = (c.solid == 0) & (X >= xl) & (X <= xr) & (Y >= yb) & (Y <= yt)
    pool = np.flatnonzero(ok.ravel())
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(pool, size=count, replace=False)).astype(np.int64)


def c5_directions(c: Case, count: int = 32, seed: int = 32) -> np.ndarray:
    """``count`` seeded perturbation directions of the initial state (count, 4,
    ny, nx): standard normal factors times alpha rho and alpha on fluid cells
    (relative perturbations of the two fields the gradient is taken for), zero
    in the momenta and in solid cells."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = np.zeros((count, 4, c.ny, c.nx))
    fluid = c.solid == 0
    for k in range(count):
        d[k, 0] = rng.standard_normal((c.ny, c.nx)) * c.q[0]
        d[k, 3] = rng.standard_normal((c.ny, c.nx)) * c.q[3]
        d[k][:, ~fluid] = 0.0
    return d


H_RECT = (0.7, 0.9, 0.0, 0.2)


def heights(nx: int = 48, ny: int = 24, steps: int = 60, cfl: float = 0.45) -> Case:
    """Obstacle-height gradient workload: a 2 x 1 box, water column [0, 1] x
    [0, 0.6] with the 0.2 x 0.2 obstacle H_RECT inside it (k0 = 4.36e5), so
    that the water over the obstacle's top moves from the first step."""
    return dambreak(nx, ny, lx=2.0, ly=1.0, x_col=1.0, h_col=0.6, rects=[H_RECT], k0=4.36e5,
                    cfl=cfl, steps=steps, name=f"heights_{nx}x{ny}")


def height_ids(c: Case, rects=None) -> np.ndarray:
    """Height parameters of obstacles: an int32 (ny, nx) map holding k at the
    fluid cells that sit directly on the top solid cell of rectangle k's
    columns (rects default to the case's own, ``meta['rects']``), -1 elsewhere.
    Raising obstacle k by theta dy turns those cells into the partial cells
    of reading R-h."""
    rects = c.meta.get("rects", []) if rects is None else rects
    out = np.full((c.ny, c.nx), -1, dtype=np.int32)
    xc, yc = c.xc(), c.yc()
    for k, (xl, xr, yb, yt) in enumerate(rects):
        for i in np.flatnonzero((xc >= xl) & (xc <= xr)):
            rows = np.flatnonzero((yc >= yb) & (yc <= yt) & (c.solid[:, i] == 1))
            if rows.size == 0:
                continue
            j = int(rows.max()) + 1
            if j < c.ny and c.solid[j, i] == 0:
                out[j, i] = k
    return out


def generic(c: Case, seed: int, scale: float = 1e-3) -> Case:
    """``perturbed`` plus a seeded perturbation of the volume fraction
    (liquid alpha = 1 - scale U(0,1), gas alpha = eps (1 + 0.1 N(0,1)) clipped
    to [eps/2, 2 eps]), alpha rho rescaled to keep the density: a state with no
    two cells exactly equal in any component."""
    p = perturbed(c, seed, scale)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    q = p.q.copy()
    fluid = c.solid == 0
    a = q[3]
    liquid = a > 0.5
    rho = np.where(fluid, q[0] / np.where(a > 0, a, 1.0), 0.0)
    a_new = np.where(liquid, 1.0 - scale * rng.uniform(size=a.shape),
                     np.clip(c.eps * (1.0 + 0.1 * rng.standard_normal(a.shape)), 0.5 * c.eps,
                             2.0 * c.eps))
    u = np.where(fluid, q[1] / np.where(q[0] > 0, q[0], 1.0), 0.0)
    v = np.where(fluid, q[2] / np.where(q[0] > 0, q[0], 1.0), 0.0)
    q[3] = a_new
    q[0] = a_new * rho
    q[1] = q[0] * u
    q[2] = q[0] * v
    q[:, ~fluid] = 0.0
    return replace(c, q=q, name=c.name + f"_g{seed}")


def c2(nx: int = 4096, ny: int = 2048, steps: int = 1000) -> Case:
    """Throughput workload: the dam break at 4096 x 2048 with 8 seeded obstacles."""
    return dambreak(nx, ny, rects=c2_rects(), name=f"dambreak8_{nx}x{ny}", steps=steps)


def c2_lake(nx: int = 4096, ny: int = 2048, steps: int = 1000) -> Case:
    return dambreak(nx, ny, rects=c2_rects(), lake_level=1.0, name=f"lake8_{nx}x{ny}",
                    steps=steps)


def drop(n: int = 2048, *, half: float = 2.0, a0: float = 100.0, k0: float = 2.25e9,
         radius: float = 1.0, eps: float = EPS_GAS, alpha_liquid: float = 1.0,
         steps: int = 2000, cfl: float = 0.9) -> Case:
    """Oscillating elliptical drop (Section 5.2) with g = 0: a disc of liquid at
    rho0 with velocity (-a0 x, a0 y) inside a gas at rest."""
    d = 2.0 * half / n
    c = Case(name=f"drop_{n}", nx=n, ny=n, x0=-half, y0=-half, dx=d, dy=d, k0=k0, g=0.0,
             eps=eps, steps=steps, cfl=cfl)
    X, Y = np.meshgrid(c.xc(), c.yc())
    inside = X * X + Y * Y < radius * radius
    alpha = np.where(inside, alpha_liquid, eps)
    q = np.zeros((4, n, n))
    q[0] = alpha * RHO0
    q[1] = np.where(inside, q[0] * (-a0 * X), 0.0)
    q[2] = np.where(inside, q[0] * (a0 * Y), 0.0)
    q[3] = alpha
    c.solid = np.zeros((n, n), dtype=np.uint8)
    c.q = q
    return c


def weir_domains(count: int = 256, seed: int = 4960, nmin: int = 64, nmax: int = 1024):
    """Ensemble of dam breaks over a one-cell-thick weir on [0,4] x [0,2]:
    N, M ~ U{nmin..nmax}, column height H ~ U(0.3,1.0), k0 = Mach-0.3 rule for H,
    weir at the cell column containing x = 2.5 with height ~ U(0.05,0.3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        nx = int(rng.integers(nmin, nmax + 1))
        ny = int(rng.integers(nmin, nmax + 1))
        h = float(rng.uniform(0.3, 1.0))
        hw = float(rng.uniform(0.05, 0.3))
        dx = 4.0 / nx
        iw = int(math.floor(2.5 / dx))
        rect = (iw * dx, (iw + 1) * dx, 0.0, hw)
        c = dambreak(nx, ny, h_col=h, rects=[rect], name=f"weir{k}_{nx}x{ny}", steps=500)
        out.append(c)
    return out


def weir_e5(nx: int = 800, ny: int = 250, cfl: float = 0.45) -> Case:
    """Flow over a sharp-crested weir (Section 5.5): [-7.5,7.5] x [0,2.1], a
    weir of height 0.7 and one cell thick in the cell column right of x = 0
    (a removed strip, walls all round), water [-7.5,0] x [0,1.5] in
    hydrostatic balance, k0 = 6.54e5 (Mach 0.3 for H = 1.5), at rest; the
    paper runs 800 x 250 to t = 1."""
    dx = 15.0 / nx
    rect = (0.0, dx, 0.0, 0.7)
    c = dambreak(nx, ny, lx=15.0, ly=2.1, x0=-7.5, x_col=0.0, h_col=1.5, rects=[rect],
                 k0=6.54e5, name=f"weir_e5_{nx}x{ny}", steps=0, cfl=cfl)
    c.meta.update(crest=0.7, weir_col=int(round(7.5 / dx)), t_end=1.0)
    return c


def impact_e11(nx: int = 1000, ny: int = 500, cfl: float = 0.45) -> Case:
    """Dam break and impact against a vertical wall (Section 5.7): [0,3.2] x
    [0,1.8], water [0,1.2] x [0,0.6] in hydrostatic balance, k0 = 2.62e5,
    walls on three sides and a transmissive top; the paper runs 1000 x 500
    to t = 1 (efficiency) and shows t = 0.6 .. 1.7."""
    c = dambreak(nx, ny, lx=3.2, ly=1.8, x_col=1.2, h_col=0.6, k0=2.62e5,
                 name=f"impact_e11_{nx}x{ny}", steps=0, cfl=cfl,
                 sides=(BC_WALL, BC_WALL, BC_WALL, BC_TRANSMISSIVE))
    c.meta.update(t_end=1.0)
    return c


def _crossings(a: np.ndarray, y: np.ndarray, level: float = 0.5):
    """Heights where the column profile a(y) crosses `level`, by linear
    interpolation between cell centres, with the direction (+1: rising with y)."""
    out = []
    for j in range(len(a) - 1):
        lo, hi = a[j] - level, a[j + 1] - level
        if (lo < 0.0) != (hi < 0.0):
            t = lo / (lo - hi)
            out.append((y[j] + t * (y[j + 1] - y[j]), 1 if hi >= 0.0 else -1))
    return out


def weir_nappe(c: Case, q: np.ndarray, x_max: float = 0.8):
    """Over-topping profile of the weir flow from a state q (Section 5.5, Eq.
    (OverToppingProfile)): the lower streamline y_l(x) of the nappe right of
    the weir, found as the first alpha = 0.5 crossing below the upper free
    surface when scanning each column downwards; its maximum (x_m, y_m); and
    h0, the height of the free surface above the crest in the weir column.
    Returns (xs, y_low, x_m, y_m, h0); y_low is NaN where no nappe is found."""
    a = q[3]
    xc, yc = c.xc(), c.yc()
    iw = c.meta["weir_col"]
    crest = (np.nonzero(c.solid[:, iw])[0].max() + 1) * c.dy   # snapped crest height
    col = a[:, iw].copy()
    col[c.solid[:, iw] == 1] = 1.0                             # the weir itself counts as full
    tops = [y for y, d in _crossings(col, yc) if d < 0]
    h0 = (max(tops) - crest) if tops else float("nan")
    xs, ys = [], []
    for i in range(iw + 1, c.nx):
        if xc[i] > x_max:
            break
        cr = _crossings(a[:, i], yc)
        # downwards from the top: the first falling-into-liquid crossing is the
        # upper surface, the next one below it (rising with y) the lower one
        below = [y for y, d in sorted(cr, key=lambda z: -z[0])]
        dirs = [d for y, d in sorted(cr, key=lambda z: -z[0])]
        y_low = float("nan")
        for k in range(len(below) - 1):
            if dirs[k] < 0 and dirs[k + 1] > 0:
                y_low = below[k + 1]
                break
        xs.append(xc[i])
        ys.append(y_low)
    xs, ys = np.array(xs), np.array(ys)
    ok = np.isfinite(ys)
    if not ok.any():
        return xs, ys, float("nan"), float("nan"), h0
    k = int(np.nanargmax(np.where(ok, ys, -np.inf)))
    return xs, ys, float(xs[k]), float(ys[k]), float(h0)


def overtopping_profile(x, x_m: float, y_m: float, h0: float):
    """Lower streamline of the experimental reference, Eq. (OverToppingProfile):
    y = y_m - 0.47 h0 ((x - x_m) / h0)^1.85 for x >= x_m."""
    x = np.asarray(x, dtype=float)
    return y_m - 0.47 * h0 * (np.maximum(x - x_m, 0.0) / h0) ** 1.85


def smooth_bump(n: int, *, amp: float = 1e-3, sigma: float = 0.08, k0: float = 4.36e5,
                g: float = GRAV) -> Case:
    """All-liquid unit box at hydrostatic rest (free surface at the lid) with a
    small Gaussian density bump at the centre: a smooth problem for convergence."""
    d = 1.0 / n
    c = Case(name=f"bump_{n}", nx=n, ny=n, x0=0.0, y0=0.0, dx=d, dy=d, k0=k0, g=g)
    X, Y = np.meshgrid(c.xc(), c.yc())
    kappa = g * RHO0 / k0
    rho = RHO0 * np.exp(-kappa * (Y - 1.0)) * (1.0 + amp * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2)
                                                                   / sigma ** 2))
    q = np.zeros((4, n, n))
    q[0] = rho
    q[3] = 1.0
    c.solid = np.zeros((n, n), dtype=np.uint8)
    c.q = q
    return c


def riemann_x(nx: int, *, rho_l: float, rho_r: float, u_l: float = 0.0, u_r: float = 0.0,
              ny: int = 4, length: float = 1.0, k0: float = 4.36e5, x_split: float = 0.5) -> Case:
    """1D Riemann problem along x for the all-liquid (alpha = 1), g = 0 model:
    isothermal gas dynamics with constant sound speed sqrt(k0/rho0)."""
    d = length / nx
    c = Case(name=f"riemann_{nx}", nx=nx, ny=ny, x0=0.0, y0=0.0, dx=d, dy=d, k0=k0, g=0.0,
             sides=(BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_WALL, BC_WALL))
    X, _ = np.meshgrid(c.xc(), c.yc())
    left = X < x_split
    rho = np.where(left, rho_l, rho_r)
    u = np.where(left, u_l, u_r)
    q = np.zeros((4, ny, nx))
    q[0] = rho
    q[1] = rho * u
    q[3] = 1.0
    c.solid = np.zeros((ny, nx), dtype=np.uint8)
    c.q = q
    return c


def contact_x(nx: int, *, u0: float = 1.0, ny: int = 4, length: float = 1.0,
              k0: float = 4.36e5, eps: float = EPS_GAS) -> Case:
    """Volume-fraction contact at p = 0 (rho = rho0) moving with uniform speed u0
    on a periodic-free strip: alpha is a smooth bump, exactly advected."""
    d = length / nx
    c = Case(name=f"contact_{nx}", nx=nx, ny=ny, x0=0.0, y0=0.0, dx=d, dy=d, k0=k0, g=0.0,
             eps=eps, sides=(BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_WALL, BC_WALL))
    X, _ = np.meshgrid(c.xc(), c.yc())
    alpha = 0.5 + 0.4 * np.exp(-((X - 0.3) / 0.08) ** 2)
    q = np.zeros((4, ny, nx))
    q[0] = alpha * RHO0
    q[1] = alpha * RHO0 * u0
    q[3] = alpha
    c.solid = np.zeros((ny, nx), dtype=np.uint8)
    c.q = q
    return c


def mirror_x(c: Case) -> Case:
    """The same problem reflected about the vertical mid-line (u -> -u)."""
    q = c.q[:, :, ::-1].copy()
    q[1] = -q[1]
    out = replace(c, q=np.ascontiguousarray(q), solid=np.ascontiguousarray(c.solid[:, ::-1]),
                  sides=(c.sides[1], c.sides[0], c.sides[2], c.sides[3]), name=c.name + "_mx")
    return out


def perturbed(c: Case, seed: int, scale: float = 1e-3) -> Case:
    """Random relative perturbation of the fluid density and small velocities:
    a generic, non-symmetric state for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = c.q.copy()
    fluid = c.solid == 0
    rho = np.where(fluid, q[0] / np.where(q[3] > 0, q[3], 1.0), 0.0)
    rho = rho * (1.0 + scale * rng.standard_normal(rho.shape))
    u = scale * 100.0 * rng.standard_normal(rho.shape)
    v = scale * 100.0 * rng.standard_normal(rho.shape)
    q[0] = q[3] * rho
    q[1] = q[0] * u
    q[2] = q[0] * v
    q[:, ~fluid] = 0.0
    return replace(c, q=q, name=c.name + f"_p{seed}")

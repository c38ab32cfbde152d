"""Exact rational-arithmetic brute force of the lid-driven cavity step, for tiny grids.

Independent of ``oracle/`` (no shared code or tables) and written in a different form, so that
the two only agree if both state the method of Sec. 2 correctly:
  * velocities are enumerated in their own order, weights derived from |c|^2 (Sec. 2.1);
  * streaming is a PUSH (send f*_j(x) to x + c_j) instead of the oracle's pull (Eq. 1);
  * wall nodes use the post-collision closed form of non-equilibrium extrapolation,
    f*_b = f^eq(rho_f, u_w) + (1 - 1/tau) [f(x_f) - f^eq(rho_f, u_f)],
    which is what "rebuild by Sec. 2.2 (ii), then collide by Eq. 1" gives, because the
    non-equilibrium part carries no mass and no momentum;
  * all arithmetic is exact (fractions.Fraction), so a rational tau and U give an exact result.
Reading of the geometry: walls are the outer ring of the nx*ny grid, the lid is the top row
without its two corner nodes, and x_f is the inner neighbour along the inward normal (diagonal
for the corners).
"""
from fractions import Fraction as Fr

# Velocity set of Sec. 2.1, enumerated lexicographically; weight by speed class.
VEL = [(cx, cy) for cx in (-1, 0, 1) for cy in (-1, 0, 1)]


def weight(c):
    s = c[0] * c[0] + c[1] * c[1]
    return {0: Fr(4, 9), 1: Fr(1, 9), 2: Fr(1, 36)}[s]


WTS = [weight(c) for c in VEL]


def equilibrium(rho, ux, uy):
    """Eq. 2 with c_s^2 = 1/3, exact."""
    cs2 = Fr(1, 3)
    usq = ux * ux + uy * uy
    out = []
    for (cx, cy), w in zip(VEL, WTS):
        cu = cx * ux + cy * uy
        out.append(w * rho * (1 + cu / cs2 + cu * cu / (2 * cs2 * cs2) - usq / (2 * cs2)))
    return out


def macroscopic(f):
    """Eq. 3."""
    rho = sum(f)
    mx = sum(cx * v for (cx, _), v in zip(VEL, f))
    my = sum(cy * v for (_, cy), v in zip(VEL, f))
    return rho, mx / rho, my / rho


def wall_velocity(x, y, nx, ny, U):
    if y == ny - 1 and 0 < x < nx - 1:
        return U, Fr(0)
    return Fr(0), Fr(0)


def is_wall(x, y, nx, ny):
    return x in (0, nx - 1) or y in (0, ny - 1)


def initial(nx, ny, U):
    """Sec. 2.2 (i): rho = 1, u = 0 except the lid, f = f^eq."""
    return {(x, y): equilibrium(Fr(1), *wall_velocity(x, y, nx, ny, U))
            for x in range(nx) for y in range(ny)}


def step(fs, nx, ny, tau, U):
    """One time step on a dict {(x, y): [9 post-collision populations]}."""
    streamed = {(x, y): [None] * 9 for x in range(nx) for y in range(ny)}
    for (x, y), f in fs.items():
        for k, (cx, cy) in enumerate(VEL):
            tx, ty = x + cx, y + cy
            if 0 <= tx < nx and 0 <= ty < ny:
                streamed[(tx, ty)][k] = f[k]
    omega = 1 / tau
    out = {}
    for x in range(nx):
        for y in range(ny):
            if not is_wall(x, y, nx, ny):
                f = streamed[(x, y)]
                rho, ux, uy = macroscopic(f)
                eq = equilibrium(rho, ux, uy)
                out[(x, y)] = [a - omega * (a - e) for a, e in zip(f, eq)]
    for x in range(nx):
        for y in range(ny):
            if is_wall(x, y, nx, ny):
                xf = min(max(x, 1), nx - 2)
                yf = min(max(y, 1), ny - 2)
                ff = streamed[(xf, yf)]
                rho_f, uxf, uyf = macroscopic(ff)
                eq_w = equilibrium(rho_f, *wall_velocity(x, y, nx, ny, U))
                eq_f = equilibrium(rho_f, uxf, uyf)
                out[(x, y)] = [ew + (1 - omega) * (a - ef) for ew, a, ef in zip(eq_w, ff, eq_f)]
    return out


def to_oracle_layout(fs, nx, ny):
    """Return a nested list [ny][nx][9] in the oracle's velocity order
    0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)."""
    order = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    idx = [VEL.index(c) for c in order]
    return [[[fs[(x, y)][k] for k in idx] for x in range(nx)] for y in range(ny)]

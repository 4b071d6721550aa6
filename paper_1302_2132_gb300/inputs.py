"""Seeded synthetic inputs (primitive variables and turbulence fields) for the tests and the bench.

This module is shared by both sides of the parity tests, so it holds none of the scheme's
arithmetic: it only draws the initial primitive states (rho, u_1..u_D, p), cell widths, boundary
data and the prescribed turbulence fields.  Each side converts primitives to conservative
variables on its own.

Workloads (stand-ins for the paper's wind-tunnel cases, whose geometries and data are not public
inputs of this library):
  sod_1d            Sod shock tube, 1D
  turbulence        decaying compressible turbulence, periodic box, 2D or 3D: random-phase
                    solenoidal velocity with E(k) ~ k^4 exp(-2 (k/k0)^2) scaled to a turbulent Mach
                    number, rho = 1, p = 1/gamma; log-normal k and epsilon fields from 8 Fourier modes
  riemann_quadrant  2D four-state Riemann problem with seeded states
  near_vacuum       expansion kinks in a smooth background (the first-order fallback of MUSCL)
  shock_boundary_layer  Mach 2.85 flat-plate boundary layer under an oblique shock on a
                    wall-clustered grid, with log-law k-omega profiles (and the wall corner of the
                    full-size grid, shock_boundary_layer_crop)
  compression_corner  Mach 2.85 boundary layer over a ramp of alpha degrees on a body-fitted,
                    wall-clustered channel grid (nodes given), log-law k-omega profiles
  naca0012_case     C-grid round a NACA 0012 section with a wake cut (transonic free stream)
  wavy_nodes        smoothly skewed periodic grids (with smooth_state_at, positive_fields_at) for the
                    curvilinear invariance and parity tests
"""
import math

import numpy as np

GAMMA = 1.4


def sod_1d(n, length=1.0, x0=0.5):
    """Sod: (rho, u, p) = (1, 0, 1) left of x0, (0.125, 0, 0.1) right; uniform cells."""
    x = (np.arange(n) + 0.5) * (length / n)
    prim = np.zeros((3, n))
    left = x < x0
    prim[0] = np.where(left, 1.0, 0.125)
    prim[2] = np.where(left, 1.0, 0.1)
    return dict(dim=1, n=(n,), dx=[np.full(n, length / n)], bc=[[1, 1]], prim=prim)


def _solenoidal_velocity(rng, n, dim, k0):
    """Random-phase velocity with energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2), divergence-free."""
    shape = (n,) * dim
    kk = np.meshgrid(*([np.fft.fftfreq(n, d=1.0 / n)] * dim), indexing="ij")  # integer wavenumbers
    kmag = np.sqrt(sum(k * k for k in kk))
    kmag_safe = np.where(kmag == 0, 1.0, kmag)
    E = kmag ** 4 * np.exp(-2.0 * (kmag / k0) ** 2)
    shell = 2.0 * math.pi * kmag_safe if dim == 2 else 4.0 * math.pi * kmag_safe ** 2
    amp = np.sqrt(E / shell)
    amp[kmag == 0] = 0.0
    uh = []
    for _ in range(dim):
        phase = rng.uniform(0.0, 2.0 * math.pi, shape)
        uh.append(amp * np.exp(1j * phase) * rng.normal(size=shape))
    # project out the component along k
    dot = sum(u * k for u, k in zip(uh, kk)) / kmag_safe ** 2
    uh = [u - dot * k for u, k in zip(uh, kk)]
    vel = [np.real(np.fft.ifftn(u)) for u in uh]
    return vel


def _lognormal_field(rng, n, dim, ref, sigma=0.5, modes=8, kmax=4):
    """ref * exp(sigma * sum_m A_m cos(kappa_m . x + phi_m) / sqrt(modes)) on [0, 2 pi)^dim."""
    x = [np.arange(n) * (2.0 * math.pi / n)] * dim
    X = np.meshgrid(*x, indexing="ij")
    s = np.zeros((n,) * dim)
    for _ in range(modes):
        kap = rng.integers(-kmax, kmax + 1, size=dim)
        while not np.any(kap):
            kap = rng.integers(-kmax, kmax + 1, size=dim)
        A = rng.normal()
        phi = rng.uniform(0.0, 2.0 * math.pi)
        s += A * np.cos(sum(k * xx for k, xx in zip(kap, X)) + phi)
    return ref * np.exp(sigma * s / math.sqrt(modes))


def turbulence(n, dim, seed, k0=None, mach_t=None, C_mu=0.09, nu_ref=2e-5, gamma=GAMMA):
    """Decaying compressible turbulence on [0, 2 pi)^dim, periodic; returns primitives in
    [var][z][y][x] order (x fastest) and float32-representable k, epsilon fields."""
    if k0 is None:
        k0 = 8.0 if dim == 2 else 4.0
    if mach_t is None:
        mach_t = 0.3 if dim == 2 else 0.5
    rng = np.random.default_rng(seed)
    vel = _solenoidal_velocity(rng, n, dim, k0)
    urms = math.sqrt(np.mean(sum(v * v for v in vel)))
    c = 1.0  # rho = 1, p = 1/gamma
    vel = [v * (mach_t * c / urms) for v in vel]
    urms = mach_t * c
    prim = np.zeros((dim + 2,) + (n,) * dim)
    prim[0] = 1.0
    # arrays are indexed [x][y][z] above; store x fastest: transpose to [z][y][x]
    for i, v in enumerate(vel):
        prim[1 + i] = v.T
    prim[dim + 1] = 1.0 / gamma
    frng = np.random.default_rng(seed + 1)
    k_ref = 1.5 * urms * urms
    eps_ref = C_mu * k_ref * k_ref / nu_ref
    kf = _lognormal_field(frng, n, dim, k_ref).T
    ef = _lognormal_field(frng, n, dim, eps_ref).T
    h = 2.0 * math.pi / n
    return dict(dim=dim, n=(n,) * dim, dx=[np.full(n, h)] * dim, bc=[[0, 0]] * dim, prim=prim,
                f1=kf.astype(np.float32).astype(np.float64), f2=ef.astype(np.float32).astype(np.float64))


def riemann_quadrant(n, seed):
    """2D four-quadrant Riemann problem on [0,1]^2, transmissive boundaries, seeded states with
    rho, p in [0.1, 1.5] and u, v in [-0.8, 0.8]."""
    rng = np.random.default_rng(seed)
    st = [(rng.uniform(0.1, 1.5), rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(0.1, 1.5))
          for _ in range(4)]
    x = (np.arange(n) + 0.5) / n
    Y, X = np.meshgrid(x, x, indexing="ij")
    q = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
    prim = np.zeros((4, n, n))
    for k in range(4):
        for v in range(4):
            prim[v][q == k] = st[k][v]
    return dict(dim=2, n=(n, n), dx=[np.full(n, 1.0 / n)] * 2, bc=[[1, 1], [1, 1]], prim=prim)


def near_vacuum(n, dim, seed, kinks=4, a=1.0, p_lo=0.02, p_hi=0.5):
    """Expansion kinks in a smooth background on [0,1]^dim with transmissive boundaries: the data where a
    MUSCL reconstruction of the conservative variables gives a face state with negative pressure,
    while every other face keeps a moderate Mach number.  Background: rho = 1 + 0.1 r, each velocity
    component 0.1 r, p = p_hi (r seeded uniform in [-1, 1] per cell).  Each kink, at a seeded cell
    away from the boundaries, along a seeded axis a: the velocity component along that axis is -a, 0,
    +a on the three cells through it, the pressure p_hi, p_lo, p_hi.  With a = 1, p_lo = 0.02 and
    p_hi = 0.5 the reconstructed states on both faces of the middle cell have p = 0.4 (p_lo/0.4 - a^2/8)
    < 0 (the energy is an extremum there, so its limited slope is zero, while the momentum slope is
    a)."""
    rng = np.random.default_rng(seed)
    shape = (n,) * dim
    prim = np.zeros((dim + 2,) + shape)
    prim[0] = 1.0 + 0.1 * rng.uniform(-1.0, 1.0, shape)
    for d in range(dim):
        prim[1 + d] = 0.1 * rng.uniform(-1.0, 1.0, shape)
    prim[dim + 1] = p_hi
    used = set()
    k = 0
    while k < kinks:
        c = tuple(int(v) for v in rng.integers(3, n - 3, dim))  # array index (z, y, x order reversed below)
        ax = int(rng.integers(0, dim))  # grid axis
        arr_ax = dim - 1 - ax
        cells = []
        for off in (-1, 0, 1):
            q = list(c)
            q[arr_ax] += off
            cells.append(tuple(q))
        if any(max(abs(q[e] - u[e]) for e in range(dim)) <= 3 for q in cells for u in used):
            continue  # keep kinks four cells apart
        for q, u, p in zip(cells, (-a, 0.0, a), (p_hi, p_lo, p_hi)):
            prim[(1 + ax,) + q] = u
            prim[(dim + 1,) + q] = p
            used.add(q)
        k += 1
    return dict(dim=dim, n=shape, dx=[np.full(n, 1.0 / n)] * dim, bc=[[1, 1]] * dim, prim=prim)


def sod_2d(n, seed=0):
    """Planar Sod along x on [0,1] x [0, 1], periodic in y."""
    s = sod_1d(n)
    prim = np.zeros((4, n, n))
    prim[0] = s["prim"][0][None, :]
    prim[1] = s["prim"][1][None, :]
    prim[3] = s["prim"][2][None, :]
    return dict(dim=2, n=(n, n), dx=[np.full(n, 1.0 / n)] * 2, bc=[[1, 1], [0, 0]], prim=prim)


def random_smooth_2d(n, seed, amp=0.1):
    """A smooth positive periodic 2D state (for conservation tests)."""
    rng = np.random.default_rng(seed)
    x = np.arange(n) * (2 * math.pi / n)
    Y, X = np.meshgrid(x, x, indexing="ij")
    prim = np.zeros((4, n, n))
    f = lambda: sum(rng.normal() * np.cos(kx * X + ky * Y + rng.uniform(0, 6.28))
                    for kx, ky in ((1, 0), (0, 1), (1, 1), (2, -1)))
    prim[0] = 1.0 + amp * f()
    prim[1] = 0.3 * f()
    prim[2] = 0.3 * f()
    prim[3] = 1.0 + amp * f()
    return dict(dim=2, n=(n, n), dx=[np.full(n, 2 * math.pi / n)] * 2, bc=[[0, 0], [0, 0]], prim=prim)


# ------------------------------------------------------------------------------------------------
# Mach 2.85 shock / boundary-layer interaction
# ------------------------------------------------------------------------------------------------
def _oblique_shock(M1, theta, gamma=GAMMA):
    """Weak-branch wave angle and the post-shock (rho2/rho1, p2/p1, M2) for deflection theta
    (theta-beta-M relation and normal-shock relations, any gas-dynamics text)."""
    def tb(beta):
        return 2.0 / math.tan(beta) * (M1 ** 2 * math.sin(beta) ** 2 - 1) / (
            M1 ** 2 * (gamma + math.cos(2 * beta)) + 2) - math.tan(theta)
    mu = math.asin(1.0 / M1)
    # the weak solution lies between the Mach angle and the angle of maximum deflection
    best = None
    for k in range(1, 4000):
        b = mu + (math.pi / 2 - mu) * k / 4000
        if tb(b) > 0:
            best = b
            break
    lo, hi = best - (math.pi / 2 - mu) / 4000, best
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if tb(mid) > 0:
            hi = mid
        else:
            lo = mid
    beta = 0.5 * (lo + hi)
    Mn1 = M1 * math.sin(beta)
    r = (gamma + 1) * Mn1 ** 2 / ((gamma - 1) * Mn1 ** 2 + 2)
    pr = 1 + 2 * gamma / (gamma + 1) * (Mn1 ** 2 - 1)
    Mn2 = math.sqrt((1 + 0.5 * (gamma - 1) * Mn1 ** 2) / (gamma * Mn1 ** 2 - 0.5 * (gamma - 1)))
    M2 = Mn2 / math.sin(beta - theta)
    return beta, r, pr, M2


def shock_boundary_layer(nx, ny, M=2.85, delta=0.1, theta_deg=24.0, Re_delta=1.6e6, ratio=1.08,
                         dy1=2e-5, xlen=2.0, ylen=1.0, x_shock=0.4, gamma=GAMMA):
    """Flat plate at the bottom (isothermal no-slip wall), Dirichlet inflow with a 1/7-power
    profile below delta, supersonic outflow, and a top boundary carrying the post-shock state of a
    theta deflection over x >= x_shock (free stream before).  Rows grow geometrically with the given
    ratio up to a cap chosen so that the heights sum to ylen.  Free stream rho = 1, p = 1/gamma
    (c = 1), u = M.  Returns primitives and k, omega fields of log-law profiles."""
    # wall-clustered row heights, growth capped
    def heights(cap):
        h = dy1 * ratio ** np.arange(ny)
        return np.minimum(h, cap)
    lo, hi = dy1, ylen
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if heights(mid).sum() > ylen:
            hi = mid
        else:
            lo = mid
    dy = heights(0.5 * (lo + hi))
    dy *= ylen / dy.sum()
    dx = np.full(nx, xlen / nx)
    yc = np.cumsum(dy) - 0.5 * dy
    xc = (np.arange(nx) + 0.5) * (xlen / nx)
    T_inf = 1.0 / gamma  # p/rho
    T_wall = T_inf * (1.0 + 0.89 * 0.5 * (gamma - 1.0) * M * M)
    U = M
    mu = U * delta / Re_delta
    prof = np.where(yc < delta, (np.maximum(yc, 0.0) / delta) ** (1.0 / 7.0), 1.0)
    # temperature linear in the velocity ratio across the layer, pressure constant
    Tprof = T_wall + (T_inf - T_wall) * prof
    prim = np.zeros((4, ny, nx))
    prim[0] = (1.0 / gamma / Tprof)[:, None]
    prim[1] = (U * prof)[:, None]
    prim[3] = 1.0 / gamma
    inflow = np.stack([prim[0][:, 0], prim[1][:, 0], prim[2][:, 0], prim[3][:, 0]], axis=1)
    beta, r2, p2, M2 = _oblique_shock(M, math.radians(theta_deg), gamma)
    c2 = math.sqrt(gamma * (p2 / gamma) / r2)
    th = math.radians(theta_deg)
    post = (r2, M2 * c2 * math.cos(th), -M2 * c2 * math.sin(th), p2 / gamma)
    free = (1.0, U, 0.0, 1.0 / gamma)
    top = np.array([post if x >= x_shock else free for x in xc])
    # log-law k-omega, beta* = 0.09, kappa = 0.41, c_f = 0.0016
    bstar, kap = 0.09, 0.41
    utau = U * math.sqrt(0.0016 / 2.0)
    nu_w = mu * gamma * T_wall  # mu / rho_wall, rho_wall = p / T_wall
    yplus = yc * utau / nu_w
    om_sub = 6.0 * nu_w / (0.075 * yc ** 2)
    om_log = utau / (math.sqrt(bstar) * kap * yc)
    omega = np.maximum(om_sub, om_log)
    kprof = utau ** 2 / math.sqrt(bstar) * np.minimum(1.0, (yplus / 10.0) ** 2)
    kprof = np.where(yc < delta, kprof, 1e-6 * U * U)
    omega = np.where(yc < delta, omega, U / delta)
    f1 = np.repeat(kprof[:, None], nx, axis=1)
    f2 = np.repeat(omega[:, None], nx, axis=1)
    bc = [[3, 4], [2, 3]]
    bc_prim = [[inflow, None], [None, top]]
    return dict(dim=2, n=(nx, ny), dx=[dx, dy], bc=bc, bc_prim=bc_prim, prim=prim, T_wall=T_wall, mu=mu,
                f1=f1.astype(np.float32).astype(np.float64), f2=f2.astype(np.float32).astype(np.float64))


# ------------------------------------------------------------------------------------------------
# Curvilinear (body-fitted) 2D grids: node arrays nodes[n1 + 1, n0 + 1, 2] = (x, y), right-handed
# ------------------------------------------------------------------------------------------------
def shock_boundary_layer_crop(nx, ny, full=(1024, 384)):
    """The wall corner of the full-size shock / boundary-layer workload: its first nx columns and ny
    rows (the same cell sizes, so the same wall-clustered first rows, time step and physical time
    per step), inflow rows and wall as in the full grid, outflow on the right, and the full grid's
    initial state just above the crop as Dirichlet data on top."""
    f = shock_boundary_layer(*full)
    prim = np.ascontiguousarray(f["prim"][:, :ny, :nx])
    inflow = np.ascontiguousarray(f["bc_prim"][0][0][:ny])
    top = np.ascontiguousarray(f["prim"][:, ny, :nx].T)
    return dict(dim=2, n=(nx, ny), dx=[f["dx"][0][:nx].copy(), f["dx"][1][:ny].copy()], bc=[[3, 4], [2, 3]],
                bc_prim=[[inflow, None], [None, top]], prim=prim, T_wall=f["T_wall"], mu=f["mu"],
                f1=np.ascontiguousarray(f["f1"][:ny, :nx]), f2=np.ascontiguousarray(f["f2"][:ny, :nx]))


def uniform_nodes(n0, n1, lx=1.0, ly=1.0):
    """The nodes of a uniform rectilinear grid on [0, lx] x [0, ly]."""
    X, Y = np.meshgrid(np.linspace(0.0, lx, n0 + 1), np.linspace(0.0, ly, n1 + 1), indexing="xy")
    return np.stack([X, Y], axis=-1)


def rectilinear_nodes(dx, dy):
    """The nodes of the tensor-product grid with column widths dx and row heights dy."""
    xs = np.concatenate([[0.0], np.cumsum(dx)])
    ys = np.concatenate([[0.0], np.cumsum(dy)])
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    return np.stack([X, Y], axis=-1)


def wavy_nodes(n0, n1, lx=1.0, ly=1.0, amp=0.03, shear=0.05):
    """A smoothly distorted grid on an lx x ly box that is periodic by translation:
    x = X + shear ly sin(2 pi Y/ly) + amp lx sin(2 pi X/lx) sin(2 pi Y/ly),
    y = Y + shear lx sin(2 pi X/lx) + amp ly sin(2 pi X/lx) sin(4 pi Y/ly);
    node (n0, j) is node (0, j) moved by (lx, 0), node (i, n1) is node (i, 0) moved by (0, ly).
    Cells are skewed by up to about 20 degrees and change area by up to about 40%."""
    U = uniform_nodes(n0, n1, lx, ly)
    X, Y = U[..., 0], U[..., 1]
    sx, sy = np.sin(2 * math.pi * X / lx), np.sin(2 * math.pi * Y / ly)
    x = X + shear * ly * sy + amp * lx * sx * sy
    y = Y + shear * lx * sx + amp * ly * sx * np.sin(4 * math.pi * Y / ly)
    return np.stack([x, y], axis=-1)


def rotate_nodes(nodes, theta):
    c, s = math.cos(theta), math.sin(theta)
    x, y = nodes[..., 0], nodes[..., 1]
    return np.stack([c * x - s * y, s * x + c * y], axis=-1)


def rotate_prim(prim, theta):
    """Primitive state (rho, u, v, p)[4, ...] with the velocity turned by theta."""
    c, s = math.cos(theta), math.sin(theta)
    out = np.array(prim, dtype=np.float64, copy=True)
    out[1] = c * prim[1] - s * prim[2]
    out[2] = s * prim[1] + c * prim[2]
    return out


def cell_points(nodes):
    """One sample point per cell (the mean of its four nodes), [n1, n0, 2]: where the input
    generators evaluate initial fields."""
    return 0.25 * (nodes[:-1, :-1] + nodes[:-1, 1:] + nodes[1:, :-1] + nodes[1:, 1:])


def smooth_state_at(points, seed, lx=1.0, ly=1.0, amp=0.1):
    """A smooth positive state periodic on the lx x ly box, evaluated at points[..., 2]."""
    rng = np.random.default_rng(seed)
    X = points[..., 0] * (2 * math.pi / lx)
    Y = points[..., 1] * (2 * math.pi / ly)
    f = lambda: sum(rng.normal() * np.cos(kx * X + ky * Y + rng.uniform(0, 6.28))
                    for kx, ky in ((1, 0), (0, 1), (1, 1), (2, -1)))
    prim = np.zeros((4,) + X.shape)
    prim[0] = 1.0 + amp * f()
    prim[1] = 0.3 * f()
    prim[2] = 0.3 * f()
    prim[3] = 1.0 + amp * f()
    return prim


def positive_fields_at(points, seed, lx=1.0, ly=1.0, k_ref=0.01, om_ref=20.0):
    """Smooth positive turbulence fields (k, second variable) periodic on the box."""
    rng = np.random.default_rng(seed)
    X = points[..., 0] * (2 * math.pi / lx)
    Y = points[..., 1] * (2 * math.pi / ly)
    g = lambda: sum(rng.normal() * np.cos(kx * X + ky * Y + rng.uniform(0, 6.28)) for kx, ky in ((1, 0), (0, 1), (1, -1)))
    return k_ref * np.exp(0.3 * g()), om_ref * np.exp(0.3 * g())


def _row_heights(ny, dy1, ratio, total):
    def heights(cap):
        return np.minimum(dy1 * ratio ** np.arange(ny), cap)
    lo, hi = dy1, total
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if heights(mid).sum() > total:
            hi = mid
        else:
            lo = mid
    h = heights(0.5 * (lo + hi))
    return h * (total / h.sum())


def compression_corner(nx, ny, alpha_deg=24.0, M=2.85, delta=0.1, Re_delta=1.6e6, ratio=1.08, dy1=2e-5,
                       xlen=2.0, ylen=1.0, gamma=GAMMA):
    """Supersonic compression corner in a channel (the geometry type of the paper's Settles cases;
    the exact experimental geometry is not an input here): the lower wall is flat for x < 0 and
    turns up by alpha at x = 0; the grid lines x = const run from the wall to the flat top y = ylen,
    rows clustered at the wall by the given growth ratio (first row dy1, as a fraction of the local
    channel height).  Isothermal no-slip lower wall, Dirichlet inflow carrying a 1/7-power boundary
    layer of thickness delta and log-law k, omega, supersonic outflow at the right and the top.
    Free stream rho = 1, p = 1/gamma (c = 1), u = M.  Returns nodes, primitives at the cells, the
    inflow state, k and omega."""
    xs = np.linspace(-0.5 * xlen, 0.5 * xlen, nx + 1)
    yw = np.where(xs > 0.0, xs * math.tan(math.radians(alpha_deg)), 0.0)
    eta = np.concatenate([[0.0], np.cumsum(_row_heights(ny, dy1, ratio, 1.0))])
    X = np.repeat(xs[None, :], ny + 1, axis=0)
    Y = yw[None, :] + (ylen - yw[None, :]) * eta[:, None]
    nodes = np.stack([X, Y], axis=-1)
    pts = cell_points(nodes)
    ywc = 0.5 * (yw[:-1] + yw[1:])
    dist = np.maximum(pts[..., 1] - ywc[None, :], 1e-12)  # distance above the wall along the grid line
    T_inf = 1.0 / gamma
    T_wall = T_inf * (1.0 + 0.89 * 0.5 * (gamma - 1.0) * M * M)
    mu = M * delta / Re_delta
    prof = np.where(dist < delta, (dist / delta) ** (1.0 / 7.0), 1.0)
    Tprof = T_wall + (T_inf - T_wall) * prof
    prim = np.zeros((4, ny, nx))
    prim[0] = 1.0 / gamma / Tprof
    prim[1] = M * prof
    prim[3] = 1.0 / gamma
    inflow = np.stack([prim[v][:, 0] for v in range(4)], axis=1)
    bstar, kap = 0.09, 0.41
    utau = M * math.sqrt(0.0016 / 2.0)
    nu_w = mu * gamma * T_wall
    om = np.maximum(6.0 * nu_w / (0.075 * dist ** 2), utau / (math.sqrt(bstar) * kap * dist))
    kk = utau ** 2 / math.sqrt(bstar) * np.minimum(1.0, (dist * utau / nu_w / 10.0) ** 2)
    kk = np.where(dist < delta, kk, 1e-6 * M * M)
    om = np.where(dist < delta, om, M / delta)
    bc = [[3, 4], [2, 4]]
    bc_prim = [[inflow, None], [None, None]]
    return dict(dim=2, n=(nx, ny), nodes=nodes, bc=bc, bc_prim=bc_prim, prim=prim, T_wall=T_wall, mu=mu,
                f1=kk.astype(np.float32).astype(np.float64), f2=om.astype(np.float32).astype(np.float64))


def naca0012_thickness(x):
    """Half thickness of the NACA 0012 section (closed trailing edge form of the four-digit formula)."""
    return 0.6 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1036 * x ** 4)


def naca0012_cgrid(n_wake, n_surf, n_normal, R=5.0, x_out=6.0, dy1=2e-3, ratio=1.15):
    """A C-grid around a NACA 0012 section of unit chord (the grid type of the paper's aerofoil cases;
    the paper's own grids are not inputs here).  The inner grid line (j = 0) runs along the lower
    wake from x_out to the trailing edge, round the section (cosine spacing) and back along the
    upper wake; the outer line is y = -R for the lower wake, the half ellipse with centre (1, 0) and
    semi-axes (1 + R, R) round the section, and y = +R for the upper wake; grid lines join the two
    (vertical in the wake), rows clustered at the inner line.  n0 = 2 n_wake + n_surf (n_surf even),
    the first and last n_wake cells of the j-lo side form the wake cut."""
    assert n_surf % 2 == 0
    n0 = 2 * n_wake + n_surf
    xw = x_out - np.arange(n_wake + 1) * ((x_out - 1.0) / n_wake)  # x_out .. 1
    th_lo = np.linspace(0.0, math.pi, n_surf // 2 + 1)              # trailing edge -> leading edge
    th_up = np.linspace(math.pi, 2 * math.pi, n_surf // 2 + 1)
    inner, outer = [], []
    a = 1.0 + R
    for x in xw[:-1]:
        inner.append((x, 0.0))
        outer.append((x, -R))
    for th in th_lo[:-1]:
        x = 0.5 * (1.0 + math.cos(th))
        al = -0.5 * math.pi - 0.5 * th
        inner.append((x, -naca0012_thickness(x)))
        outer.append((1.0 + a * math.cos(al), R * math.sin(al)))
    for th in th_up[:-1]:
        x = 0.5 * (1.0 + math.cos(th))
        al = -math.pi - 0.5 * (th - math.pi)
        inner.append((x, naca0012_thickness(x)))
        outer.append((1.0 + a * math.cos(al), R * math.sin(al)))
    for x in xw[::-1]:
        inner.append((x, 0.0))
        outer.append((x, R))
    inner, outer = np.array(inner), np.array(outer)
    assert inner.shape[0] == n0 + 1
    inner[n_wake] = (1.0, 0.0)
    inner[n0 - n_wake] = (1.0, 0.0)
    eta = np.concatenate([[0.0], np.cumsum(_row_heights(n_normal, dy1, ratio, 1.0))])
    nodes = inner[None, :, :] + eta[:, None, None] * (outer - inner)[None, :, :]
    return nodes


def naca0012_case(n_wake, n_surf, n_normal, mach=0.8, alpha_deg=2.26, Re=9.0e6, gamma=GAMMA, **grid):
    """Flow round the C-grid section: uniform free stream (rho = 1, p = 1/gamma, |U| = mach) at
    incidence alpha, isothermal no-slip section at the free-stream stagnation temperature, wake cut,
    Dirichlet free stream on the outer line, outflow at the two wake ends; mu from Re on the chord;
    uniform free-stream k = 1e-4 |U|^2 and omega = 10 |U| (per unit chord)."""
    nodes = naca0012_cgrid(n_wake, n_surf, n_normal, **grid)
    n0, n1 = nodes.shape[1] - 1, nodes.shape[0] - 1
    al = math.radians(alpha_deg)
    free = (1.0, mach * math.cos(al), mach * math.sin(al), 1.0 / gamma)
    prim = np.zeros((4, n1, n0))
    for v in range(4):
        prim[v] = free[v]
    T_inf = 1.0 / gamma
    T_wall = T_inf * (1.0 + 0.5 * (gamma - 1.0) * mach * mach)
    outer = np.tile(free, (n0, 1))
    return dict(dim=2, n=(n0, n1), nodes=nodes, bc=[[4, 4], [2, 3]], bc_prim=[[None, None], [None, outer]],
                prim=prim, T_wall=T_wall, mu=mach / Re, wake_cut=n_wake,
                dx=[np.full(n0, 1.0 / n0), np.full(n1, 1.0 / n1)],
                f1=np.full(n0 * n1, 1e-4 * mach * mach), f2=np.full(n0 * n1, 10.0 * mach))


# ------------------------------------------------------------------------------------------------
# Serving request stream
# ------------------------------------------------------------------------------------------------
def turbulence_1d(n, seed, k0=8.0, mach=0.3, gamma=GAMMA):
    """Periodic 1D random-phase velocity with E(k) ~ k^4 exp(-2 (k/k0)^2), rho = 1, p = 1/gamma."""
    rng = np.random.default_rng(seed)
    k = np.fft.rfftfreq(n, d=1.0 / n)
    amp = np.sqrt(k ** 4 * np.exp(-2.0 * (k / k0) ** 2))
    uh = amp * np.exp(1j * rng.uniform(0, 2 * math.pi, k.size))
    uh[0] = 0.0
    u = np.fft.irfft(uh, n)
    u *= mach / max(np.sqrt(np.mean(u * u)), 1e-300)
    prim = np.zeros((3, n))
    prim[0] = 1.0
    prim[1] = u
    prim[2] = 1.0 / gamma
    return dict(dim=1, n=(n,), dx=[np.full(n, 2 * math.pi / n)], bc=[[0, 0]], prim=prim,
                lo=[0.0], hi=[2 * math.pi])


def serving_request(i, seed):
    """Request i of the seeded serving stream: 50% 1D with n log-uniform in [256, 4096], 50% 2D with
    n^2 log-uniform in [64^2, 512^2]; Sod, Riemann quadrant (2D only) or periodic turbulence; steps
    uniform in [50, 500].  Returns a spec with the initial primitive state and run parameters."""
    rng = np.random.default_rng([seed, i])
    steps = int(rng.integers(50, 501))
    if rng.random() < 0.5:
        n = int(round(math.exp(rng.uniform(math.log(256), math.log(4096)))))
        if rng.random() < 0.5:
            s = sod_1d(n)
            s.update(lo=[0.0], hi=[1.0], kind="sod1d")
        else:
            s = turbulence_1d(n, seed=int(rng.integers(1 << 30)))
            s.update(kind="turb1d")
    else:
        n = int(round(math.exp(0.5 * rng.uniform(math.log(64 * 64), math.log(512 * 512)))))
        kind = rng.integers(3)
        if kind == 0:
            s = sod_2d(n)
            s.update(lo=[0.0, 0.0], hi=[1.0, 1.0], kind="sod2d")
        elif kind == 1:
            s = riemann_quadrant(n, seed=int(rng.integers(1 << 30)))
            s.update(lo=[0.0, 0.0], hi=[1.0, 1.0], kind="quadrant")
        else:
            s = turbulence(n, 2, seed=int(rng.integers(1 << 30)), k0=min(8.0, n / 8.0))
            s.update(lo=[0.0, 0.0], hi=[2 * math.pi, 2 * math.pi], kind="turb2d")
    s["nsteps"] = steps
    return s


def poisson_arrivals(count, rate, seed):
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))

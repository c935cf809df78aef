"""Seeded synthetic workloads for RBF mesh deformation (geometry only).

This module produces the inputs that both the CUDA path and the CPU oracle
consume: boundary (surface) points with their prescribed displacements and
volume points.  It contains none of the method's arithmetic (no basis
function, no interpolation, no grouping): it only builds point clouds.

The paper deforms the ONERA M6 wing (Sec. 4.1: 10,499 surface nodes,
1,353,105 volume nodes, first-layer height 1e-5) and the DLR-F6
wing-body-nacelle-pylon (Sec. 4.2: 79,079 surface nodes, 4,007,571 volume
nodes).  Those meshes are public benchmark geometries that are not available
here, so these generators stand in for them with synthetic surfaces of the
same kind and comparable size:

* a swept, tapered half wing made of symmetric 12 %-thick 4-digit-style
  sections (root chord 0.8, taper 0.56, leading-edge sweep 30 deg, span 1);
* a wing-body-nacelle-pylon assembly built from a cylinder fuselage, the
  wing at 3x scale, an annular nacelle and a pylon plate.

Axes: x chordwise, y spanwise, z vertical.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# Wing planform and section
# ----------------------------------------------------------------------------
SPAN = 1.0
ROOT_CHORD = 0.8
TAPER = 0.56
SWEEP_DEG = 30.0
THICKNESS = 0.12


def chord_at(y, span=SPAN, root_chord=ROOT_CHORD, taper=TAPER):
    """Local chord c(y) = c_r (1 - (1 - lambda) y / b)."""
    return root_chord * (1.0 - (1.0 - taper) * np.asarray(y) / span)


def leading_edge_x(y, sweep_deg=SWEEP_DEG):
    """Leading-edge x position x_LE(y) = y tan(sweep)."""
    return np.asarray(y) * math.tan(math.radians(sweep_deg))


def half_thickness(xc, tau=THICKNESS):
    """Symmetric 4-digit half-thickness t(x/c), closed trailing edge.

    Standard NACA 4-digit thickness polynomial with the closed-trailing-edge
    last coefficient, so t(0) = t(1) = 0.
    """
    xc = np.clip(np.asarray(xc, dtype=np.float64), 0.0, 1.0)
    return 5.0 * tau * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc**2
                        + 0.2843 * xc**3 - 0.1036 * xc**4)


def section_ring(n_chord):
    """Unit-chord section contour: (x/c, z/c) for theta_i = 2 pi i / n_chord.

    x/c = (1 + cos theta)/2, upper surface (z > 0) for theta in (0, pi), lower
    for theta in (pi, 2 pi).  i = 0 is the single trailing-edge point; for even
    n_chord, i = n_chord/2 is the leading edge.  No two ring points coincide.
    """
    theta = 2.0 * np.pi * np.arange(n_chord) / n_chord
    xc = 0.5 * (1.0 + np.cos(theta))
    sign = np.where(theta < np.pi, 1.0, -1.0)
    zc = sign * half_thickness(xc)
    return xc, zc


def wing_surface(n_span, n_chord, *, span=SPAN, root_chord=ROOT_CHORD,
                 taper=TAPER, sweep_deg=SWEEP_DEG, origin=(0.0, 0.0, 0.0),
                 scale=1.0):
    """Structured half-wing surface: n_span stations x n_chord ring points.

    Returns (points (n_span*n_chord, 3) float64, normals (same), station y of
    each point in the unscaled wing frame).  Station s lies at
    y_s = b s / (n_span - 1).  Normals are outward unit normals of the section
    contour in the x-z plane (central differences around the ring).
    """
    xc, zc = section_ring(n_chord)
    ys = span * np.arange(n_span) / max(n_span - 1, 1)
    c = chord_at(ys, span, root_chord, taper)[:, None]
    xle = leading_edge_x(ys, sweep_deg)[:, None]
    x = xle + xc[None, :] * c
    z = zc[None, :] * c
    y = np.broadcast_to(ys[:, None], x.shape)
    pts = np.stack([x, y, z], axis=-1).reshape(-1, 3)
    # ring tangent by central differences; outward normal of a counter-clockwise
    # contour in the (x, z) plane is (dz, -dx)
    xn = np.roll(x, -1, axis=1) - np.roll(x, 1, axis=1)
    zn = np.roll(z, -1, axis=1) - np.roll(z, 1, axis=1)
    nrm = np.stack([zn, np.zeros_like(xn), -xn], axis=-1)
    nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
    nrm = nrm.reshape(-1, 3)
    y_station = np.repeat(ys, n_chord)
    o = np.asarray(origin, dtype=np.float64)
    return pts * scale + o, nrm, y_station


def inside_wing(p, *, span=SPAN, root_chord=ROOT_CHORD, taper=TAPER,
                sweep_deg=SWEEP_DEG, origin=(0.0, 0.0, 0.0), scale=1.0):
    """True where a point lies strictly inside the (scaled, shifted) wing."""
    q = (np.asarray(p, dtype=np.float64) - np.asarray(origin)) / scale
    x, y, z = q[..., 0], q[..., 1], q[..., 2]
    ok = (y >= 0.0) & (y <= span)
    yc = np.clip(y, 0.0, span)
    c = chord_at(yc, span, root_chord, taper)
    xle = leading_edge_x(yc, sweep_deg)
    xc = (x - xle) / c
    ok &= (xc > 0.0) & (xc < 1.0)
    return ok & (np.abs(z) < c * half_thickness(xc))


def wing_bending_twist(pts, *, span=SPAN, root_chord=ROOT_CHORD, taper=TAPER,
                       sweep_deg=SWEEP_DEG, bend=0.05, twist_deg=5.0,
                       origin=(0.0, 0.0, 0.0), scale=1.0):
    """Prescribed surface displacement: quadratic bending plus linear twist.

    dz_bend = bend * scale * (y/b)^2; twist angle theta(y) = twist_deg * y/b
    (nose up positive) about the quarter-chord line
    x_qc = x_LE + c/4.  Returns (n, 3) float64 with dy = 0.
    """
    p = np.asarray(pts, dtype=np.float64)
    o = np.asarray(origin, dtype=np.float64)
    q = (p - o) / scale
    yb = np.clip(q[:, 1] / span, 0.0, 1.0)
    c = chord_at(yb * span, span, root_chord, taper)
    xqc = leading_edge_x(yb * span, sweep_deg) + 0.25 * c
    th = math.radians(twist_deg) * yb
    dxq = (q[:, 0] - xqc) * scale
    zq = q[:, 2] * scale
    d = np.zeros_like(p)
    d[:, 0] = dxq * (np.cos(th) - 1.0) + zq * np.sin(th)
    d[:, 2] = -dxq * np.sin(th) + zq * (np.cos(th) - 1.0) + bend * scale * yb**2
    return d


def wing_sine_mode(pts, *, span=SPAN, root_chord=ROOT_CHORD, taper=TAPER,
                   sweep_deg=SWEEP_DEG, twist_max_deg=30.0):
    """The paper's bending-twisting mode of Sec. 4.1 (Eqs. 7-8) in this
    module's axes (y spanwise, z up): bending dz = 0.05 y sin(pi y / (2 b))
    and twist theta = theta_m sin(pi y / (2 b)) about the quarter-chord line,
    with b the root chord and theta_m = 30 deg.  Returns (n, 3) float64."""
    p = np.asarray(pts, dtype=np.float64)
    b = root_chord
    y = np.clip(p[:, 1], 0.0, span)
    s = np.sin(np.pi * y / (2.0 * b))
    c = chord_at(y, span, root_chord, taper)
    xqc = leading_edge_x(y, sweep_deg) + 0.25 * c
    th = math.radians(twist_max_deg) * s
    dx = p[:, 0] - xqc
    d = np.zeros_like(p)
    d[:, 0] = dx * (np.cos(th) - 1.0) + p[:, 2] * np.sin(th)
    d[:, 2] = -dx * np.sin(th) + p[:, 2] * (np.cos(th) - 1.0) + 0.05 * p[:, 1] * s
    return d


# ----------------------------------------------------------------------------
# Volume points
# ----------------------------------------------------------------------------
def volume_uniform_box(n, lo, hi, rng, reject):
    """n points uniform in the box [lo, hi] with reject(p) == False."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    out = []
    have = 0
    while have < n:
        p = lo + (hi - lo) * rng.random((max(2 * (n - have), 1024), 3))
        p = p[~reject(p)]
        out.append(p)
        have += len(p)
    return np.concatenate(out)[:n]


def volume_log_clustered(n, surf_pts, surf_nrm, rng, reject, d_min=1e-5,
                         d_max=1.5):
    """n points offset from random surface points along their normals.

    The offset is d = d_min (d_max/d_min)^u with u ~ U(0, 1), so points are
    log-uniformly clustered toward the surface (the paper's meshes have a
    first-layer height of 1e-5).  Points with reject(p) True are redrawn.
    """
    out = []
    have = 0
    ns = len(surf_pts)
    while have < n:
        k = max(2 * (n - have), 1024)
        idx = rng.integers(0, ns, size=k)
        u = rng.random(k)
        d = d_min * (d_max / d_min) ** u
        p = surf_pts[idx] + d[:, None] * surf_nrm[idx]
        p = p[~reject(p)]
        out.append(p)
        have += len(p)
    return np.concatenate(out)[:n]


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------
def wing_case(n_span, n_chord, n_vol, *, vol_seed, vol_kind="box",
              radius=2.0, tol_rel=1e-3):
    """One synthetic wing deformation problem.

    Returns a dict with float64 arrays ``xb`` (N_b, 3), ``db`` (N_b, 3),
    ``xv`` (N_v, 3), the support radius and the relative tolerance.
    """
    xb, nb_, _ = wing_surface(n_span, n_chord)
    db = wing_bending_twist(xb)
    rng = np.random.Generator(np.random.PCG64(vol_seed))
    if n_vol == 0:
        xv = np.zeros((0, 3))
    elif vol_kind == "box":
        lo, hi = xb.min(0), xb.max(0)
        ctr = 0.5 * (lo + hi)
        side = 3.0 * max(hi[0] - lo[0], hi[1] - lo[1])
        xv = volume_uniform_box(n_vol, ctr - side / 2, ctr + side / 2, rng,
                                inside_wing)
    else:
        xv = volume_log_clustered(n_vol, xb, nb_, rng, inside_wing,
                                  d_max=1.5 * SPAN)
    return dict(xb=xb, db=db, xv=xv, radius=float(radius),
                tol_rel=float(tol_rel), name=f"wing{n_span}x{n_chord}")


def wing_small(n_vol=20_000):
    """Plain-greedy wing: 16 x 125 = 2,000 surface points, 20k box points,
    R = 2 x span, tolerance 1e-3 of the largest displacement, seed 0."""
    return wing_case(16, 125, n_vol, vol_seed=0, vol_kind="box", radius=2.0,
                     tol_rel=1e-3)


def wing_gcb(n_vol=2_000_000):
    """GCB wing: 100 x 500 = 50,000 surface points, volume log-clustered
    toward the surface (2e6 points, seed 2), R = 2, tolerance 1e-4."""
    return wing_case(100, 500, n_vol, vol_seed=2, vol_kind="log", radius=2.0,
                     tol_rel=1e-4)


def tiny_wing(n_span=4, n_chord=20, n_vol=200, seed=0, radius=2.0,
              tol_rel=1e-3):
    """A small wing for brute-force and unit checks."""
    return wing_case(n_span, n_chord, n_vol, vol_seed=seed, vol_kind="box",
                     radius=radius, tol_rel=tol_rel)


# ----------------------------------------------------------------------------
# Wing-body-nacelle-pylon assembly (stand-in for the Sec. 4.2 configuration)
# ----------------------------------------------------------------------------
WBNP_FUS_LEN = 6.0          # fuselage: cylinder along x in [0, 6]
WBNP_FUS_R = 0.35
WBNP_WING_SCALE = 3.0       # the unit wing at 3x scale (span 3)
WBNP_WING_ORIGIN = (2.2, 0.0, 0.50)   # root leading edge, lower surface clears the fuselage
WBNP_NAC_Y = 1.0            # nacelle axis: spanwise station, height, length, radii
WBNP_NAC_Z = 0.05
WBNP_NAC_LEN = 0.6
WBNP_NAC_R_OUT = 0.15
WBNP_NAC_R_IN = 0.13
WBNP_PYL_HALF = 0.01        # pylon plate: half thickness, z range
WBNP_PYL_Z = (0.21, 0.36)


def _wbnp_frame():
    """Nacelle and pylon x ranges, tied to the wing's leading edge at the
    nacelle station."""
    s = WBNP_WING_SCALE
    xle = WBNP_WING_ORIGIN[0] + s * float(leading_edge_x(WBNP_NAC_Y / s))
    nac_x = (xle - 0.35, xle - 0.35 + WBNP_NAC_LEN)
    pyl_x = (xle - 0.15, xle + 0.20)
    return nac_x, pyl_x


def _ring_surface(x0, x1, n_ax, n_circ, yc, zc, r, outward=True):
    """Points of a circular cylinder about the x-parallel axis (yc, zc),
    n_ax stations x n_circ angles, with unit normals (outward = away from
    the axis)."""
    xs = x0 + (x1 - x0) * np.arange(n_ax) / max(n_ax - 1, 1)
    ang = 2.0 * np.pi * np.arange(n_circ) / n_circ
    cy, sz = np.cos(ang), np.sin(ang)
    x = np.repeat(xs, n_circ)
    y = yc + r * np.tile(cy, n_ax)
    z = zc + r * np.tile(sz, n_ax)
    sg = 1.0 if outward else -1.0
    nrm = np.stack([np.zeros_like(x), sg * np.tile(cy, n_ax), sg * np.tile(sz, n_ax)], axis=-1)
    return np.stack([x, y, z], axis=-1), nrm


def _plate(x0, x1, z0, z1, n_x, n_z, y):
    xs = x0 + (x1 - x0) * np.arange(n_x) / max(n_x - 1, 1)
    zs = z0 + (z1 - z0) * np.arange(n_z) / max(n_z - 1, 1)
    x = np.repeat(xs, n_z)
    z = np.tile(zs, n_x)
    return np.stack([x, np.full_like(x, y), z], axis=-1)


def inside_wbnp(p):
    """True where a point lies inside a component of the assembly (the
    fuselage cylinder, the wing, the nacelle wall or the pylon plate)."""
    p = np.asarray(p, dtype=np.float64)
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    fus = (x >= 0.0) & (x <= WBNP_FUS_LEN) & (y * y + z * z < WBNP_FUS_R**2)
    wing = inside_wing(p, origin=WBNP_WING_ORIGIN, scale=WBNP_WING_SCALE)
    nac_x, pyl_x = _wbnp_frame()
    rn = np.sqrt((y - WBNP_NAC_Y) ** 2 + (z - WBNP_NAC_Z) ** 2)
    nac = (x >= nac_x[0]) & (x <= nac_x[1]) & (rn > WBNP_NAC_R_IN) & (rn < WBNP_NAC_R_OUT)
    pyl = ((x >= pyl_x[0]) & (x <= pyl_x[1]) & (np.abs(y - WBNP_NAC_Y) < WBNP_PYL_HALF)
           & (z >= WBNP_PYL_Z[0]) & (z <= WBNP_PYL_Z[1]))
    return fus | wing | nac | pyl


def wbnp_surface(density=1.0):
    """Surface points of the assembly, their outward normals, prescribed
    displacements and component labels (0 fuselage, 1 wing, 2 nacelle,
    3 pylon).

    At density 1: fuselage 300 x 400 = 120,000 points; wing 200 x 600 =
    120,000; nacelle outer and inner walls 2 x 100 x 200 = 40,000; pylon two
    faces 2 x 100 x 100 = 20,000; 300,000 in all.  ``density`` scales every
    count by sqrt(density) per direction.

    Displacement: the wing bends by 0.15 (y/b)^2 (b = 3) and twists 5 deg
    linearly about its quarter chord (the unit wing's field at 3x scale);
    nacelle and pylon translate rigidly by the wing's bending at the nacelle
    station; the fuselage is fixed.
    """
    f = math.sqrt(density)
    n = lambda k: max(2, int(round(k * f)))
    s = WBNP_WING_SCALE
    fus, fus_n = _ring_surface(0.0, WBNP_FUS_LEN, n(300), n(400), 0.0, 0.0, WBNP_FUS_R)
    wing, wing_n, _ = wing_surface(n(200), n(600), origin=WBNP_WING_ORIGIN, scale=s)
    nac_x, pyl_x = _wbnp_frame()
    nac_o, nac_on = _ring_surface(nac_x[0], nac_x[1], n(100), n(200), WBNP_NAC_Y, WBNP_NAC_Z,
                                  WBNP_NAC_R_OUT)
    nac_i, nac_in = _ring_surface(nac_x[0], nac_x[1], n(100), n(200), WBNP_NAC_Y, WBNP_NAC_Z,
                                  WBNP_NAC_R_IN, outward=False)
    pyl_a = _plate(pyl_x[0], pyl_x[1], WBNP_PYL_Z[0], WBNP_PYL_Z[1], n(100), n(100),
                   WBNP_NAC_Y - WBNP_PYL_HALF)
    pyl_b = _plate(pyl_x[0], pyl_x[1], WBNP_PYL_Z[0], WBNP_PYL_Z[1], n(100), n(100),
                   WBNP_NAC_Y + WBNP_PYL_HALF)
    pyl_an = np.tile([0.0, -1.0, 0.0], (len(pyl_a), 1))
    pyl_bn = np.tile([0.0, 1.0, 0.0], (len(pyl_b), 1))
    pts = np.concatenate([fus, wing, nac_o, nac_i, pyl_a, pyl_b])
    nrm = np.concatenate([fus_n, wing_n, nac_on, nac_in, pyl_an, pyl_bn])
    lab = np.concatenate([np.zeros(len(fus), np.int8), np.ones(len(wing), np.int8),
                          np.full(len(nac_o) + len(nac_i), 2, np.int8),
                          np.full(len(pyl_a) + len(pyl_b), 3, np.int8)])
    d = np.zeros_like(pts)
    wsel = lab == 1
    d[wsel] = wing_bending_twist(pts[wsel], origin=WBNP_WING_ORIGIN, scale=s)
    rigid = 0.05 * s * (WBNP_NAC_Y / s) ** 2
    d[lab >= 2, 2] = rigid
    return pts, nrm, d, lab


def wbnp_case(n_vol=10_000_000, *, density=1.0, vol_seed=3, radius=6.0, tol_rel=1e-4):
    """Wing-body-nacelle-pylon problem: 300,000 surface points at density 1,
    n_vol volume points log-clustered toward all surfaces (offsets
    d = 1e-5 (4.5/1e-5)^u along the normals, points inside a component
    redrawn), R = 6, tolerance 1e-4 of the largest displacement."""
    xb, nrm, db, lab = wbnp_surface(density)
    rng = np.random.Generator(np.random.PCG64(vol_seed))
    if n_vol == 0:
        xv = np.zeros((0, 3))
    else:
        xv = volume_log_clustered(n_vol, xb, nrm, rng, inside_wbnp,
                                  d_max=1.5 * WBNP_WING_SCALE)
    return dict(xb=xb, db=db, xv=xv, labels=lab, radius=float(radius),
                tol_rel=float(tol_rel), name=f"wbnp{len(xb)}")


def wbnp_sine_mode(pts):
    """The paper's mode of Sec. 4.2 (Eq. 10) on the assembly, in this module's
    axes: every surface node moves vertically by
    dz = 0.3 c (y / b)^2 sin(8 pi y / b), b the span (3) and c the mean
    aerodynamic chord of the 3x-scale wing, 2/3 c_r (1 + l + l^2) / (1 + l)."""
    p = np.asarray(pts, dtype=np.float64)
    b = WBNP_WING_SCALE * SPAN
    cr = WBNP_WING_SCALE * ROOT_CHORD
    mac = 2.0 / 3.0 * cr * (1.0 + TAPER + TAPER ** 2) / (1.0 + TAPER)
    d = np.zeros_like(p)
    d[:, 2] = 0.3 * mac * (p[:, 1] / b) ** 2 * np.sin(8.0 * np.pi * p[:, 1] / b)
    return d


def wing_paper_mode_case(n_span=16, n_chord=125, n_vol=20_000, *, vol_seed=0,
                         radius=7.0, tol_abs=1e-6):
    """The synthetic wing under the Sec. 4.1 mode (Eqs. 7-8) with the paper's
    radius 7 and absolute tolerance 1e-6; box volume points as configuration 1."""
    c = wing_case(n_span, n_chord, n_vol, vol_seed=vol_seed, vol_kind="box", radius=radius)
    c["db"] = wing_sine_mode(c["xb"])
    c["tol_abs"] = float(tol_abs)
    c["name"] = f"wing{n_span}x{n_chord}-eq7-8"
    return c


def wbnp_paper_mode_case(n_vol=0, *, density=1.0, vol_seed=3, radius=5.0, tol_abs=2e-6):
    """The assembly under the Sec. 4.2 mode (Eq. 10) with the paper's radius 5
    and absolute tolerance 2e-6."""
    c = wbnp_case(n_vol, density=density, vol_seed=vol_seed, radius=radius)
    c["db"] = wbnp_sine_mode(c["xb"])
    c["tol_abs"] = float(tol_abs)
    c["name"] = f"wbnp{len(c['xb'])}-eq10"
    return c


def random_cloud(n, seed, scale=1.0):
    """n distinct points uniform in a cube of side ``scale`` (float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.random((n, 3))


def random_field(n, seed, sigma=1.0):
    """i.i.d. Gaussian (n, 3) field with standard deviation sigma."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return sigma * rng.standard_normal((n, 3))


def line_near_tie(n=64, big=10, near=50, rel=2.0 ** -35):
    """Nodes at (i, 0, 0), i = 0..n-1, all displaced by t = 2^-4 along x,
    except node ``big`` (2t, the largest displacement) and node ``near``
    (t (1 + rel)).  With support radius 1.5 the seed nodes are ``big``, n-1
    and the node farthest from both, and every node more than one step from a
    seed keeps its own displacement as its error.  So the next pick is decided
    by a relative difference ``rel`` (exactly representable, far above FP64
    rounding, below 2^-28), and the picks after it by exact ties."""
    t = 2.0 ** -4
    xb = np.zeros((n, 3))
    xb[:, 0] = np.arange(n, dtype=np.float64)
    db = np.zeros((n, 3))
    db[:, 0] = t
    db[big, 0] = 2.0 * t
    db[near, 0] = t * (1.0 + rel)
    return dict(xb=xb, db=db, radius=1.5, t=t, big=big, near=near,
                name=f"line{n}-near-tie")

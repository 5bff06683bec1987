"""Error metric for comparing moment fields of two runs (host-side numpy).

A field's error is max |got - want| divided by max(max |want|, 1e-3 * S), where
S is the largest per-node sum of the absolute terms of that moment: a moment
that cancels to below a thousandth of its own terms cannot be reproduced to a
fixed fraction of its value by sums taken in another order, so it is judged
against that floor. The two velocity and the two heat-flux components are
normalised jointly. The moments are those of Sec. 2 (density, velocity,
temperature, heat flux, shear stress).
"""
import numpy as np

FIELDS_2D = ("rho", "ux", "uy", "T", "qx", "qy", "sxy")
FIELDS_1D = ("rho", "ux", "T", "qx")
FIELDS_3D = FIELDS_2D + ("uz", "qz")


def _axis_velocities(Q1, zv):
    """Velocities of one axis with Q1 of them: -N..N, or on the 2N+2 hierarchy
    (zv) the odd integers -(Q1-1)..Q1-1."""
    if zv:
        return np.arange(-(Q1 - 1), Q1, 2)
    return np.arange(-((Q1 - 1) // 2), (Q1 - 1) // 2 + 1)


def term_scales(F, want, dims=2, q1x=None, zv=0):
    """Largest per-node sum of absolute terms of each moment of populations F
    (velocity-major array [Q, ny, nx] in 2D, [Q, nx] in 1D); want holds the
    moments in the order of FIELDS_2D / FIELDS_1D. q1x is the number of x
    velocities of an anisotropic product (default: the square lattice); zv the
    mask of axes on the 2N+2 hierarchy (1: x, 2: y)."""
    Q = F.shape[0]
    if dims == 3:
        Q1 = int(round(Q ** (1.0 / 3.0)))
        v = _axis_velocities(Q1, 0).astype(float)
        ex = (slice(None), None, None, None)
        cx = np.tile(v, Q1 * Q1)[ex]
        cy = np.tile(np.repeat(v, Q1), Q1)[ex]
        cz = np.repeat(v, Q1 * Q1)[ex]
        rho, ux, uy, uz = want[0], want[1], want[2], want[7]
        dx, dy, dz = cx - ux, cy - uy, cz - uz
        d2 = dx * dx + dy * dy + dz * dz
        su = max((np.abs(c) * F).sum(0).max() for c in (cx, cy, cz)) / rho.min()
        sq = 0.5 * (np.sqrt(d2) ** 3 * F).sum(0).max()
        return {"rho": F.sum(0).max(), "ux": su, "uy": su, "uz": su,
                "T": (d2 * F).sum(0).max() / 3 / rho.min(), "qx": sq, "qy": sq, "qz": sq,
                "sxy": (np.abs(dx * dy) * F).sum(0).max()}
    if dims == 2:
        Q1x = q1x or int(round(np.sqrt(Q)))
        Q1y = Q // Q1x
        cx = np.tile(_axis_velocities(Q1x, zv & 1), Q1y).astype(float)[:, None, None]
        cy = np.repeat(_axis_velocities(Q1y, zv & 2), Q1x).astype(float)[:, None, None]
        rho, ux, uy = want[0], want[1], want[2]
        dx, dy = cx - ux, cy - uy
        d2 = dx * dx + dy * dy
        su = max((np.abs(cx) * F).sum(0).max(), (np.abs(cy) * F).sum(0).max()) / rho.min()
        sq = 0.5 * (np.sqrt(d2) ** 3 * F).sum(0).max()
        return {"rho": F.sum(0).max(), "ux": su, "uy": su, "T": (d2 * F).sum(0).max() / 2 / rho.min(),
                "qx": sq, "qy": sq, "sxy": (np.abs(dx * dy) * F).sum(0).max()}
    N = (Q - 1) // 2
    c = np.arange(-N, N + 1).astype(float)[:, None]
    rho, ux = want[0], want[1]
    d = c - ux
    return {"rho": F.sum(0).max(), "ux": (np.abs(c) * F).sum(0).max() / rho.min(),
            "T": (d * d * F).sum(0).max() / rho.min(), "qx": 0.5 * (np.abs(d) ** 3 * F).sum(0).max()}


def rel_errors(got, want, dims=2, F=None, q1x=None, zv=0):
    """Per-field max |got - want| / max(max |want|, 1e-3 S); got maps field names
    to arrays, want is the stacked reference moments. F (populations of the
    reference) gives the term scales S; q1x and zv as in term_scales."""
    names = FIELDS_3D if dims == 3 else (FIELDS_2D if dims == 2 else FIELDS_1D)
    w = {n: want[i] for i, n in enumerate(names)}
    groups = {"ux": ("ux", "uy"), "uy": ("ux", "uy"), "qx": ("qx", "qy"), "qy": ("qx", "qy")}
    if dims == 3:
        groups = {k: ("ux", "uy", "uz") for k in ("ux", "uy", "uz")}
        groups.update({k: ("qx", "qy", "qz") for k in ("qx", "qy", "qz")})
    S = term_scales(F, want, dims, q1x, zv) if F is not None else {}
    out = {}
    for n in names:
        scale = max(np.abs(w[m]).max() for m in groups.get(n, (n,)) if m in w)
        scale = max(scale, 1e-3 * S.get(n, 0.0))
        out[n] = float(np.abs(got[n] - w[n]).max() / max(scale, 1e-300))
    return out


def plain_errors(got, want, dims=2):
    """Per-field max |got - want| / max |want| (the plain field max-norm, no
    floor); a field whose reference is zero everywhere reports None unless it
    is matched exactly (0.0)."""
    names = FIELDS_3D if dims == 3 else (FIELDS_2D if dims == 2 else FIELDS_1D)
    out = {}
    for i, n in enumerate(names):
        d = float(np.abs(got[n] - want[i]).max())
        m = float(np.abs(want[i]).max())
        out[n] = d / m if m > 0 else (0.0 if d == 0 else None)
    return out

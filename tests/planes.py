"""Parity statistics per region of the lattice: each non-periodic face plane
and the interior, next to the all-node relative L2 error.

A relative L2 error over all nodes dilutes a mistake confined to one face
plane by sqrt(plane nodes / all nodes); the boundary rules are where the
step passes differ most from one another, so every parity comparison also
reports each face plane and the interior on its own: the root-mean-square
error over the region's nodes divided by the root-mean-square value of the
reference over the whole field.  That is the all-node relative L2 error
with the region's nodes alone in the numerator, rescaled to the region's
size, so it is not diluted; and it stays meaningful on a plane whose
reference is (near) zero, such as the velocity on a wall at rest or on an
outlet the flow has not yet reached."""
import numpy as np


def regions(n, bc_lo, bc_hi):
    """(name, boolean mask [N]) for every non-periodic face plane, then the
    interior (the nodes on no non-periodic face)."""
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    r = (x.ravel(), y.ravel(), z.ravel())
    out, face = [], np.zeros(r[0].size, dtype=bool)
    for a in range(3):
        for side, bc in ((0, bc_lo[a]), (1, bc_hi[a])):
            if bc == 0:
                continue
            m = r[a] == (0 if side == 0 else n[a] - 1)
            out.append((f"axis {a} {'low' if side == 0 else 'high'} face", m))
            face |= m
    if (~face).any():
        out.append(("interior", ~face))
    return out


def _rel(a, b, rms):
    d = np.linalg.norm(a - b)
    return float(d / max(rms * np.sqrt(b.size), 1e-300))


def region_errors(rg, ug, ro, uo, n, bc_lo, bc_hi):
    """{region: (error of rho, error of u)}, each the region's RMS error over
    the field's RMS value; u is [3, N]."""
    rg, ro = np.asarray(rg), np.asarray(ro)
    ug, uo = np.asarray(ug).reshape(3, -1), np.asarray(uo).reshape(3, -1)
    rms_r = float(np.sqrt(np.mean(ro ** 2)))
    rms_u = float(np.sqrt(np.mean(uo ** 2)))
    return {name: (_rel(rg[m], ro[m], rms_r), _rel(ug[:, m], uo[:, m], rms_u))
            for name, m in regions(n, bc_lo, bc_hi)}


def assert_regions(rg, ug, ro, uo, n, bc_lo, bc_hi, tol, tag=""):
    errs = region_errors(rg, ug, ro, uo, n, bc_lo, bc_hi)
    bad = {k: v for k, v in errs.items() if not (v[0] < tol and v[1] < tol)}
    assert not bad, f"{tag} regions over {tol}: " + ", ".join(
        f"{k}: rho {v[0]:.2e} u {v[1]:.2e}" for k, v in bad.items())
    return errs

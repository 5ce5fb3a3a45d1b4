"""Sampled outputs of a large lattice that the oracle computes window by
window (test harness; no arithmetic of the method).

After k steps the state of a node depends only on the nodes within 3k + 2
of it: per step a population moves one node, the forcing reads the lattice
gradient of rho u one node further, and a boundary node's populations come
from its inner node, one more; the initial forcing history adds the same
once.  So the oracle run on a window of the lattice reproduces the full run
exactly on the window's core: the nodes at least R = 3k + 2 nodes inside
every side where the window cuts the lattice.  A side that is a real face of
the lattice keeps its rule; a cut side is periodic (when the window cuts both
sides of an axis) or an outflow (when the other side is a real face), and
whatever it does stays outside the core.
"""
import numpy as np


def grid_index(n, lo, size):
    """Flat node indices (axis 0 fastest) of the box lo .. lo + size - 1."""
    z, y, x = np.meshgrid(*(np.arange(lo[a], lo[a] + size[a]) for a in (2, 1, 0)), indexing="ij")
    return (x + n[0] * (y + n[1] * z)).ravel()


class Window:
    """A box of lattice n with its rules per side and its core.

    bc_lo / bc_hi are the lattice's rules; lo, size the box; R the radius of
    dependence."""

    def __init__(self, n, bc_lo, bc_hi, lo, size, R, outflow=3, periodic=0):
        self.n, self.lo, self.size = tuple(n), tuple(lo), tuple(size)
        self.idx = grid_index(n, lo, size)
        blo, bhi, clo, chi = [], [], [], []
        for a in range(3):
            real_lo = lo[a] == 0
            real_hi = lo[a] + size[a] == n[a]
            if real_lo and real_hi:
                blo.append(bc_lo[a])
                bhi.append(bc_hi[a])
                cut_lo = cut_hi = False
            elif bc_lo[a] == periodic:  # a periodic axis cut on both sides
                blo.append(periodic)
                bhi.append(periodic)
                cut_lo = cut_hi = True
            else:
                if not real_lo and not real_hi:
                    blo.append(periodic)
                    bhi.append(periodic)
                else:
                    blo.append(bc_lo[a] if real_lo else outflow)
                    bhi.append(bc_hi[a] if real_hi else outflow)
                cut_lo, cut_hi = not real_lo, not real_hi
            c0 = R if cut_lo else 0
            c1 = size[a] - (R if cut_hi else 0)
            assert c1 > c0, "window too small for its radius"
            clo.append(c0)
            chi.append(c1)
        self.bc_lo, self.bc_hi = tuple(blo), tuple(bhi)
        self.core = grid_index(self.size, clo, [chi[a] - clo[a] for a in range(3)])  # inside the window
        self.core_global = grid_index(n, [lo[a] + clo[a] for a in range(3)], [chi[a] - clo[a] for a in range(3)])

    def nodes(self, a):
        """[..., N] array of the lattice -> [..., window nodes]."""
        return np.ascontiguousarray(np.asarray(a)[..., self.idx])

    def face(self, axis, side, u):
        """Face array [3, face nodes] of face (axis, side) of the lattice ->
        the window's part of it (None when the window does not reach it)."""
        if self.lo[axis] + (self.size[axis] - 1 if side else 0) != (self.n[axis] - 1 if side else 0):
            return None
        a, b = sorted(((axis + 1) % 3, (axis + 2) % 3))
        ia = np.arange(self.lo[a], self.lo[a] + self.size[a])
        ib = np.arange(self.lo[b], self.lo[b] + self.size[b])
        sel = (ia[None, :] + self.n[a] * ib[:, None]).ravel()
        return np.ascontiguousarray(np.asarray(u)[:, sel])


def oracle_cycle(n, bc_lo, bc_hi, tau, charts, steps, win=None, rho0=None, u0=None):
    """The oracle through one cycle of a dynamic channel: init (rho0, u0 or
    rest) on charts[0] with its face velocities, steps[0] steps, the chart
    change to charts[1] with its face velocities, steps[1] steps; returns the
    Cartesian (rho, u) of the whole lattice, or of the window win."""
    import oracle
    sel = (lambda a: a) if win is None else win.nodes
    lo, hi = (bc_lo, bc_hi) if win is None else (win.bc_lo, win.bc_hi)
    o = oracle.Lattice(n if win is None else win.size, lo, hi, tau=tau)
    (c0, f0), (c1, f1) = charts

    def faces(f):
        for (a, s), u in f.items():
            o.set_face_velocity(a, s, u if win is None else win.face(a, s, u))

    o.set_metric(sel(c0.g6), sel(c0.dg18))
    faces(f0)
    o.init(None if rho0 is None else sel(rho0), None if u0 is None else sel(u0))
    o.step(steps[0])
    o.transform(sel(c1.g6), sel(c1.dg18), sel(c0.J9), sel(c1.J9))
    faces(f1)
    o.step(steps[1])
    return o.moments(sel(c1.J9))

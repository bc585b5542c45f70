"""Plain reference of dynamic h-adaptation (Sec. 3.4): refinement criteria,
forest adaptation with 2:1 balance, the mesh of a leaf set, the remap of a
nodal DG state between meshes and the refinement indicators of Sec. 4.4 and
Sec. 5.

TEST INFRASTRUCTURE ONLY: only the tests use it.  It shares no code with the
library (whose forest logic is C++ and whose remap is a CUDA kernel).

Forest: an nx0 x ny0 grid of coarse cells of size hx0 x hy0 with origin
(x0, y0); a leaf (l, I, J) is the cell [x0 + I hx0 / 2^l, ...] x [...] at
level l (the paper's mesh level n_K = l + 1).  Leaves are ordered along the
Morton curve of their lower-left corners on the grid of level max_level.

Criteria (Sec. 3.4): with eta_max = max eta_K, refine K when eta_K > theta_r
eta_max, l < max_level and H_K = max(hx, hy) > H_min; coarsen K when eta_K <
theta_c eta_max and l > 0 (refinement wins where both hold).  Four siblings
that are all leaves and all marked for coarsening merge into their parent.
Then leaves are split until every face joins leaves at most one level apart
(2:1 balance); the smallest balanced refinement is unique.

Remap: a cell that keeps its place keeps its values; a child takes its
parent's polynomial at its own support points (exact); a parent takes the L2
projection of its four children's polynomials onto its own space, with the
parent and child integrals taken by Gauss-Legendre rules exact for the
degree-2r products (conserving the integral of every field).
"""
from __future__ import annotations

import numpy as np

from .oracle import rule

FACES = ((-1, 0), (1, 0), (0, -1), (0, 1))


class Forest:
    def __init__(self, nx0, ny0, x0, y0, hx0, hy0, max_level, h_min=0.0, tags=(0, 0, 0, 0),
                 periodic=(False, False)):
        self.nx0, self.ny0, self.x0, self.y0 = nx0, ny0, x0, y0
        self.hx0, self.hy0, self.max_level, self.h_min = hx0, hy0, max_level, h_min
        self.tags, self.periodic = tags, periodic

    def size(self, l):
        return self.hx0 / (1 << l), self.hy0 / (1 << l)

    def geom(self, c):
        l, i, j = c
        hx, hy = self.size(l)
        return self.x0 + i * hx, self.y0 + j * hy, hx, hy

    def wrap(self, l, i, j):
        nxl, nyl = self.nx0 << l, self.ny0 << l
        if self.periodic[0]:
            i %= nxl
        if self.periodic[1]:
            j %= nyl
        return (i, j) if (0 <= i < nxl and 0 <= j < nyl) else None

    @staticmethod
    def covering(leaves, l, i, j):
        while l >= 0:
            if (l, i, j) in leaves:
                return (l, i, j)
            l, i, j = l - 1, i // 2, j // 2
        return None

    def leaves_of_mesh(self, mesh):
        out = []
        for (x, y), (hx, hy) in zip(mesh.x0y0, mesh.hxhy):
            l = int(round(np.log2(self.hx0 / hx)))
            out.append((l, int(round((x - self.x0) / hx)), int(round((y - self.y0) / hy))))
        return out

    def order(self, leaves):
        L = self.max_level

        def key(c):
            l, i, j = c
            x, y = i << (L - l), j << (L - l)
            k = 0
            for bit in range(30):
                k |= ((x >> bit) & 1) << (2 * bit) | ((y >> bit) & 1) << (2 * bit + 1)
            return k

        return sorted(leaves, key=key)

    def flags(self, leaves, eta, theta_r, theta_c):
        """+1 refine, -1 coarsen, 0 keep (Sec. 3.4 criteria)"""
        emax = max(eta)
        out = []
        for (l, i, j), e in zip(leaves, eta):
            hx, hy = self.size(l)
            if e > theta_r * emax and l < self.max_level and max(hx, hy) > self.h_min:
                out.append(1)
            elif e < theta_c * emax and l > 0:
                out.append(-1)
            else:
                out.append(0)
        return out

    def adapt(self, leaves, flags):
        kids = lambda c: [(c[0] + 1, 2 * c[1] + a, 2 * c[2] + b) for b in (0, 1) for a in (0, 1)]
        S = set()
        for c, f in zip(leaves, flags):
            S.update(kids(c) if f == 1 else [c])
        marked = {c for c, f in zip(leaves, flags) if f == -1}
        parents = {(l - 1, i // 2, j // 2) for (l, i, j) in marked}
        for p in parents:
            ch = kids(p)
            if all(c in S and c in marked for c in ch):
                S.difference_update(ch)
                S.add(p)
        changed = True
        while changed:
            changed = False
            for c in list(S):
                if c not in S:
                    continue
                l, i, j = c
                for di, dj in FACES:
                    w = self.wrap(l, i + di, j + dj)
                    if w is None or self.covering(S, l, *w) is not None:
                        continue
                    # finer leaves there: the two level-(l+1) cells along the face must be leaves
                    ii, jj = w
                    if di != 0:
                        a = 0 if di > 0 else 1
                        along = [(l + 1, 2 * ii + a, 2 * jj + b) for b in (0, 1)]
                    else:
                        b = 0 if dj > 0 else 1
                        along = [(l + 1, 2 * ii + a, 2 * jj + b) for a in (0, 1)]
                    if not all(x in S for x in along):
                        S.remove(c)
                        S.update(kids(c))
                        changed = True
                        break
        return self.order(S)

    def mesh(self, leaves):
        """x0y0 [n, 2], hxhy [n, 2], nbr [n, 4, 2] of an ordered leaf list"""
        index = {c: k for k, c in enumerate(leaves)}
        S = set(leaves)
        n = len(leaves)
        x0y0 = np.zeros((n, 2))
        hxhy = np.zeros((n, 2))
        nbr = np.full((n, 4, 2), -1, dtype=np.int32)
        for k, c in enumerate(leaves):
            gx, gy, hx, hy = self.geom(c)
            x0y0[k] = (gx, gy)
            hxhy[k] = (hx, hy)
            l, i, j = c
            for f, (di, dj) in enumerate(FACES):
                w = self.wrap(l, i + di, j + dj)
                if w is None:
                    nbr[k, f, 0] = -1 - self.tags[f]
                    continue
                ii, jj = w
                if (l, ii, jj) in S:
                    nbr[k, f, 0] = index[(l, ii, jj)]
                elif l > 0 and (l - 1, ii // 2, jj // 2) in S:
                    nbr[k, f, 0] = index[(l - 1, ii // 2, jj // 2)]
                else:
                    if di != 0:
                        a = 0 if di > 0 else 1
                        along = [(l + 1, 2 * ii + a, 2 * jj + b) for b in (0, 1)]
                    else:
                        b = 0 if dj > 0 else 1
                        along = [(l + 1, 2 * ii + a, 2 * jj + b) for a in (0, 1)]
                    nbr[k, f, 0] = index[along[0]]
                    nbr[k, f, 1] = index[along[1]]
        return x0y0, hxhy, nbr


def _lagrange(xs, x):
    v = np.ones(len(xs))
    for a in range(len(xs)):
        for b in range(len(xs)):
            if b != a:
                v[a] *= (x - xs[b]) / (xs[a] - xs[b])
    return v


def _dlagrange(xs, x):
    """derivatives of the Lagrange polynomials (product rule)"""
    n = len(xs)
    d = np.zeros(n)
    for a in range(n):
        for k in range(n):
            if k == a:
                continue
            t = 1.0 / (xs[a] - xs[k])
            for b in range(n):
                if b != a and b != k:
                    t *= (x - xs[b]) / (xs[a] - xs[b])
            d[a] += t
    return d


def _eval(xs, u, xi, eta):
    """value of the nodal polynomial u [(r+1)^2] at reference (xi, eta)"""
    return float(np.outer(_lagrange(xs, eta), _lagrange(xs, xi)).ravel() @ u)


def remap(forest, old_leaves, old_fields, new_leaves, degree):
    """fields [k][n_old, nd] on old_leaves -> [k][n_new, nd] on new_leaves"""
    xs, _ = rule(1, degree + 1)
    xg, wg = rule(0, degree + 1)
    nd = (degree + 1) ** 2
    oidx = {c: k for k, c in enumerate(old_leaves)}
    # 1D mass matrix of the support basis, exact (Gauss-Legendre r+1 points)
    M1 = np.zeros((degree + 1, degree + 1))
    for q, wq in zip(xg, wg):
        lq = _lagrange(xs, q)
        M1 += wq * np.outer(lq, lq)
    Minv = np.kron(np.linalg.inv(M1), np.linalg.inv(M1))  # index a + (r+1) b
    out = [np.zeros((len(new_leaves), nd)) for _ in old_fields]
    for k, c in enumerate(new_leaves):
        if c in oidx:
            for f, u in enumerate(old_fields):
                out[f][k] = u[oidx[c]]
            continue
        anc = Forest.covering(oidx, *c)
        if anc is not None:  # a child: the ancestor's polynomial at the child's nodes
            la, ia, ja = anc
            l, i, j = c
            s = 1.0 / (1 << (l - la))
            for f, u in enumerate(old_fields):
                for b in range(degree + 1):
                    for a in range(degree + 1):
                        xi = (i * s - ia) + xs[a] * s
                        et = (j * s - ja) + xs[b] * s
                        out[f][k, a + (degree + 1) * b] = _eval(xs, u[oidx[anc]], xi, et)
            continue
        # a parent of four old leaves: L2 projection (reference measure of the parent)
        l, i, j = c
        kids = [(l + 1, 2 * i + a, 2 * j + b) for b in (0, 1) for a in (0, 1)]
        for f, u in enumerate(old_fields):
            rhs = np.zeros(nd)
            for (kl, ki, kj) in kids:
                ox, oy = ki - 2 * i, kj - 2 * j
                for qb, wb in zip(xg, wg):
                    for qa, wa in zip(xg, wg):
                        val = _eval(xs, u[oidx[(kl, ki, kj)]], qa, qb)
                        xi, et = 0.5 * (ox + qa), 0.5 * (oy + qb)
                        rhs += 0.25 * wa * wb * val * np.outer(_lagrange(xs, et),
                                                               _lagrange(xs, xi)).ravel()
            out[f][k] = Minv @ rhs
    return out


def _vel(h, eps):
    """desingularised velocity factor f(h) (Eq. velocity) and df/dh"""
    if h <= 0.0:
        return 0.0, 0.0
    if h >= eps:
        return 1.0 / h, -1.0 / (h * h)
    e4, h4 = eps ** 4, h ** 4
    return np.sqrt(2.0) * h / np.sqrt(e4 + h4), np.sqrt(2.0) * (e4 - h4) / (e4 + h4) ** 1.5


def indicator(ora, mesh, state, degree, kind, eps):
    """eta_K = max over the volume Gauss-Legendre points of |curl u| (kind 0,
    Sec. 4.4; u = f(h) q with h the sub-grid depth and grad h = A grad zeta) or
    of |grad c| (kind 1, Sec. 5)"""
    xs, _ = rule(1, degree + 1)
    xv, _ = rule(0, (3 * degree) // 2 + 1)
    nv = len(xv)
    zeta, qx, qy, c = state
    eta = np.zeros(mesh.n)

    def grad(u, xi, et, hx, hy):
        la, lb = _lagrange(xs, xi), _lagrange(xs, et)
        dla, dlb = _dlagrange(xs, xi), _dlagrange(xs, et)
        v = np.outer(lb, la).ravel() @ u
        gx = np.outer(lb, dla).ravel() @ u / hx
        gy = np.outer(dlb, la).ravel() @ u / hy
        return v, gx, gy

    for k in range(mesh.n):
        hx, hy = mesh.hxhy[k]
        best = 0.0
        for ib in range(nv):
            for ia in range(nv):
                xi, et = xv[ia], xv[ib]
                if kind == 1:
                    _, gx, gy = grad(c[k], xi, et, hx, hy)
                    val = np.hypot(gx, gy)
                else:
                    z, zx, zy = grad(zeta[k], xi, et, hx, hy)
                    u, ux_, uy_ = grad(qx[k], xi, et, hx, hy)
                    v, vx_, vy_ = grad(qy[k], xi, et, hx, hy)
                    V, A = ora.subgrid_point(k, 0, ia + nv * ib, z)
                    f, df = _vel(V, eps)
                    val = abs(f * (vx_ - uy_) + df * A * (v * zx - u * zy))
                best = max(best, val)
        eta[k] = best
    return eta

"""PyTorch (CPU, float64) restatement of the residual of Sec. 3.2, for the
discrete adjoint.

TEST INFRASTRUCTURE ONLY: only the tests use it.  It restates the same
definitions as ``swdg_oracle.c`` (which it is pinned against, value for value)
as dense tensor expressions, so that ``torch.autograd`` yields the exact
vector-Jacobian product of the discrete residual with respect to the nodal
state, the per-cell Manning coefficient n_K and a per-cell bathymetry offset
delta_K (every pixel depth of cell K, or every sampled depth in mode P,
shifted by delta_K).  It shares no code with the CUDA library.

Definitions (each evaluated directly, no sum factorisation):
  * basis: Lagrange polynomials on the r+1 Gauss-Lobatto support points
    (Sec. 3.2), evaluated at every quadrature or face point;
  * volume terms on the (floor(3r/2)+1)^2 Gauss-Legendre points, face terms
    on r+2 Gauss-Lobatto points per (sub)face (Eqs. mass_rhs, discharge_rhs,
    discharge_rhs_implicit, r_concentration);
  * sub-grid wet depth V_p(eta) = sum_k w_k max(eta + z_k + delta, 0) over the
    pixel-area fractions w_k of the sub-cell of point p (Sec. 3.3, Eq. mask;
    mode S) or max(eta + z_b(x_p) + delta, 0) (mode P);
  * Rusanov flux with the hydrostatic reconstruction h*+- = min of both
    sides' operators at that side's elevation (Eqs. lxf_parameter,
    hydro_rec_vars), the non-conservative pressure term (Eq.
    pressure_tumolo), the desingularised velocity (Eq. velocity) and Manning
    friction (Eq. manning);
  * wall and tidal-elevation ghost states on boundary faces;
  * optionally the tracer numerical diffusion -int nu_c h grad c . grad psi_i
    (Eq. numdiff).

Derivative conventions at the kinks (the reading the adjoint takes):
  * max(x, 0) inside V has derivative [x > 0] (Eq. mask's strict inequality);
  * the min of the reconstruction follows its first argument at ties (the
    side's own operator); the max of the wave speeds takes the mean of both
    sides' derivatives at an exact tie (the symmetric subgradient, which does
    not depend on the numbering of the cells);
  * |x| and sqrt(x) have derivative 0 at x = 0;
  * the constant-field rule (a field with equal nodal values is evaluated as
    that constant) is a rounding device: the polynomial is differentiated.
"""
from __future__ import annotations

import numpy as np
import torch

from .oracle import rule

NRM = ((-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0))


def _lagrange(xs, x):
    """values and derivatives of the Lagrange polynomials on nodes xs at x"""
    n = len(xs)
    v = np.ones(n)
    d = np.zeros(n)
    for a in range(n):
        for b in range(n):
            if b != a:
                v[a] *= (x - xs[b]) / (xs[a] - xs[b])
        for k in range(n):
            if k == a:
                continue
            t = 1.0 / (xs[a] - xs[k])
            for b in range(n):
                if b != a and b != k:
                    t *= (x - xs[b]) / (xs[a] - xs[b])
            d[a] += t
    return v, d


def _breaks(w):
    s = np.concatenate([[0.0], np.cumsum(w)])
    s[-1] = 1.0
    return s


def _fractions(lo, hi, P, Pmax):
    """overlap of [lo, hi] (pixel units of a tile) with pixels 0..P-1, divided by hi - lo"""
    f = np.zeros(Pmax)
    for i in range(P):
        o = min(hi, i + 1.0) - max(lo, float(i))
        if o > 0.0:
            f[i] = o / (hi - lo)
    return f


def _where_pos(x):
    return torch.where(x > 0, x, torch.zeros_like(x))


def _sqrt0(x):
    """sqrt with derivative 0 at 0 (x >= 0)"""
    pos = x > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, x, torch.ones_like(x))), torch.zeros_like(x))


def _min_first(a, b):
    return torch.where(a <= b, a, b)



def _max_sym(a, b):
    """max(a, b) whose derivative at an exact tie is the mean of both sides'
    (the symmetric element of the subdifferential); the value is unchanged"""
    return torch.where(a > b, a, torch.where(a < b, b, 0.5 * (a + b)))


class TorchResidual:
    """The residual (F, Gx, Gy, R, Lx, Ly) of one mesh + raster as a
    differentiable function of (zeta, qx, qy, c, manning, delta)."""

    def __init__(self, mesh, raster, degree, subgrid_mode=0, g=9.81, eps_vel=0.01,
                 boundaries=(), tracer_diffusivity=None):
        self.r = degree
        self.nd1 = degree + 1
        self.nd = self.nd1 ** 2
        self.mode = subgrid_mode
        self.g = g
        self.eps = eps_vel
        self.bc = {tag: (kind, amp, per, ph) for (tag, kind, amp, per, ph) in boundaries}
        self.nu = None if tracer_diffusivity is None else \
            torch.tensor(np.asarray(tracer_diffusivity, dtype=np.float64))[:, None]
        n = mesh.n
        self.n = n
        x0, y0 = mesh.x0y0[:, 0], mesh.x0y0[:, 1]
        hx, hy = mesh.hxhy[:, 0], mesh.hxhy[:, 1]
        self.hx, self.hy = hx, hy
        xs, _ = rule(1, self.nd1)
        xv, wv = rule(0, (3 * degree) // 2 + 1)
        xm, wm = rule(1, degree + 2)
        sv, sm = _breaks(wv), _breaks(wm)
        nv, nm = len(xv), len(xm)
        self.nm = nm
        z = np.asarray(raster.z, dtype=np.float64)
        self.raster = raster
        # ---- per-cell pixel tiles (mode S) or sampled depths (mode P)
        if subgrid_mode == 0:
            P = np.rint(hx / raster.dx).astype(int)
            i0 = np.rint((x0 - raster.xo) / raster.dx).astype(int)
            j0 = np.rint((y0 - raster.yo) / raster.dy).astype(int)
            Pmax = int(P.max())
            tiles = np.zeros((n, Pmax * Pmax))
            for k in range(n):
                t = z[j0[k]:j0[k] + P[k], i0[k]:i0[k] + P[k]]
                tt = np.zeros((Pmax, Pmax))
                tt[:P[k], :P[k]] = t
                tiles[k] = tt.ravel()
            self.P, self.Pmax = P, Pmax
            self.tiles = torch.tensor(tiles)

        self.x0, self.y0, self.z = x0, y0, z
        site = self.site

        # ---- volume points: basis rows and sites
        Bv, Dx, Dy, wts = [], [], [], []
        for ib in range(nv):
            for ia in range(nv):
                la, dla = _lagrange(xs, xv[ia])
                lb, dlb = _lagrange(xs, xv[ib])
                Bv.append(np.outer(lb, la).ravel())
                Dx.append(np.outer(lb, dla).ravel())
                Dy.append(np.outer(dlb, la).ravel())
                wts.append(wv[ia] * wv[ib])
        self.Bv = torch.tensor(np.array(Bv))   # [npv, nd]
        self.Dx = torch.tensor(np.array(Dx))
        self.Dy = torch.tensor(np.array(Dy))
        self.wv = torch.tensor(np.array(wts))
        self.vol_site = self.cell_sites(xv, sv)  # [n, npv, Pmax^2] or [n, npv]

        # ---- face points: one item per (cell, face, subface)
        items = []  # (K, f, nb, tag, t0, L)
        for k in range(n):
            for f in range(4):
                s0, s1 = int(mesh.nbr[k, f, 0]), int(mesh.nbr[k, f, 1])
                tang_x = f >= 2
                own_t0, own_L = (x0[k], hx[k]) if tang_x else (y0[k], hy[k])
                if s0 < 0:
                    items.append((k, f, -1, -1 - s0, own_t0, own_L))
                elif s1 >= 0:
                    for nb in (s0, s1):
                        t0, L = (x0[nb], hx[nb]) if tang_x else (y0[nb], hy[nb])
                        items.append((k, f, nb, 0, t0, L))
                else:
                    items.append((k, f, s0, 0, own_t0, own_L))
        self.items = items

        def face_ref(k, f, t):
            if f < 2:
                return (0.0 if f == 0 else 1.0), (t - y0[k]) / hy[k]
            return (t - x0[k]) / hx[k], (0.0 if f == 2 else 1.0)

        def face_site(k, f, t0, L, al):
            lo, hi, tp = t0 + sm[al] * L, t0 + sm[al + 1] * L, t0 + xm[al] * L
            if f < 2:
                X0, X1, px = ((x0[k], x0[k] + sm[1] * hx[k], x0[k]) if f == 0 else
                              (x0[k] + sm[nm - 1] * hx[k], x0[k] + hx[k], x0[k] + hx[k]))
                return site(k, X0, X1, lo, hi, px, tp)
            Y0, Y1, py = ((y0[k], y0[k] + sm[1] * hy[k], y0[k]) if f == 2 else
                          (y0[k] + sm[nm - 1] * hy[k], y0[k] + hy[k], y0[k] + hy[k]))
            return site(k, lo, hi, Y0, Y1, tp, py)

        Phi_m, Phi_p, s_m, s_p, wl = [], [], [], [], []
        for (k, f, nb, tag, t0, L) in items:
            pm, pp, am, ap, ww = [], [], [], [], []
            for al in range(nm):
                tp = t0 + xm[al] * L
                xi, et = face_ref(k, f, tp)
                la, _ = _lagrange(xs, xi)
                lb, _ = _lagrange(xs, et)
                pm.append(np.outer(lb, la).ravel())
                am.append(face_site(k, f, t0, L, al))
                if nb >= 0:
                    xn, en = face_ref(nb, f ^ 1, tp)
                    la, _ = _lagrange(xs, xn)
                    lb, _ = _lagrange(xs, en)
                    pp.append(np.outer(lb, la).ravel())
                    ap.append(face_site(nb, f ^ 1, t0, L, al))
                else:
                    pp.append(np.zeros(self.nd))
                    ap.append(am[-1])
                ww.append(L * wm[al])
            Phi_m.append(pm)
            Phi_p.append(pp)
            s_m.append(am)
            s_p.append(ap)
            wl.append(ww)
        self.iK = torch.tensor([it[0] for it in items])
        self.iN = torch.tensor([max(it[2], 0) for it in items])
        self.has_nb = torch.tensor([it[2] >= 0 for it in items])
        self.tag = [it[3] for it in items]
        self.nrm = torch.tensor([NRM[it[1]] for it in items])  # [ni, 2]
        self.Phi_m = torch.tensor(np.array(Phi_m))   # [ni, nm, nd]
        self.Phi_p = torch.tensor(np.array(Phi_p))
        self.site_m = torch.tensor(np.array(s_m))    # [ni, nm, (Pmax^2)]
        self.site_p = torch.tensor(np.array(s_p))
        self.wl = torch.tensor(np.array(wl))         # [ni, nm]

    # -- sampling sites: pixel-area fractions of a rectangle over cell k's tile
    # (mode S) or the bottom depth at a point (mode P)
    def _rect_w(self, k, X0, X1, Y0, Y1):
        ras = self.raster
        Pk = int(self.P[k])
        fx = _fractions((X0 - self.x0[k]) / ras.dx, (X1 - self.x0[k]) / ras.dx, Pk, self.Pmax)
        fy = _fractions((Y0 - self.y0[k]) / ras.dy, (Y1 - self.y0[k]) / ras.dy, Pk, self.Pmax)
        return np.outer(fy, fx).ravel()

    def _bilinear(self, x, y):
        ras, z = self.raster, self.z
        fi = min(max((x - ras.xo) / ras.dx - 0.5, 0.0), z.shape[1] - 1.0)
        fj = min(max((y - ras.yo) / ras.dy - 0.5, 0.0), z.shape[0] - 1.0)
        ii, jj = min(int(np.floor(fi)), z.shape[1] - 2), min(int(np.floor(fj)), z.shape[0] - 2)
        a, b = fi - ii, fj - jj
        return ((1 - a) * (1 - b) * z[jj, ii] + a * (1 - b) * z[jj, ii + 1] +
                (1 - a) * b * z[jj + 1, ii] + a * b * z[jj + 1, ii + 1])

    def site(self, k, X0, X1, Y0, Y1, px, py):
        if self.mode == 0:
            return self._rect_w(k, X0, X1, Y0, Y1)
        return self._bilinear(px, py)

    def cell_sites(self, xq, sq):
        """sites of the tensor rule (nodes xq, breakpoints sq) of every cell,
        point index ia + len(xq) ib"""
        m = len(xq)
        out = []
        for k in range(self.n):
            x0, y0, hx, hy = self.x0[k], self.y0[k], self.hx[k], self.hy[k]
            out.append([self.site(k, x0 + sq[ia] * hx, x0 + sq[ia + 1] * hx,
                                  y0 + sq[ib] * hy, y0 + sq[ib + 1] * hy,
                                  x0 + xq[ia] * hx, y0 + xq[ib] * hy)
                        for ib in range(m) for ia in range(m)])
        return torch.tensor(np.array(out))

    # -- sub-grid wet depth: site [a, q, ...] of cells k [a] at elevations eta [a, q]
    def V(self, site, k, eta, delta):
        e = eta + delta[k][:, None]
        if self.mode == 0:
            d = e[:, :, None] + self.tiles[k][:, None, :]
            return (site * _where_pos(d)).sum(-1)
        return _where_pos(e + site)

    def vel(self, h):
        e = self.eps
        pos = h > 0
        hs = torch.where(pos, h, torch.ones_like(h))
        h4 = hs ** 4
        small = np.sqrt(2.0) * hs / torch.sqrt(e ** 4 + h4)
        f = torch.where(hs >= e, 1.0 / hs, small)
        return torch.where(pos, f, torch.zeros_like(h))

    def gamma(self, n, h, qx, qy):
        e = self.eps
        pos = (h > 0) & (n != 0)
        hs = torch.where(h > 0, h, torch.ones_like(h))
        h4 = hs ** 4
        hdes = torch.where(hs >= e, hs, torch.sqrt(e ** 4 + h4) / (np.sqrt(2.0) * hs))
        gam = self.g * n * n * _sqrt0(qx * qx + qy * qy) / hdes ** (7.0 / 3.0)
        return torch.where(pos, gam, torch.zeros_like(gam))

    def __call__(self, zeta, qx, qy, c, manning, delta, t=0.0):
        g = self.g
        n = self.n
        hx = torch.tensor(self.hx)[:, None]
        hy = torch.tensor(self.hy)[:, None]
        J = hx * hy
        cells = torch.arange(n)
        # ---- volume terms
        z = zeta @ self.Bv.T
        zx = (zeta @ self.Dx.T) / hx
        zy = (zeta @ self.Dy.T) / hy
        vqx, vqy, vc = qx @ self.Bv.T, qy @ self.Bv.T, c @ self.Bv.T
        h = self.V(self.vol_site, cells, z, delta)
        f = self.vel(h)
        ux, uy = f * vqx, f * vqy
        gam = self.gamma(manning[:, None], h, vqx, vqy)
        w = J * self.wv[None, :]
        px = self.Dx[None] / hx[:, :, None]   # [n, npv, nd]
        py = self.Dy[None] / hy[:, :, None]
        ps = self.Bv[None]

        def integ(a, b, v):
            # sum_p w (a d_x psi + b d_y psi + v psi)
            out = 0.0
            if a is not None:
                out = out + torch.einsum("kp,kpi->ki", w * a, px)
            if b is not None:
                out = out + torch.einsum("kp,kpi->ki", w * b, py)
            if v is not None:
                out = out + torch.einsum("kp,kpi->ki", w * v, ps.expand(n, -1, -1))
            return out

        F = integ(vqx, vqy, None)
        Gx = integ(vqx * ux, vqx * uy, -g * h * zx)
        Gy = integ(vqy * ux, vqy * uy, -g * h * zy)
        R = integ(vc * vqx, vc * vqy, None)
        if self.nu is not None:  # tracer numerical diffusion (Eq. numdiff)
            cx, cy = (c @ self.Dx.T) / hx, (c @ self.Dy.T) / hy
            R = R - integ(self.nu * h * cx, self.nu * h * cy, None)
        Lx = integ(None, None, -gam * vqx)
        Ly = integ(None, None, -gam * vqy)
        # ---- face terms
        iK, iN = self.iK, self.iN
        nb = self.has_nb[:, None]
        zm = torch.einsum("aqi,ai->aq", self.Phi_m, zeta[iK])
        qxm = torch.einsum("aqi,ai->aq", self.Phi_m, qx[iK])
        qym = torch.einsum("aqi,ai->aq", self.Phi_m, qy[iK])
        cm = torch.einsum("aqi,ai->aq", self.Phi_m, c[iK])
        zp = torch.einsum("aqi,ai->aq", self.Phi_p, zeta[iN])
        qxp = torch.einsum("aqi,ai->aq", self.Phi_p, qx[iN])
        qyp = torch.einsum("aqi,ai->aq", self.Phi_p, qy[iN])
        cp = torch.einsum("aqi,ai->aq", self.Phi_p, c[iN])
        nx, ny = self.nrm[:, 0:1], self.nrm[:, 1:2]
        # ghost states of boundary faces
        zg, qxg, qyg = zm.clone(), qxm.clone(), qym.clone()
        for a, tag in enumerate(self.tag):
            if self.has_nb[a]:
                continue
            kind, amp, per, ph = self.bc.get(tag, (0, 0.0, 1.0, 0.0))
            if kind == 1:
                zg[a] = amp * np.sin(2.0 * np.pi * t / per + ph)
            else:
                qn = qxm[a] * nx[a] + qym[a] * ny[a]
                qxg[a] = qxm[a] - 2.0 * qn * nx[a]
                qyg[a] = qym[a] - 2.0 * qn * ny[a]
        zp = torch.where(nb, zp, zg)
        qxp = torch.where(nb, qxp, qxg)
        qyp = torch.where(nb, qyp, qyg)
        cp = torch.where(nb, cp, cm)
        # the "+" operator of a boundary face is the own one: its cell index is K
        kP = torch.where(self.has_nb, iN, iK)
        hm = self.V(self.site_m, iK, zm, delta)
        hp = self.V(self.site_p, kP, zp, delta)
        hsm = _min_first(hm, self.V(self.site_p, kP, zm, delta))
        hsp = _min_first(hp, self.V(self.site_m, iK, zp, delta))
        fm, fp = self.vel(hm), self.vel(hp)
        umx, umy, upx, upy = fm * qxm, fm * qym, fp * qxp, fp * qyp
        unm, unp = umx * nx + umy * ny, upx * nx + upy * ny
        # wave speed bound: at an exact tie the derivative is the mean of both
        # sides' (independent of which cell of the face is which)
        lam = _max_sym(torch.abs(unm) + _sqrt0(g * hm), torch.abs(unp) + _sqrt0(g * hp))
        qsmx, qsmy, qspx, qspy = hsm * umx, hsm * umy, hsp * upx, hsp * upy
        fF = 0.5 * ((qsmx + qspx) * nx + (qsmy + qspy) * ny) + 0.5 * lam * (hsm - hsp)
        pres = g * 0.5 * (hsm + hsp) * 0.5 * (hsm - hsp)
        fGx = 0.5 * (qsmx * unm + qspx * unp) + 0.5 * lam * (qsmx - qspx) - pres * nx
        fGy = 0.5 * (qsmy * unm + qspy * unp) + 0.5 * lam * (qsmy - qspy) - pres * ny
        fR = 0.5 * ((qsmx * cm + qspx * cp) * nx + (qsmy * cm + qspy * cp) * ny) + \
            0.5 * lam * (hsm * cm - hsp * cp)
        outs = []
        for base, fl in ((F, fF), (Gx, fGx), (Gy, fGy), (R, fR)):
            contrib = torch.einsum("aq,aqi->ai", self.wl * fl, self.Phi_m)
            outs.append(base.index_add(0, iK, -contrib))
        return outs[0], outs[1], outs[2], outs[3], Lx, Ly


def residual_vjp(tr: TorchResidual, state, manning, delta, cot, t=0.0):
    """(zeta_bar, qx_bar, qy_bar, c_bar, manning_bar, delta_bar) = the cotangents
    ``cot`` (F, Gx, Gy, R, Lx, Ly bars) pulled back through the residual"""
    xs = [torch.tensor(np.asarray(a, dtype=np.float64), requires_grad=True) for a in state]
    nman = torch.tensor(np.asarray(manning, dtype=np.float64), requires_grad=True)
    dl = torch.tensor(np.asarray(delta, dtype=np.float64), requires_grad=True)
    out = tr(*xs, nman, dl, t)
    s = sum((o * torch.tensor(np.asarray(b, dtype=np.float64))).sum() for o, b in zip(out, cot))
    grads = torch.autograd.grad(s, xs + [nman, dl], allow_unused=True)
    return [g.detach().numpy() if g is not None else np.zeros(v.shape)
            for g, v in zip(grads, xs + [nman, dl])]


def residual_value(tr: TorchResidual, state, manning, delta, t=0.0):
    with torch.no_grad():
        out = tr(*[torch.tensor(np.asarray(a, dtype=np.float64)) for a in state],
                 torch.tensor(np.asarray(manning, dtype=np.float64)),
                 torch.tensor(np.asarray(delta, dtype=np.float64)), t)
    return dict(zip(("F", "Gx", "Gy", "R", "Lx", "Ly"), [o.numpy() for o in out]))

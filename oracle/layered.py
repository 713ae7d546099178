"""Green's functions of a planar stratified background (the layered media of Table I: dielectric
layers on a perfectly conducting ground plane under air) for sources and observers in the same
layer, in the mixed-potential form the RWG / pulse Galerkin operators use. Test infrastructure
(oracle), FP64, exp(j w t), lengths in micrometres.

Transmission-line form (the spectral fields of a stratified medium are voltages and currents on
a TE and a TM line along z, one line section per layer). In layer n (bottom z_b, top z_t,
d = z_t - z_b, k_z = sqrt(k_n^2 - k_rho^2) with Im k_z <= 0) a unit shunt current source at z'
gives the voltage, and a unit series voltage source the current,
  V_i = (Z/2)   [e^{-j k_z |u|} + ( G_b e1 + G_t e2 + G_b G_t (e3 + e4)) / D]
  I_v = (1/2Z)  [e^{-j k_z |u|} + (-G_b e1 - G_t e2 + G_b G_t (e3 + e4)) / D]
with u = z - z', e1 = e^{-j k_z (z + z' - 2 z_b)}, e2 = e^{-j k_z (2 z_t - z - z')},
e3 = e^{-j k_z (2d + u)}, e4 = e^{-j k_z (2d - u)}, D = 1 - G_b G_t e^{-2 j k_z d}, and G_b, G_t the
reflection coefficients of the line seen downward at z_b and upward at z_t (the signs of the
four terms follow from continuity of V and the unit jump of I at the source, or the reverse).
Line impedances (normalised by eta0): TM Z^e = k_z / (k0 eps_n), TE Z^h = k0 / k_z.

Potentials (normalised so that in a homogeneous medium each equals G(k_n, R)):
  G^A_xx = G^A_yy = S0{ v^h / (2 j k_z) },                       v^h = the TE bracket of V_i
  G^A_zz = S0{ i^e / (2 j k_z) },                                 i^e = the TM bracket of I_v
  G^Phi  = S0{ (j / (2 k_rho^2 k_z)) [k_z^2 v^e - k_n^2 v^h] }    (charge potential, times eps_n)
with S0{f} = (1/2 pi) int_0^inf f(k_rho) J0(k_rho rho) k_rho dk_rho (Sommerfeld integral). The
x-z coupling G^A_zx of horizontal currents is not included.

Every function splits as G(rho, z, z') = G_T(rho, z - z') + G_H(rho, z + z'): the direct term and
the two doubly reflected terms (e3, e4) depend on z - z' (Toeplitz in z on a grid), the singly
reflected terms (e1, e2) on z + z' (Hankel). The direct term is the closed form G(k_n, R); the
reflected terms are integrated numerically: a half-ellipse in the first quadrant of the k_rho
plane from 0 to beyond every layer's wavenumber (away from the branch point of the top half-space
and the surface-wave poles, which lie on or below the real axis for exp(j w t)), then the real
axis, where the reflected terms decay as e^{-k_rho zeta} (zeta > 0 for points strictly inside
the layer), in Gauss-Legendre panels no longer than a fraction of the oscillation period of J0
and of the decay length.

On top of these: the grid step of the AIM inside a layer (LayeredGrid: Toeplitz tables by FFT
convolution, Hankel tables by convolution of the z-reversed sources), the Galerkin operators
of objects inside a layer (the free-space operators at the layer's wavenumber for the direct
term, the reflected parts by a 7-point rule on both triangles with tabulated, spline-
interpolated Green's functions), and the layered O-AIM with its precorrected near region.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import jv

_GL_X, _GL_W = np.polynomial.legendre.leggauss(16)


def _kz(k, kr):
    """sqrt(k^2 - k_rho^2) on the branch Im <= 0 (real and non-negative when propagating)."""
    q = np.sqrt(np.asarray(k, dtype=complex) ** 2 - np.asarray(kr, dtype=complex) ** 2)
    return np.where(q.imag > 0, -q, q)


def green(k, R):
    return np.exp(-1j * k * R) / (4.0 * math.pi * R)


class Stack:
    """Layers bottom-up, (thickness um, complex relative permittivity) each, on a PEC ground plane
    at z = 0 (ground=True) or on a lower half-space of permittivity bottom_eps; a half-space of
    permittivity top_eps above. Non-magnetic throughout."""

    def __init__(self, k0, layers, top_eps=1.0, ground=True, bottom_eps=1.0):
        self.k0 = float(k0)
        self.d = np.array([float(t) for t, _ in layers])
        self.eps = np.array([complex(e) for _, e in layers])
        self.top_eps = complex(top_eps)
        self.bottom_eps = complex(bottom_eps)
        self.ground = bool(ground)
        self.z = np.concatenate([[0.0], np.cumsum(self.d)])  # interfaces z_0 = 0 ... z_N

    def k(self, eps):
        k = self.k0 * np.sqrt(complex(eps))
        return -k if k.imag > 0 else k

    def layer_of(self, z):
        n = int(np.searchsorted(self.z, z, side="right")) - 1
        if n < 0 or n >= len(self.d) or not (self.z[n] < z < self.z[n + 1]):
            raise ValueError("points must lie strictly inside a layer")
        return n

    def _Z(self, eps, kr, pol):
        kz = _kz(self.k(eps), kr)
        return kz / (self.k0 * eps) if pol == "e" else self.k0 / kz

    def gammas(self, n, kr, pol):
        """(G_b, G_t) of layer n for the TM ('e') or TE ('h') line at k_rho (array)."""
        kr = np.asarray(kr, dtype=complex)
        # downward: from the ground (short, -1) or the lower half-space, up to layer n's bottom
        if self.ground:
            g = -np.ones_like(kr)
        else:
            Zb, Z0 = self._Z(self.bottom_eps, kr, pol), self._Z(self.eps[0], kr, pol)
            g = (Zb - Z0) / (Zb + Z0)
        for l in range(1, n + 1):
            kzl = _kz(self.k(self.eps[l - 1]), kr)
            gl = g * np.exp(-2j * kzl * self.d[l - 1])  # at the top of layer l - 1
            Zl1, Zl = self._Z(self.eps[l - 1], kr, pol), self._Z(self.eps[l], kr, pol)
            r = (Zl1 - Zl) / (Zl1 + Zl)
            g = (r + gl) / (1 + r * gl)
        Gb = g
        # upward: from the top half-space (matched) down to layer n's top
        N = len(self.d)
        Zt, ZN = self._Z(self.top_eps, kr, pol), self._Z(self.eps[N - 1], kr, pol)
        g = (Zt - ZN) / (Zt + ZN)
        for l in range(N - 2, n - 1, -1):
            kzl = _kz(self.k(self.eps[l + 1]), kr)
            gl = g * np.exp(-2j * kzl * self.d[l + 1])  # at the bottom of layer l + 1
            Zu, Zl = self._Z(self.eps[l + 1], kr, pol), self._Z(self.eps[l], kr, pol)
            r = (Zu - Zl) / (Zu + Zl)
            g = (r + gl) / (1 + r * gl)
        return Gb, g

    # ---- spectral reflected parts -------------------------------------------------------
    def _brackets(self, n, kr, part, arg, pol, current):
        """Reflected terms of the bracket of V_i (current=False) or I_v (current=True) for the
        Toeplitz part (arg = u = z - z') or the Hankel part (arg = v = z + z')."""
        kz = _kz(self.k(self.eps[n]), kr)
        Gb, Gt = self.gammas(n, kr, pol)
        d, zb, zt = self.d[n], self.z[n], self.z[n + 1]
        D = 1.0 - Gb * Gt * np.exp(-2j * kz * d)
        if part == "T":
            u = arg
            return Gb * Gt * (np.exp(-1j * kz * (2 * d + u)) + np.exp(-1j * kz * (2 * d - u))) / D, kz
        v = arg
        s = -1.0 if current else 1.0
        return s * (Gb * np.exp(-1j * kz * (v - 2 * zb)) + Gt * np.exp(-1j * kz * (2 * zt - v))) / D, kz

    def spectral(self, n, kr, part, arg, kind):
        """Reflected part of the spectral Green's function `kind` ('xx', 'zz', 'phi')."""
        kr = np.asarray(kr, dtype=complex)
        if kind == "xx":
            r, kz = self._brackets(n, kr, part, arg, "h", False)
            return r / (2j * kz)
        if kind == "zz":
            r, kz = self._brackets(n, kr, part, arg, "e", True)
            return r / (2j * kz)
        if kind == "phi":
            re_, kz = self._brackets(n, kr, part, arg, "e", False)
            rh, _ = self._brackets(n, kr, part, arg, "h", False)
            kn2 = self.k(self.eps[n]) ** 2
            return (1j / (2 * kr ** 2 * kz)) * (kz ** 2 * re_ - kn2 * rh)
        raise ValueError(kind)

    # ---- Sommerfeld integral ------------------------------------------------------------
    def _kmax(self):
        ks = [abs(self.k(e).real) for e in list(self.eps) + [self.top_eps] +
              ([] if self.ground else [self.bottom_eps])]
        return max(ks)

    def path(self, rmax, zeta):
        """Nodes and weights of the integration path for rho <= rmax and a decay e^{-k zeta}:
        a half-ellipse k(t) = a/2 (1 - cos t) + j b sin t (t in [0, pi], 64 panels of 16 points,
        a = twice the largest wavenumber, b <= 1/rmax keeps |J0| below e), then the real axis
        from a in panels no longer than a quarter period of J0, a fifth of the decay length or a
        fifth of the distance from the origin, up to where e^{-k zeta} < 1e-18."""
        if zeta <= 0:
            raise ValueError("the reflected terms need zeta > 0")
        a = 2.0 * self._kmax()
        b = min(a / 2.0, 1.0 / rmax) if rmax > 0 else a / 2.0
        edges = np.linspace(0.0, math.pi, 65)
        t = (0.5 * (edges[1:] - edges[:-1])[:, None] * _GL_X[None, :] +
             0.5 * (edges[1:] + edges[:-1])[:, None]).ravel()
        wt = (0.5 * (edges[1:] - edges[:-1])[:, None] * _GL_W[None, :]).ravel()
        k1 = 0.5 * a * (1 - np.cos(t)) + 1j * b * np.sin(t)
        w1 = (0.5 * a * np.sin(t) + 1j * b * np.cos(t)) * wt
        kend = a + 42.0 / zeta
        step_cap = min(0.25 * math.pi / rmax if rmax > 0 else np.inf, 0.2 / zeta)
        lo = a
        los, his = [], []
        while lo < kend:
            h = min(step_cap, 0.2 * lo)
            los.append(lo)
            his.append(min(lo + h, kend))
            lo = his[-1]
        los, his = np.array(los), np.array(his)
        k2 = (0.5 * (his - los)[:, None] * _GL_X[None, :] + 0.5 * (his + los)[:, None]).ravel()
        w2 = (0.5 * (his - los)[:, None] * _GL_W[None, :]).ravel()
        return np.concatenate([k1, k2.astype(complex)]), np.concatenate([w1, w2.astype(complex)])

    def sommerfeld(self, f, rho, zeta):
        """(1/2 pi) int_0^inf f(k) J0(k rho) k dk for a spectral function f decaying at least as
        e^{-k zeta} (zeta > 0) along the real axis; rho a scalar or an array (one path for all,
        set by the largest rho)."""
        rho = np.atleast_1d(np.asarray(rho, dtype=float))
        k, w = self.path(float(rho.max()), zeta)
        fk = f(k) * k * w
        out = np.array([np.sum(fk * jv(0, k * r)) for r in rho]) / (2.0 * math.pi)
        return out if out.size > 1 else out[0]

    def sommerfeld_many(self, fs, rho, zeta):
        """The same for several spectral functions on one path (zeta: the smallest decay among
        them): [len(fs), len(rho)]."""
        rho = np.atleast_1d(np.asarray(rho, dtype=float))
        k, w = self.path(float(rho.max()), zeta)
        J = jv(0, k[:, None] * rho[None, :]) * (k * w)[:, None] / (2.0 * math.pi)
        return np.stack([f(k) @ J for f in fs])

    # ---- spatial Green's functions --------------------------------------------------------
    def toeplitz(self, n, rho, u, kind):
        """G_T(rho, u): the direct term (closed form; 0 at R = 0, the grid's convention) plus the
        doubly reflected terms. rho a scalar or an array."""
        d = self.d[n]
        if abs(u) >= d:
            raise ValueError("|z - z'| must be below the layer thickness")
        R = np.hypot(rho, u)
        with np.errstate(divide="ignore", invalid="ignore"):
            direct = np.where(R > 0, green(self.k(self.eps[n]), R), 0.0)
        refl = self.sommerfeld(lambda kr: self.spectral(n, kr, "T", u, kind), rho, 2 * d - abs(u))
        return direct + refl

    def hankel(self, n, rho, v, kind):
        """G_H(rho, v), v = z + z': the singly reflected terms. rho a scalar or an array."""
        zb, zt = self.z[n], self.z[n + 1]
        zeta = min(v - 2 * zb, 2 * zt - v)
        return self.sommerfeld(lambda kr: self.spectral(n, kr, "H", v, kind), rho, zeta)

    def mgf(self, rho, z, zp, kind):
        """G(rho, z, z') for z, z' inside the same layer."""
        n = self.layer_of(z)
        if self.layer_of(zp) != n:
            raise ValueError("source and observer must lie in the same layer")
        return self.toeplitz(n, rho, z - zp, kind) + self.hankel(n, rho, z + zp, kind)


class LayeredGrid:
    """The AIM grid step H inside layer n of a stack: phi(a) = sum_b G(a, b) sigma(b) over the
    nodes of a uniform grid (x fastest, nodes strictly inside the layer) with G one of the
    stack's Green's functions, as a Toeplitz part (the three-level Toeplitz table
    T[dz, dy, dx] = G_T(rho, dz h_z), zero-padded FFT convolution, as in free space) plus a
    Hankel part in z (table H[s, dy, dx] = G_H(rho, 2 z_0 + s h_z), s = k_a + k_b: a convolution of
    the z-reversed sources). The tables are Sommerfeld integrals over the distinct rho."""

    def __init__(self, stack: Stack, kind, origin, h, n):
        self.stack, self.kind = stack, kind
        self.origin = np.asarray(origin, dtype=float)
        self.h = np.asarray(h, dtype=float)
        self.n = tuple(int(v) for v in n)
        nx, ny, nz = self.n
        z0, zl = self.origin[2], self.origin[2] + (nz - 1) * self.h[2]
        self.layer = stack.layer_of(z0)
        if stack.layer_of(zl) != self.layer:
            raise ValueError("the grid must lie inside one layer")
        dx, dy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")   # [ny, nx]
        rho = np.hypot(dx * self.h[0], dy * self.h[1])
        ur, inv = np.unique(np.round(rho, 12), return_inverse=True)
        inv = inv.reshape(rho.shape)
        n_, hz = self.layer, self.h[2]
        d, zb, zt = stack.d[n_], stack.z[n_], stack.z[n_ + 1]
        dzs = np.arange(-(nz - 1), nz)
        # reflected parts on one integration path per part (the smallest decay among the rows)
        Tr = stack.sommerfeld_many([lambda kr, u=dz * hz: stack.spectral(n_, kr, "T", u, kind)
                                    for dz in dzs], ur, 2 * d - (nz - 1) * hz)
        vs = 2 * z0 + np.arange(2 * nz - 1) * hz
        Hr = stack.sommerfeld_many([lambda kr, v=v: stack.spectral(n_, kr, "H", v, kind)
                                    for v in vs], ur, min(vs[0] - 2 * zb, 2 * zt - vs[-1]))
        R = np.hypot(ur[None, :], dzs[:, None] * hz)
        with np.errstate(divide="ignore", invalid="ignore"):
            direct = np.where(R > 0, green(stack.k(stack.eps[n_]), R), 0.0)
        self.T = (direct + Tr)[:, inv]          # [2nz-1, ny, nx], dz = -(nz-1) .. nz-1
        self.H = Hr[:, inv]                     # [2nz-1, ny, nx], s = 0 .. 2nz-2

    def kernel(self, ia, ib):
        """G between nodes ia, ib (index triples (x, y, z))."""
        dx, dy = abs(ia[0] - ib[0]), abs(ia[1] - ib[1])
        nz = self.n[2]
        return self.T[ia[2] - ib[2] + nz - 1, dy, dx] + self.H[ia[2] + ib[2], dy, dx]

    def apply_direct(self, sigma):
        """sum_b G(a, b) sigma(b) by direct summation (small grids)."""
        nx, ny, nz = self.n
        s = np.asarray(sigma).reshape(nz, ny, nx)
        out = np.zeros_like(s, dtype=complex)
        idx = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
        for a in idx:
            out[a[2], a[1], a[0]] = sum(self.kernel(a, b) * s[b[2], b[1], b[0]] for b in idx)
        return out.ravel()

    def apply(self, sigma):
        """The same by FFT: the Toeplitz part as a zero-padded convolution in x, y and z; the
        Hankel part as a convolution in x and y and, in z, of the reversed sources (index
        k' = nz - 1 - k_b, so k_a + k_b = k_a - k' + nz - 1)."""
        nx, ny, nz = self.n
        s = np.asarray(sigma, dtype=complex).reshape(nz, ny, nx)
        shape = (2 * nz, 2 * ny, 2 * nx)

        def full_xy(tab):  # [m, ny, nx] over |dx|, |dy| -> [m, 2ny-1, 2nx-1] over signed offsets
            t = np.concatenate([tab[:, :0:-1, :], tab], axis=1)
            return np.concatenate([t[:, :, :0:-1], t], axis=2)

        def conv(kern, src, zoff):
            # kern[m, j, i] at offsets (m - zoff, j - (ny - 1), i - (nx - 1))
            K = np.zeros(shape, dtype=complex)
            m = np.arange(kern.shape[0]) - zoff
            j = np.arange(-(ny - 1), ny)
            i = np.arange(-(nx - 1), nx)
            K[np.ix_(m % shape[0], j % shape[1], i % shape[2])] = kern
            return np.fft.ifftn(np.fft.fftn(K) * np.fft.fftn(src, s=shape, axes=(0, 1, 2)))[:nz, :ny, :nx]

        out = conv(full_xy(self.T), s, nz - 1)
        out += conv(full_xy(self.H), s[::-1], nz - 1)
        return out.ravel()


# ---------------------------------------------------------------------------------------
# Galerkin operators and the AIM inside a layer
# ---------------------------------------------------------------------------------------
class ReflectedTable:
    """The reflected (smooth) part of one Green's function of layer n, G_T,refl(rho, u) +
    G_H(rho, v), tabulated on tensor grids of spacing `step` and interpolated by cubic
    splines in each variable (real and imaginary parts apart). Ranges: rho in [0, rho_max],
    u = z - z' in [-du, du], v = z + z' in [v_lo, v_hi]."""

    def __init__(self, stack: Stack, n, kind, rho_max, du, v_lo, v_hi, step):
        from scipy.interpolate import RegularGridInterpolator as RGI
        d = stack.d[n]
        if du >= d or v_lo <= 2 * stack.z[n] or v_hi >= 2 * stack.z[n + 1]:
            raise ValueError("table ranges must stay inside the layer")

        def axis(lo, hi):
            m = max(4, int(math.ceil((hi - lo) / step)) + 1)
            return np.linspace(lo, hi, m)

        self.rho = axis(0.0, rho_max)
        self.u = axis(-du, du)
        self.v = axis(v_lo, v_hi)
        T = stack.sommerfeld_many([lambda kr, u=u: stack.spectral(n, kr, "T", u, kind)
                                   for u in self.u], self.rho, 2 * d - du).T          # [rho, u]
        zeta_h = min(v_lo - 2 * stack.z[n], 2 * stack.z[n + 1] - v_hi)
        H = stack.sommerfeld_many([lambda kr, v=v: stack.spectral(n, kr, "H", v, kind)
                                   for v in self.v], self.rho, zeta_h).T
        self._T = [RGI((self.rho, self.u), T.real, method="cubic"),
                   RGI((self.rho, self.u), T.imag, method="cubic")]
        self._H = [RGI((self.rho, self.v), H.real, method="cubic"),
                   RGI((self.rho, self.v), H.imag, method="cubic")]

    def __call__(self, rho, u, v):
        pu = np.stack([np.ravel(rho), np.ravel(u)], axis=-1)
        pv = np.stack([np.ravel(rho), np.ravel(v)], axis=-1)
        out = self._T[0](pu) + 1j * self._T[1](pu) + self._H[0](pv) + 1j * self._H[1](pv)
        return out.reshape(np.shape(rho))


def reflected_parts(rw, tables):
    """Reflected parts of L^A (RWG x RWG; G^A_xx on the x and y components, G^A_zz on z) and
    L^Phi (triangle x triangle), Radon's 7-point rule on both triangles; `tables` maps 'xx',
    'zz', 'phi' to callables (rho, u, v) -> value."""
    from .quad import radon7, rule_points
    b, w = radon7()
    X = rw.verts[rw.tris]
    rq = rule_points(X, b)                              # [nt, 7, 3]
    wq = rw.area[:, None] * w[None, :]
    nt, ne = rw.nt, rw.ne
    p = rq.reshape(-1, 3)
    rho = np.hypot(p[:, None, 0] - p[None, :, 0], p[:, None, 1] - p[None, :, 1])
    u = p[:, None, 2] - p[None, :, 2]
    v = p[:, None, 2] + p[None, :, 2]
    G = {k: tables[k](rho, u, v).reshape(nt, 7, nt, 7) for k in ("xx", "zz", "phi")}
    LP = np.einsum("tq,tqsp,sp->ts", wq, G["phi"], wq)
    LA = np.zeros((ne, ne), dtype=np.complex128)
    for i in range(3):
        mi = rw.t_edges[:, i]
        ci = rw.t_esign[:, i] * rw.elen[mi] / (2.0 * rw.area)
        fi = ci[:, None, None] * (rq - rw.verts[rw.t_evert[:, i]][:, None, :]) * wq[:, :, None]
        for j in range(3):
            nj = rw.t_edges[:, j]
            cj = rw.t_esign[:, j] * rw.elen[nj] / (2.0 * rw.area)
            fj = cj[:, None, None] * (rq - rw.verts[rw.t_evert[:, j]][:, None, :]) * wq[:, :, None]
            vals = (np.einsum("tqd,spd,tqsp->ts", fi[..., :2], fj[..., :2], G["xx"]) +
                    np.einsum("tq,sp,tqsp->ts", fi[..., 2], fj[..., 2], G["zz"]))
            np.add.at(LA, (mi[:, None], nj[None, :]), vals)
    return LA, LP


def dense_layered_operators(rw, stack: Stack, step=None):
    """Dense L^A and L^Phi of objects inside one layer of the stack: the direct term (the
    free-space operators at the layer's wavenumber, singular rules included) plus the
    reflected parts."""
    from .operators import dense_lphi, dense_rwg
    z = rw.verts[:, 2]
    n = stack.layer_of(float(z.min()))
    if stack.layer_of(float(z.max())) != n:
        raise ValueError("the objects must lie inside one layer")
    lo, hi = float(z.min()), float(z.max())
    span = np.ptp(rw.verts[:, :2], axis=0)
    rho_max = float(np.hypot(*span)) * 1.001 + 1e-9
    zeta = min(2 * lo - 2 * stack.z[n], 2 * stack.z[n + 1] - 2 * hi)
    step = step or zeta / 32.0
    tabs = {k: ReflectedTable(stack, n, k, rho_max, (hi - lo) * 1.001 + 1e-9, 2 * lo - 1e-9,
                              2 * hi + 1e-9, step) for k in ("xx", "zz", "phi")}
    k = stack.k(stack.eps[n])
    LAr, LPr = reflected_parts(rw, tabs)
    return dense_rwg(rw, k, "A") + LAr, dense_lphi(rw, k) + LPr


class LayeredAim:
    """The AIM external operators inside one layer: the projection and interpolation of
    oracle/aim.py, the grid step of LayeredGrid per component (G^A_xx for the x and y
    components, G^A_zz for z, G^Phi for the charges), and the near region precorrected for
    that grid step: L_NR = L_exact - sum_c P_c^T G_grid,c P_c on the near pairs."""

    KIND = ("xx", "xx", "zz")

    def __init__(self, rw, stack: Stack, origin, h, n, r_near=2):
        from .aim import Aim
        z0 = float(np.asarray(origin)[2])
        self.layer = stack.layer_of(z0)
        k = stack.k(stack.eps[self.layer])
        self.A = Aim(rw, origin, h, n, k, r_near)
        self.grids = {kind: LayeredGrid(stack, kind, origin, h, n) for kind in ("xx", "zz", "phi")}
        self.LNR_A = self.LNR_P = None

    def _grid_pairs(self, grid, W_m, W_n, anc_m, anc_n):
        """sum_{a,b} W_m[a] G_grid(x_a, x_b) W_n[b] per pair, from the grid's tables."""
        from .aim import OFFS
        nz = grid.n[2]
        out = np.zeros(len(anc_m), dtype=np.complex128)
        for c0 in range(0, len(anc_m), 2048):
            sl = slice(c0, c0 + 2048)
            na = anc_m[sl][:, None, :] + OFFS[None, :, :]        # [P, 27, 3] (x, y, z)
            nb = anc_n[sl][:, None, :] + OFFS[None, :, :]
            dx = np.abs(na[:, :, None, 0] - nb[:, None, :, 0])
            dy = np.abs(na[:, :, None, 1] - nb[:, None, :, 1])
            dz = na[:, :, None, 2] - nb[:, None, :, 2]
            sz = na[:, :, None, 2] + nb[:, None, :, 2]
            G = grid.T[dz + nz - 1, dy, dx] + grid.H[sz, dy, dx]
            out[sl] = np.einsum("pa,pab,pb->p", W_m[sl], G, W_n[sl])
        return out

    def build_near(self, LA_exact, LP_exact):
        import scipy.sparse as sps
        A, rw = self.A, self.A.rw
        M, N = A.near_e
        pre = sum(self._grid_pairs(self.grids[self.KIND[c]], A.WA[M, c, :], A.WA[N, c, :],
                                   A.anc_e[M], A.anc_e[N]) for c in range(3))
        self.LNR_A = sps.csr_matrix((LA_exact[M, N] - pre, (M, N)), shape=(rw.ne, rw.ne))
        T, S = A.near_t
        pre = self._grid_pairs(self.grids["phi"], A.WP[T], A.WP[S], A.anc_t[T], A.anc_t[S])
        self.LNR_P = sps.csr_matrix((LP_exact[T, S] - pre, (T, S)), shape=(rw.nt, rw.nt))
        return self

    def far_A(self, j):
        A = self.A
        return sum(A.PA[c] @ self.grids[self.KIND[c]].apply(A.PA[c].T @ j) for c in range(3))

    def far_P(self, q):
        return self.A.PP @ self.grids["phi"].apply(self.A.PP.T @ q)

    def LA(self, j):
        return self.far_A(j) + self.LNR_A @ j

    def LPhi(self, q):
        return self.far_P(q) + self.LNR_P @ q

"""A perfectly conducting ground plane under the background medium: the bottom layer of the
paper's layered stacks (Table I), the first piece of a layered-medium Green's function (the
dielectric layers above the plane are not modelled here). Test infrastructure (oracle), FP64.

Image theory for the plane z = z_g (the Green's function of a PEC half-space): with
r_i = (x, y, 2 z_g - z) the image of r and R_i = |r - r'_i|,
  vector potential   G^A = diag(G(R) - G(R_i), G(R) - G(R_i), G(R) + G(R_i))
                     (a horizontal current images with the opposite sign, a vertical one with
                     the same sign),
  scalar potential   G^Phi = G(R) - G(R_i)  (a charge images with the opposite sign),
so that on the plane, where R = R_i, the tangential vector potential and the scalar potential
vanish, and with them the tangential electric field -j w A - grad Phi.

Galerkin operators: L^A_mn = int int f_m . G^A f_n, L^Phi_ts = int_t int_s G^Phi. The image
parts are regular for objects above the plane and use the 7-point rule on both triangles; the
free-space parts are those of oracle/operators.py.

On the AIM grid the image part of the convolution is a correlation in z (Toeplitz in x and y,
Hankel in z): phi_img(a) = sum_b G_grid(a - b_i) sigma(b) with b_i the image of node b. When the
plane lies on a node plane of the grid, b_i is a node (of the grid extended below the plane),
and the image part is the ordinary convolution of the z-reflected sources.
"""
from __future__ import annotations

import math

import numpy as np

from .aim import green_grid
from .operators import dense_lphi, dense_rwg
from .quad import radon7, rule_points
from .rwg import RWG

D_IMG = np.array([1.0, 1.0, -1.0])  # the image of a current: (-J_x, -J_y, +J_z) = -D J


def image(r, zg):
    """r_i = (x, y, 2 z_g - z)."""
    r = np.array(r, dtype=np.float64, copy=True)
    r[..., 2] = 2.0 * zg - r[..., 2]
    return r


def green(k, R):
    return np.exp(-1j * k * R) / (4.0 * math.pi * R)


def kernels(k, r, rp, zg):
    """(G^A diagonal [..., 3], G^Phi [...]) between points r and r' above the plane."""
    R = np.linalg.norm(np.asarray(r) - np.asarray(rp), axis=-1)
    Ri = np.linalg.norm(np.asarray(r) - image(rp, zg), axis=-1)
    g, gi = green(k, R), green(k, Ri)
    GA = np.stack([g - gi, g - gi, g + gi], axis=-1)
    return GA, g - gi


def _image_parts(rw: RWG, k, zg):
    """Image parts of L^A (RWG x RWG) and L^Phi (triangle x triangle), 7 x 7 points per pair."""
    b, w = radon7()
    X = rw.verts[rw.tris]
    rq = rule_points(X, b)                          # [nt, 7, 3]
    wq = rw.area[:, None] * w[None, :]              # [nt, 7]
    if np.min(rq[..., 2]) <= zg:
        raise ValueError("the objects must lie above the ground plane")
    rqi = image(rq, zg)
    nt, ne = rw.nt, rw.ne
    # G(R_i) for every pair of rule points: [nt, 7, nt, 7]
    d = rq[:, :, None, None, :] - rqi[None, None, :, :, :]
    Gi = green(k, np.linalg.norm(d, axis=-1))
    LP = -np.einsum("tq,tqsp,sp->ts", wq, Gi, wq)
    # RWG: f_n on triangle s = c_n (r - v_n); the image term is -G(R_i) f_m . D f_n
    LA = np.zeros((ne, ne), dtype=np.complex128)
    for i in range(3):
        mi = rw.t_edges[:, i]
        ci = rw.t_esign[:, i] * rw.elen[mi] / (2.0 * rw.area)
        fi = ci[:, None, None] * (rq - rw.verts[rw.t_evert[:, i]][:, None, :])   # [nt, 7, 3]
        for j in range(3):
            nj = rw.t_edges[:, j]
            cj = rw.t_esign[:, j] * rw.elen[nj] / (2.0 * rw.area)
            fj = cj[:, None, None] * (rq - rw.verts[rw.t_evert[:, j]][:, None, :])
            ff = np.einsum("tqd,spd->tqsp", fi * wq[:, :, None], fj * (wq[:, :, None] * D_IMG))
            vals = -np.einsum("tqsp,tqsp->ts", ff, Gi)
            np.add.at(LA, (mi[:, None], nj[None, :]), vals)
    return LA, LP


def dense_ground_operators(rw: RWG, k0, zg):
    """Dense L^A and L^Phi of the background above the ground plane z = zg."""
    LAi, LPi = _image_parts(rw, k0, zg)
    return dense_rwg(rw, k0, "A") + LAi, dense_lphi(rw, k0) + LPi


def grid_image_direct(k0, h, n, origin, zg, sigma, sign):
    """sign * sum_b G_grid(a - b_i) sigma(b) by direct summation (a, b nodes of the grid)."""
    nx, ny, nz = n
    s = np.asarray(sigma).reshape(nz, ny, nx)
    pts = np.stack(np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"),
                   axis=-1).reshape(-1, 3)[:, ::-1].astype(np.float64)    # (x, y, z) indices
    pos = origin + pts * h
    posi = image(pos, zg)
    out = np.zeros(pts.shape[0], dtype=np.complex128)
    sv = s.ravel()
    for a in range(pts.shape[0]):
        R = np.linalg.norm(pos[a] - posi, axis=1)
        out[a] = np.sum(green(k0, R) * sv)
    return sign * out


def grid_image_fft(k0, h, n, origin, zg, sigma, sign):
    """The same image part as a convolution: the sources reflected into the node planes below
    the ground plane (zg must be a node plane, origin_z - m h_z for an integer m >= 0), then
    one zero-padded FFT convolution on the extended grid, read back on the original nodes."""
    nx, ny, nz = n
    m = (origin[2] - zg) / h[2]
    mi = int(round(m))
    if abs(m - mi) > 1e-9 or mi < 0:
        raise ValueError("the ground plane must be a node plane at or below the grid")
    s = np.asarray(sigma).reshape(nz, ny, nx)
    # node z index k sits at z = zg + (mi + k) h; its image at zg - (mi + k) h, i.e. index
    # -(2 mi + k) relative to node 0: extended grid from -(2 mi + nz - 1) to nz - 1
    off = 2 * mi + nz - 1
    Nz = off + nz
    ext = np.zeros((Nz, ny, nx), dtype=np.complex128)
    for k in range(nz):
        ext[off - 2 * mi - k] = s[k]
    # G_grid(a - b) over the extended grid, zero-padded FFT convolution
    shape = (2 * Nz, 2 * ny, 2 * nx)
    dz, dy, dx = np.meshgrid(np.arange(-Nz + 1, Nz), np.arange(-ny + 1, ny),
                             np.arange(-nx + 1, nx), indexing="ij")
    K = green_grid(k0, h, np.stack([dx, dy, dz], axis=-1))
    Kc = np.zeros(shape, dtype=np.complex128)
    Kc[np.ix_(np.arange(-Nz + 1, Nz) % shape[0], np.arange(-ny + 1, ny) % shape[1],
              np.arange(-nx + 1, nx) % shape[2])] = K
    full = np.fft.ifftn(np.fft.fftn(Kc) * np.fft.fftn(ext, s=shape, axes=(0, 1, 2)))
    return sign * full[off:off + nz, :ny, :nx].ravel()


class GroundAim:
    """The AIM external operators above the ground plane (O-AIM with images): the projection
    and interpolation of oracle/aim.py, the grid convolution plus its image part (sign -1 for
    the x and y components and for the charges, +1 for z; grid_image_fft), and the near region
    precorrected for both,
        L_NR = L_exact,ground - sum_c P_c^T (G_grid + s_c G_grid,image) P_c
    on the near pairs (anchors within r_near). zg must be a node plane below the grid."""

    SIGN = (-1.0, -1.0, 1.0)

    def __init__(self, rw: RWG, origin, h, n, k0, zg, r_near=2):
        from .aim import Aim
        self.A = Aim(rw, origin, h, n, k0, r_near)
        self.zg = zg
        self.LNR_A = None
        self.LNR_P = None

    def conv(self, sigma, sign):
        A = self.A
        return A.conv(sigma) + grid_image_fft(A.k0, A.h, A.n, A.origin, self.zg, sigma, sign)

    def image_precorrection(self, W_m, W_n, anc_m, anc_n, sign):
        """sign * sum_{a,b} W_m[a] G(|x_a - image(x_b)|) W_n[b] per pair (x: stencil nodes)."""
        from .aim import OFFS
        A = self.A
        xa = A.origin + (anc_m[:, None, :] + OFFS[None, :, :]) * A.h      # [P, 27, 3]
        xb = image(A.origin + (anc_n[:, None, :] + OFFS[None, :, :]) * A.h, self.zg)
        R = np.linalg.norm(xa[:, :, None, :] - xb[:, None, :, :], axis=-1)
        return sign * np.einsum("pa,pab,pb->p", W_m, green(A.k0, R), W_n)

    def build_near(self, LA_exact, LP_exact):
        """Near-region matrices from dense exact ground-plane operators (small meshes)."""
        import scipy.sparse as sps
        A, rw = self.A, self.A.rw
        M, N = A.near_e
        pre = sum(A.precorrection(A.WA[M, c, :], A.WA[N, c, :], A.anc_e[M], A.anc_e[N])
                  + self.image_precorrection(A.WA[M, c, :], A.WA[N, c, :], A.anc_e[M],
                                             A.anc_e[N], self.SIGN[c]) for c in range(3))
        self.LNR_A = sps.csr_matrix((LA_exact[M, N] - pre, (M, N)), shape=(rw.ne, rw.ne))
        T, S = A.near_t
        pre = A.precorrection(A.WP[T], A.WP[S], A.anc_t[T], A.anc_t[S]) + \
            self.image_precorrection(A.WP[T], A.WP[S], A.anc_t[T], A.anc_t[S], -1.0)
        self.LNR_P = sps.csr_matrix((LP_exact[T, S] - pre, (T, S)), shape=(rw.nt, rw.nt))
        return self

    def far_A(self, j):
        A = self.A
        return sum(A.PA[c] @ self.conv(A.PA[c].T @ j, self.SIGN[c]) for c in range(3))

    def far_P(self, q):
        A = self.A
        return A.PP @ self.conv(A.PP.T @ q, -1.0)

    def LA(self, j):
        return self.far_A(j) + self.LNR_A @ j

    def LPhi(self, q):
        return self.far_P(q) + self.LNR_P @ q

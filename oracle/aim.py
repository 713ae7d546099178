"""Adaptive integral method, written plainly. Test infrastructure (oracle), FP64.

Sec. III-A item 1, Eq. (AIM_L): L^A and L^Phi are applied as L_NR + W H P, where P projects
mesh sources onto a uniform 3-D grid, H convolves grid sources with the Green's function
(by FFT), W = P^T interpolates grid potentials back onto the testing functions, and the sparse
L_NR holds the near-region entries, precorrected so the grid's own near contribution is not
counted twice.

Readings (the paper defers these to Bleszynski 1996 / Phillips 1997):
* anchor of a source = nearest grid node of its centre, floor((c - o)/h + 1/2) per axis; the
  centre of an RWG is the mean of its two triangle centroids, of a pulse its centroid;
* stencil = the 3 x 3 x 3 nodes anchor + {-1, 0, 1}^3 (order 2);
* P[m, node] = int f_m(r) l_node(r) dS, with l_node the tensor-product quadratic Lagrange
  polynomial of the stencil (this matches all moments of degree <= 2 per axis); for pulses
  P_Phi[t, node] = int_t l_node dS. The integrals are exact (degree <= 8 rule);
* grid kernel G_grid(d) = G(k0, |d h|) for d != 0 and G_grid(0) = 0;
* H is the linear (zero-padded) convolution over the grid;
* near region: pairs whose anchors differ by at most R_near = 2 in every axis;
  L_NR[m, n] = L_exact[m, n] - sum_c (P_c^T G_grid P_c)[m, n] there, zero elsewhere.
"""
from __future__ import annotations

import math
from itertools import product

import numpy as np
import scipy.sparse as sp

from .operators import rwg_entries, pulse_entries
from .quad import gauss_tri, rule_points
from .rwg import RWG

OFFS = np.array([(ox, oy, oz) for oz in (-1, 0, 1) for oy in (-1, 0, 1) for ox in (-1, 0, 1)],
                dtype=np.int64)  # stencil node k = (oz+1)*9 + (oy+1)*3 + (ox+1), as (x, y, z)


class GridError(ValueError):
    pass


def lagrange3(u):
    """1-D quadratic Lagrange basis on nodes -1, 0, 1: returns [..., 3]."""
    return np.stack([0.5 * u * (u - 1.0), 1.0 - u * u, 0.5 * u * (u + 1.0)], axis=-1)


def anchors(centres, origin, h):
    return np.floor((centres - origin) / h + 0.5).astype(np.int64)


def green_grid(k0, h, d):
    """G_grid at integer offsets d [..., 3]."""
    R = np.sqrt(np.sum((d * h) ** 2, axis=-1))
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.exp(-1j * k0 * R) / (4.0 * math.pi * R)
    return np.where(R > 0, G, 0.0)


class Aim:
    def __init__(self, rw: RWG, origin, h, n, k0, r_near=2):
        self.rw = rw
        self.origin = np.asarray(origin, dtype=np.float64)
        self.h = np.asarray(h, dtype=np.float64)
        self.n = np.asarray(n, dtype=np.int64)
        self.k0 = k0
        self.r_near = r_near
        self.ng = int(np.prod(self.n))
        ce = 0.5 * (rw.centroid[rw.et[:, 0]] + rw.centroid[rw.et[:, 1]])
        self.anc_e = anchors(ce, self.origin, self.h)
        self.anc_t = anchors(rw.centroid, self.origin, self.h)
        for a in (self.anc_e, self.anc_t):
            if np.any(a < 1) or np.any(a > self.n - 2):
                raise GridError("a stencil falls outside the grid")
        self.WA, self.WP = self._weights()
        self.PA = [self._pmat(self.WA[:, c, :], self.anc_e) for c in range(3)]
        self.PP = self._pmat(self.WP, self.anc_t)
        self.near_e = self._near_pairs(self.anc_e)
        self.near_t = self._near_pairs(self.anc_t)
        self.LNR_A = None
        self.LNR_P = None

    # ---- projection weights -------------------------------------------------------
    def _lag_nodes(self, pts, anc):
        """l_node(r) for the 27 stencil nodes: pts [M, q, 3], anc [M, 3] -> [M, q, 27]."""
        u = (pts - (self.origin + anc * self.h)[:, None, :]) / self.h
        lx, ly, lz = lagrange3(u[..., 0]), lagrange3(u[..., 1]), lagrange3(u[..., 2])
        return (lz[..., :, None, None] * ly[..., None, :, None] * lx[..., None, None, :]).reshape(
            pts.shape[0], pts.shape[1], 27)

    def _weights(self):
        rw = self.rw
        b, w = gauss_tri(5)
        X = rw.verts[rw.tris]
        WA = np.zeros((rw.ne, 3, 27))
        for side, sgn in ((0, 1.0), (1, -1.0)):
            t = rw.et[:, side]
            v = rw.verts[rw.eopp[:, side]]
            pts = rule_points(X[t], b)                               # [ne, q, 3]
            f = sgn * (rw.elen / (2 * rw.area[t]))[:, None, None] * (pts - v[:, None, :])
            lag = self._lag_nodes(pts, self.anc_e)                   # [ne, q, 27]
            WA += np.einsum("q,m,mqc,mqk->mck", w, rw.area[t], f, lag)
        pts = rule_points(X, b)
        lag = self._lag_nodes(pts, self.anc_t)
        WP = np.einsum("q,m,mqk->mk", w, rw.area, lag)
        return WA, WP

    def node_index(self, anc):
        """Global node index of each stencil node: [M, 27]."""
        nd = anc[:, None, :] + OFFS[None, :, :]
        return (nd[..., 2] * self.n[1] + nd[..., 1]) * self.n[0] + nd[..., 0]

    def _pmat(self, W, anc):
        M = W.shape[0]
        cols = self.node_index(anc)
        rows = np.repeat(np.arange(M), 27)
        return sp.csr_matrix((W.ravel(), (rows, cols.ravel())), shape=(M, self.ng))

    # ---- grid convolution -----------------------------------------------------------
    def kernel_array(self):
        """G_grid at offsets (dz, dy, dx) in (-(n-1) .. n-1), as [2nz-1, 2ny-1, 2nx-1]."""
        nx, ny, nz = self.n
        dz, dy, dx = np.meshgrid(np.arange(-nz + 1, nz), np.arange(-ny + 1, ny),
                                 np.arange(-nx + 1, nx), indexing="ij")
        return green_grid(self.k0, self.h, np.stack([dx, dy, dz], axis=-1))

    def conv(self, sigma):
        """phi(a) = sum_b G_grid(a - b) sigma(b), linear convolution via zero-padded FFT."""
        nx, ny, nz = self.n
        s = np.asarray(sigma).reshape(nz, ny, nx)
        K = self.kernel_array()
        shape = (2 * nz, 2 * ny, 2 * nx)
        Kc = np.zeros(shape, dtype=np.complex128)
        # circulant arrangement: offset d stored at index d mod 2n
        iz = np.arange(-nz + 1, nz) % shape[0]
        iy = np.arange(-ny + 1, ny) % shape[1]
        ix = np.arange(-nx + 1, nx) % shape[2]
        Kc[np.ix_(iz, iy, ix)] = K
        out = np.fft.ifftn(np.fft.fftn(Kc) * np.fft.fftn(s, s=shape, axes=(0, 1, 2)))
        return out[:nz, :ny, :nx].ravel()

    def conv_direct(self, sigma):
        """The same convolution by direct summation (small grids)."""
        nx, ny, nz = self.n
        s = np.asarray(sigma).reshape(nz, ny, nx)
        pts = np.stack(np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"),
                       axis=-1).reshape(-1, 3)
        out = np.zeros(pts.shape[0], dtype=np.complex128)
        sv = s.ravel()
        for i, a in enumerate(pts):
            d = (a[None, :] - pts)[:, ::-1]
            out[i] = np.sum(green_grid(self.k0, self.h, d) * sv)
        return out

    # ---- near region ----------------------------------------------------------------
    def _near_pairs(self, anc):
        """All (m, n) with max-norm anchor distance <= r_near (sorted by m, then n)."""
        key = (anc[:, 2] * self.n[1] + anc[:, 1]) * self.n[0] + anc[:, 0]
        order = np.argsort(key, kind="stable")
        skey = key[order]
        M, N = [], []
        R = self.r_near
        for d in product(range(-R, R + 1), repeat=3):
            d = np.array(d)
            tgt = anc + d[None, :]
            ok = np.all((tgt >= 0) & (tgt < self.n[None, :]), axis=1)
            tkey = (tgt[:, 2] * self.n[1] + tgt[:, 1]) * self.n[0] + tgt[:, 0]
            lo = np.searchsorted(skey, tkey, side="left")
            hi = np.searchsorted(skey, tkey, side="right")
            cnt = np.where(ok, hi - lo, 0)
            m = np.repeat(np.arange(anc.shape[0]), cnt)
            starts = np.repeat(lo, cnt)
            within = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
            M.append(m)
            N.append(order[starts + within])
        M = np.concatenate(M)
        N = np.concatenate(N)
        o = np.lexsort((N, M))
        return M[o], N[o]

    def _gloc(self):
        """Gloc[D][ka, kb] = G_grid(D + o_a - o_b) for anchor differences |D|_inf <= R."""
        R = self.r_near
        out = {}
        for D in product(range(-R, R + 1), repeat=3):
            d = np.array(D)[None, None, :] + OFFS[:, None, :] - OFFS[None, :, :]
            out[D] = green_grid(self.k0, self.h, d)
        return out

    def precorrection(self, W_m, W_n, anc_m, anc_n):
        """sum_{a,b} W_m[a] G_grid(anchor_m + o_a - anchor_n - o_b) W_n[b], per pair."""
        gl = self._gloc()
        D = anc_m - anc_n
        out = np.zeros(D.shape[0], dtype=np.complex128)
        keys = [tuple(x) for x in D]
        groups: dict = {}
        for i, kk in enumerate(keys):
            groups.setdefault(kk, []).append(i)
        for kk, idx in groups.items():
            idx = np.array(idx)
            out[idx] = np.einsum("ia,ab,ib->i", W_m[idx], gl[kk], W_n[idx])
        return out

    def build_near(self, LA_exact=None, LP_exact=None, rows_e=None, rows_t=None):
        """Precorrected near-region matrices. Exact entries are computed for the near pairs
        unless dense exact matrices are supplied. rows_e / rows_t, if given, restrict the
        entries to those testing functions (the other rows stay empty): rows of L^A and L^Phi
        sampled one by one on structures too large for every near pair."""
        rw = self.rw
        M, N = self.near_e
        if rows_e is not None:
            keep = np.isin(M, np.asarray(rows_e))
            M, N = M[keep], N[keep]
        la = LA_exact[M, N] if LA_exact is not None else rwg_entries(rw, self.k0, M, N, "A")
        pre = sum(self.precorrection(self.WA[M, c, :], self.WA[N, c, :], self.anc_e[M],
                                     self.anc_e[N]) for c in range(3))
        self.LNR_A = sp.csr_matrix((la - pre, (M, N)), shape=(rw.ne, rw.ne))
        T, S = self.near_t
        if rows_t is not None:
            keep = np.isin(T, np.asarray(rows_t))
            T, S = T[keep], S[keep]
        lp = LP_exact[T, S] if LP_exact is not None else pulse_entries(rw, self.k0, T, S)
        pre = self.precorrection(self.WP[T], self.WP[S], self.anc_t[T], self.anc_t[S])
        self.LNR_P = sp.csr_matrix((lp - pre, (T, S)), shape=(rw.nt, rw.nt))
        return self

    # ---- operators ------------------------------------------------------------------
    # PA[c] and PP hold the weights as [sources, nodes]: the paper's projection P is their
    # transpose (sigma = P x) and the interpolation W = P^T is the matrix itself.
    def far_A(self, j):
        return sum(self.PA[c] @ self.conv(self.PA[c].T @ j) for c in range(3))

    def far_P(self, q):
        return self.PP @ self.conv(self.PP.T @ q)

    def LA(self, j):
        return self.far_A(j) + self.LNR_A @ j

    def LPhi(self, q):
        return self.far_P(q) + self.LNR_P @ q

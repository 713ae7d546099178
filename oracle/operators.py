"""Galerkin matrices and the SLIM system (Sec. II). Test infrastructure (oracle), FP64.

Lengths are in micrometres (ell = 1e-6 m). In these units each row of Eq. (AEFIEoutJ) keeps
its form: row 1 scales by ell^2 and row 2 by 1/ell, so the unknowns [H; c0 rho_Delta] are
unchanged, with k0 -> k0*ell. The internal operators become
  Zhat = Z/eta0    = -(1/(j k0 eps_rc)) L_{k_i}^{-1} (K_{k_i} + I_x/2)     (Eq. MFIEinZin)
  Yhat = Y_eq*eta0 =  (1/(j k0 mu_rl))  L_{k_l}^{-1} (K_{k_l} + I_x/2)     (Eq. EFIEeqYeq)
so that e = E/eta0 = Zhat h and h_eq = Yhat e.

Matrix definitions (background wavenumber k0; object wavenumber k_i with Im k_i < 0):
  L^A_mn   = int int f_m . f_n G(k0)                      (Sec. II-A, Eq. AEFIEsys)
  L^Phi_ts = int_t int_s G(k0)                            (pulse basis)
  D_tn     = +l_n on T+(n), -l_n on T-(n);  F = diag(1/A_t)
  I_x,mn   = int (n x f_m) . f_n                          (rotated-RWG testing)
  L_k,mn   = int int G(k) [f_m . f_n - k^-2 div f_m div' f_n]
  K_k,mn   = int f_m . PV int grad_r G(k) x f_n
The charge block D^T L^Phi_m B of Eq. (AEFIEsys) is read as -(F D)^T L^Phi (B = I): testing
grad Phi with f_m and integrating by parts gives -(1/eps0)(F D)^T L^Phi rho, and
c0 = 1/(eps0 eta0). The continuity row is F D J + j k0 (c0 rho) = 0.
G(k, R) = exp(-j k R) / (4 pi R), time convention exp(j w t).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import highk
from .quad import NEAR_FACTOR, radon7, subdivide4, rule_points, static_potentials
from .rwg import RWG

C0 = 299792458.0
MU0 = 4e-7 * math.pi
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0
ELL = 1e-6


def k0_of(freq):
    """Free-space wavenumber in 1/um."""
    return 2.0 * math.pi * freq / C0 * ELL


def eps_rc(sigma, freq, eps_r=1.0):
    """Complex relative permittivity eps_r - j sigma/(w eps0) (exp(j w t))."""
    return eps_r - 1j * sigma / (2.0 * math.pi * freq * EPS0)


def k_medium(k0, epsc, mur=1.0):
    """Wavenumber k0 sqrt(eps mu) on the branch Im k <= 0."""
    k = k0 * np.sqrt(complex(epsc) * mur)
    if k.imag > 0:
        k = -k
    return k


# -------------------------------------------------------------------------------------
# triangle-pair integrals
# -------------------------------------------------------------------------------------
_FOUR_PI = 4.0 * math.pi


def _kernels(k, R):
    """G, its regular part g = G - 1/(4 pi R), and gd = G'(R)/R + 1/(4 pi R^3)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.exp(-1j * k * R)
        G = e / (_FOUR_PI * R)
        g = np.where(R > 0, (e - 1.0) / (_FOUR_PI * R), -1j * k / _FOUR_PI)
        gp = -(1.0 + 1j * k * R) * e / (_FOUR_PI * R ** 3)           # G'(R)/R
        gd = np.where(R > 0, (1.0 - (1.0 + 1j * k * R) * e) / (_FOUR_PI * R ** 3), 0.0)
    return G, g, gp, gd


def tri_pair_moments(rw: RWG, k, T, S, want_K=True, chunk=4096):
    """Moments of G(k) over triangle pairs (t = T[i] testing, s = S[i] source).

    M0  = int_t int_s G            M1  = int_t int_s r G        M1p = int_t int_s r' G
    M2  = int_t int_s r . r' G
    Vs  = int_t V(r)               U   = int_t V(r) x r,  with V(r) = int_s grad_r G dS'
    Positions r and r' are measured from the centroid of t (the RWG combination in rwg_entries
    is translation invariant), so that the moments of a pair far from the coordinate origin do
    not cancel against each other there.
    """
    T = np.asarray(T, dtype=np.int64)
    S = np.asarray(S, dtype=np.int64)
    npair = T.size
    out = {key: np.zeros(npair, dtype=np.complex128) for key in ("M0", "M2")}
    for key in ("M1", "M1p", "Vs", "U"):
        out[key] = np.zeros((npair, 3), dtype=np.complex128)
    bo, wo = radon7()
    bn, wn = subdivide4(radon7())
    X = rw.verts[rw.tris]  # [nt, 3, 3]
    o = rw.centroid[T]     # per-pair origin
    dc = rw.centroid[T] - rw.centroid[S]
    dmax = np.maximum(rw.diam[T], rw.diam[S])
    near = np.einsum("ij,ij->i", dc, dc) < (NEAR_FACTOR * dmax) ** 2
    # near pairs at large |k| (Sec. II-B, high conductivity): the edge-integral scheme of
    # oracle/highk.py, or the regular rule beyond the decay range
    hk = near & (abs(k) * dmax > highk.HIGHK)
    if np.any(hk):
        if complex(k).imag != 0.0:
            sep = np.zeros(T.size, dtype=bool)
            for i in np.nonzero(hk)[0]:
                sep[i] = highk.separated(X[T[i]], X[S[i]], rw.normal[S[i]], k)
            near &= ~(hk & sep)
            hk &= ~sep
        ih = np.nonzero(hk)[0]
        if ih.size:
            oo = o[ih][:, None, :]
            m = highk.pair_moments_batch(X[T[ih]] - oo, X[S[ih]] - oo, rw.normal[S[ih]],
                                         rw.diam[S[ih]], k, want_K)
            for key, v in m.items():
                out[key][ih] = v
    for sel_near in (False, True):
        idx_all = np.nonzero((near == sel_near) & ~hk)[0]
        bi, wi = (bn, wn) if sel_near else (bo, wo)
        bp_, wp_ = bo, wo
        nqo = wp_.size
        for c0 in range(0, idx_all.size, chunk):
            idx = idx_all[c0:c0 + chunk]
            t, s = T[idx], S[idx]
            oo = o[idx][:, None, :]
            Xt, Xs = X[t] - oo, X[s] - oo
            rp = rule_points(Xt, bp_)                           # [nc, nqo, 3]
            wp = wp_[None, :] * rw.area[t][:, None]             # [nc, nqo]
            rq = rule_points(Xs, bi)                            # [nc, nq, 3]
            wq = wi[None, :] * rw.area[s][:, None]              # [nc, nq]
            Rv = rp[:, :, None, :] - rq[:, None, :, :]          # [nc, nqo, nq, 3]
            R = np.sqrt(np.einsum("abcd,abcd->abc", Rv, Rv))
            G, g, gp, gd = _kernels(k, R)
            if not sel_near:
                S0 = np.einsum("aq,apq->ap", wq, G)
                S1 = np.einsum("aq,aqd,apq->apd", wq, rq, G)
                V = np.einsum("aq,apqd,apq->apd", wq, Rv, gp) if want_K else None
            else:
                nc = idx.size
                rr = rp.reshape(-1, 3)
                trs = np.repeat(Xs, nqo, axis=0)
                nrs = np.repeat(rw.normal[s], nqo, axis=0)
                I0, Irho, gI = static_potentials(rr, trs, nrs)
                d = np.einsum("md,md->m", rr - trs[:, 0], nrs)
                rho = rr - d[:, None] * nrs
                I0 = I0.reshape(nc, nqo)
                S0 = I0 / _FOUR_PI + np.einsum("aq,apq->ap", wq, g)
                S1 = ((Irho + rho * I0.reshape(-1)[:, None]) / _FOUR_PI).reshape(nc, nqo, 3) + \
                    np.einsum("aq,aqd,apq->apd", wq, rq, g)
                if want_K:
                    V = (gI / _FOUR_PI).reshape(nc, nqo, 3) + np.einsum("aq,apqd,apq->apd", wq, Rv, gd)
                else:
                    V = None
            out["M0"][idx] = np.einsum("ap,ap->a", wp, S0)
            out["M1"][idx] = np.einsum("ap,apd,ap->ad", wp, rp, S0)
            out["M1p"][idx] = np.einsum("ap,apd->ad", wp, S1)
            out["M2"][idx] = np.einsum("ap,apd,apd->a", wp, rp, S1)
            if want_K:
                out["Vs"][idx] = np.einsum("ap,apd->ad", wp, V)
                out["U"][idx] = np.einsum("ap,apd->ad", wp, np.cross(V, rp))
    return out


def _half_rwg(rw: RWG, n, t):
    """(sign, opposite vertex position) of RWG n on triangle t (vectorized)."""
    plus = rw.et[n, 0] == t
    sgn = np.where(plus, 1.0, -1.0)
    vopp = np.where(plus[:, None], rw.verts[rw.eopp[n, 0]], rw.verts[rw.eopp[n, 1]])
    return sgn, vopp


def rwg_entries(rw: RWG, k, M, N, kind):
    """Entries (M[i], N[i]) of an RWG Galerkin matrix with wavenumber k.

    kind "A": int int f_m . f_n G
         "L": int int G [f_m . f_n - k^-2 div f_m div f_n]
         "K": int f_m . PV int grad G x f_n
    A tuple of kinds returns a tuple of entry arrays from one pass over the triangle pairs.
    """
    kinds = (kind,) if isinstance(kind, str) else tuple(kind)
    M = np.asarray(M, dtype=np.int64)
    N = np.asarray(N, dtype=np.int64)
    nt = rw.nt
    # the four triangle pairs of each RWG pair
    tt = np.stack([rw.et[M, 0], rw.et[M, 0], rw.et[M, 1], rw.et[M, 1]], axis=1)
    ss = np.stack([rw.et[N, 0], rw.et[N, 1], rw.et[N, 0], rw.et[N, 1]], axis=1)
    key = (tt * nt + ss).ravel()
    ukey, inv = np.unique(key, return_inverse=True)
    mom = tri_pair_moments(rw, k, ukey // nt, ukey % nt, want_K=("K" in kinds))
    inv = inv.reshape(-1, 4)
    MM = np.repeat(M, 4)
    NN = np.repeat(N, 4)
    t = tt.ravel()
    s = ss.ravel()
    sm, va = _half_rwg(rw, MM, t)
    sn, vb = _half_rwg(rw, NN, s)
    va = va - rw.centroid[t]  # positions from the testing triangle's centroid, as the moments
    vb = vb - rw.centroid[t]
    cf = sm * sn * rw.elen[MM] * rw.elen[NN] / (4.0 * rw.area[t] * rw.area[s])
    ii = inv.ravel()
    res = []
    for kd in kinds:
        out = np.zeros(M.size, dtype=np.complex128)
        if kd in ("A", "L"):
            M0 = mom["M0"][ii]
            val = mom["M2"][ii] - np.einsum("id,id->i", mom["M1"][ii], vb) \
                - np.einsum("id,id->i", va, mom["M1p"][ii]) + np.einsum("id,id->i", va, vb) * M0
            val = cf * val
            if kd == "L":
                dv = sm * sn * rw.elen[MM] * rw.elen[NN] / (rw.area[t] * rw.area[s])
                val = val - dv * M0 / (k * k)
        elif kd == "K":
            U = mom["U"][ii]
            Vs = mom["Vs"][ii]
            val = cf * (np.einsum("id,id->i", U, vb) - np.einsum("id,id->i", U, va)
                        + np.einsum("id,id->i", Vs, np.cross(vb, va)))
        else:
            raise ValueError(kd)
        np.add.at(out, np.repeat(np.arange(M.size), 4), val)
        res.append(out)
    return res[0] if isinstance(kind, str) else tuple(res)


def dense_rwg(rw: RWG, k, kind, e0=0, e1=None):
    """Dense RWG Galerkin matrix over the edge range [e0, e1) (a tuple of kinds gives a tuple
    of matrices from one pass over the triangle pairs)."""
    e1 = rw.ne if e1 is None else e1
    idx = np.arange(e0, e1)
    Mi, Ni = np.meshgrid(idx, idx, indexing="ij")
    out = rwg_entries(rw, k, Mi.ravel(), Ni.ravel(), kind)
    if isinstance(kind, str):
        return out.reshape(e1 - e0, e1 - e0)
    return tuple(o.reshape(e1 - e0, e1 - e0) for o in out)


def pulse_entries(rw: RWG, k, T, S):
    """L^Phi_ts = int_t int_s G(k) for the given triangle pairs."""
    return tri_pair_moments(rw, k, T, S, want_K=False)["M0"]


def dense_lphi(rw: RWG, k):
    idx = np.arange(rw.nt)
    Ti, Si = np.meshgrid(idx, idx, indexing="ij")
    return pulse_entries(rw, k, Ti.ravel(), Si.ravel()).reshape(rw.nt, rw.nt)


# -------------------------------------------------------------------------------------
# sparse operators
# -------------------------------------------------------------------------------------
def ix_matrix(rw: RWG) -> sp.csr_matrix:
    """I_x,mn = int (n x f_m) . f_n: nonzero only for edges sharing a triangle (exact rule)."""
    b, w = radon7()
    rows, cols, vals = [], [], []
    X = rw.verts[rw.tris]
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            n_i = rw.t_edges[:, i]
            n_j = rw.t_edges[:, j]
            va = rw.verts[rw.t_evert[:, i]]
            vb = rw.verts[rw.t_evert[:, j]]
            rq = rule_points(X, b)  # [nt, 7, 3]
            cr = np.cross(rq - va[:, None, :], rq - vb[:, None, :])
            integ = rw.area * np.einsum("q,tqd,td->t", w, cr, rw.normal)
            cf = rw.t_esign[:, i] * rw.t_esign[:, j] * rw.elen[n_i] * rw.elen[n_j] / (4 * rw.area ** 2)
            rows.append(n_i)
            cols.append(n_j)
            vals.append(cf * integ)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(rw.ne, rw.ne))


def fd_matrix(rw: RWG) -> sp.csr_matrix:
    """F D with D_tn = +-l_n and F = diag(1/A_t) (discrete surface divergence)."""
    rows = np.repeat(np.arange(rw.nt), 3)
    cols = rw.t_edges.ravel()
    vals = (rw.t_esign * rw.elen[rw.t_edges] / rw.area[:, None]).ravel()
    return sp.csr_matrix((vals, (rows, cols)), shape=(rw.nt, rw.ne))


def gram_matrix(rw: RWG) -> sp.csr_matrix:
    """<f_m, f_n> (exact rule), for L2 projections in the tests."""
    b, w = radon7()
    rows, cols, vals = [], [], []
    X = rw.verts[rw.tris]
    rq = rule_points(X, b)
    for i in range(3):
        for j in range(3):
            va = rw.verts[rw.t_evert[:, i]]
            vb = rw.verts[rw.t_evert[:, j]]
            integ = rw.area * np.einsum("q,tqd,tqd->t", w, rq - va[:, None], rq - vb[:, None])
            cf = rw.t_esign[:, i] * rw.t_esign[:, j] * rw.elen[rw.t_edges[:, i]] * \
                rw.elen[rw.t_edges[:, j]] / (4 * rw.area ** 2)
            rows.append(rw.t_edges[:, i])
            cols.append(rw.t_edges[:, j])
            vals.append(cf * integ)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(rw.ne, rw.ne))


def project_tangential(rw: RWG, field_fn):
    """<f_m, F(r)> for a vector field F evaluated at the 7 rule points of every triangle."""
    b, w = radon7()
    X = rw.verts[rw.tris]
    rq = rule_points(X, b)                              # [nt, 7, 3]
    Fv = field_fn(rq.reshape(-1, 3)).reshape(rw.nt, 7, 3)
    out = np.zeros(rw.ne, dtype=np.complex128)
    for i in range(3):
        v = rw.verts[rw.t_evert[:, i]]
        cf = rw.t_esign[:, i] * rw.elen[rw.t_edges[:, i]] / (2 * rw.area)
        val = cf * rw.area * np.einsum("q,tqd,tqd->t", w, rq - v[:, None], Fv)
        np.add.at(out, rw.t_edges[:, i], val)
    return out


def plane_wave_rhs(rw: RWG, k0, pol=(1.0, 0.0, 0.0), khat=(0.0, 0.0, 1.0)):
    """<f_m, E_inc> for E_inc = pol exp(-j k0 khat . r) (unit amplitude, Sec. II eq. AEFIEsys)."""
    pol = np.asarray(pol, dtype=np.float64)
    khat = np.asarray(khat, dtype=np.float64)
    return project_tangential(rw, lambda r: pol[None, :] * np.exp(-1j * k0 * (r @ khat))[:, None])


# -------------------------------------------------------------------------------------
# internal problem (Sec. II-B) and the system (Sec. II-C)
# -------------------------------------------------------------------------------------
def internal_blocks(rw: RWG, freq, sigma, ix=None, objects=None):
    """Per-object Zhat_i and Yhat_i (dense), background vacuum (mu_rl = 1). With `objects`,
    only those objects' blocks are formed (None in the other places)."""
    k0 = k0_of(freq)
    ix = ix_matrix(rw) if ix is None else ix
    Zs, Ys = [], []
    for i, (e0, e1) in enumerate(rw.obj_edge_ranges()):
        if objects is not None and i not in objects:
            Zs.append(None)
            Ys.append(None)
            continue
        ixi = ix[e0:e1, e0:e1].toarray()
        epsc = eps_rc(sigma[i], freq)
        ki = k_medium(k0, epsc)
        Li, Ki = dense_rwg(rw, ki, ("L", "K"), e0, e1)
        Zs.append(-np.linalg.solve(Li, Ki + 0.5 * ixi) / (1j * k0 * epsc))
        Ll, Kl = dense_rwg(rw, k0, ("L", "K"), e0, e1)
        Ys.append(np.linalg.solve(Ll, Kl + 0.5 * ixi) / (1j * k0))
    return Zs, Ys


def block_apply(blocks, ranges, x):
    """y = blockdiag(blocks) x over the given index ranges."""
    y = np.zeros_like(x, dtype=np.complex128)
    for B, (a, b) in zip(blocks, ranges):
        y[a:b] = B @ x[a:b]
    return y


class SlimSystem:
    """The SLIM system of Eq. (AEFIEoutJ), applied as a sequence (never assembled).

    x = [h; q] with h the n x H coefficients (N_E) and q = c0 rho_Delta (N_T):
      e   = Zhat h,  h_eq = Yhat e,  j = h - h_eq                     (Eqs. Jdeltadis, EFIEeqYZ)
      y1  = j k0 L^A j + I_x e - (F D)^T L^Phi q                     (row 1 with C of Eq. Cdef)
      y2  = F D j + j k0 q                                           (row 2)
    LA and LPhi are callables (dense exact or AIM).
    """

    def __init__(self, rw: RWG, freq, Zs, Ys, LA, LPhi, ix=None, fd=None):
        self.rw = rw
        self.freq = freq
        self.k0 = k0_of(freq)
        self.Zs, self.Ys = Zs, Ys
        self.ranges = rw.obj_edge_ranges()
        self.LA, self.LPhi = LA, LPhi
        self.ix = ix_matrix(rw) if ix is None else ix
        self.fd = fd_matrix(rw) if fd is None else fd

    @property
    def n(self):
        return self.rw.ne + self.rw.nt

    def parts(self, x):
        ne = self.rw.ne
        h, q = x[:ne], x[ne:]
        e = block_apply(self.Zs, self.ranges, h)
        heq = block_apply(self.Ys, self.ranges, e)
        j = h - heq
        return h, q, e, heq, j

    def matvec(self, x):
        x = np.asarray(x, dtype=np.complex128)
        h, q, e, heq, j = self.parts(x)
        y1 = 1j * self.k0 * self.LA(j) + self.ix @ e - self.fd.T @ self.LPhi(q)
        y2 = self.fd @ j + 1j * self.k0 * q
        return np.concatenate([y1, y2])

    def dense(self):
        n = self.n
        return np.stack([self.matvec(np.eye(n, dtype=np.complex128)[:, i]) for i in range(n)], axis=1)


def dense_system(rw: RWG, freq, sigma):
    """O-dense: the exact Galerkin SLIM system with dense L^A, L^Phi."""
    k0 = k0_of(freq)
    LA = dense_rwg(rw, k0, "A")
    LP = dense_lphi(rw, k0)
    Zs, Ys = internal_blocks(rw, freq, sigma)
    return SlimSystem(rw, freq, Zs, Ys, lambda v: LA @ v, lambda v: LP @ v), LA, LP

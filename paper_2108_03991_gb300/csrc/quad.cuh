// FP64 integrals of the Galerkin entries over triangle pairs (device code).
//
// The paper leaves the integration rules to the literature (Sec. II-A "numeric integration";
// Sec. II-B "specialized integration routines are needed when conductivity is high"). The
// library's rules:
//  * testing (outer) integrals: Radon's 7-point degree-5 rule;
//  * source (inner) integrals of well-separated pairs: the same rule;
//  * near pairs (|c_t - c_s|^2 < (2.1 max(diam_t, diam_s))^2): the 1/R parts of G and of grad G
//    in closed form (potential integrals of a flat triangle, obtained with the surface
//    divergence theorem; Wilton et al. 1984, Graglia 1993), plus the 7-point rule on the four
//    midpoint sub-triangles for the bounded remainder.
// G(k, R) = exp(-j k R)/(4 pi R) with complex k (Im k <= 0) for lossy media.
#pragma once

#include "common.cuh"

namespace bem {

constexpr double kPi = 3.14159265358979323846;
constexpr double kNearFactor = 2.1;

// rule tables, filled once per process from host computations (setup.cu, the only translation
// unit that includes this header)
// c_r7[i] = (l1, l2, l3, w) of the 7-point rule; c_r28 likewise for the subdivided rule;
// c_gl[i] = (l1, l2, l3, w) of the 5 x 5 collapsed Gauss rule (exact to degree 8)
__constant__ double c_r7[7 * 4];
__constant__ double c_r28[28 * 4];
__constant__ double c_gl[25 * 4];

struct Tri {
  double v[3][3];
  double n[3];
  double area;
  double diam;
  double c[3];
};

__device__ __forceinline__ void d_sub(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
__device__ __forceinline__ double d_dot(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void d_cross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ inline void load_tri(const double* verts, const int32_t* tris, const double* nrm,
                                const double* area, const double* diam, const double* cen, int t,
                                Tri* T) {
  for (int k = 0; k < 3; ++k) {
    int v = tris[3 * t + k];
    for (int a = 0; a < 3; ++a) T->v[k][a] = verts[3 * v + a];
  }
  for (int a = 0; a < 3; ++a) { T->n[a] = nrm[3 * t + a]; T->c[a] = cen[3 * t + a]; }
  T->area = area[t];
  T->diam = diam[t];
}

// Translate a pair so that T's centroid is the origin: the pair moments below are then measured
// from it (the RWG combinations are translation invariant), which keeps the moments of pairs far
// from the coordinate origin from cancelling against each other in the combination.
__device__ __forceinline__ void shift_pair(Tri* T, Tri* S) {
  const double o[3] = {T->c[0], T->c[1], T->c[2]};
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) {
      T->v[k][a] -= o[a];
      S->v[k][a] -= o[a];
    }
  for (int a = 0; a < 3; ++a) {
    T->c[a] -= o[a];
    S->c[a] -= o[a];
  }
}

__device__ __forceinline__ void rule_point(const Tri& T, const double* rule, int q, double* r) {
  const double l1 = rule[4 * q], l2 = rule[4 * q + 1], l3 = rule[4 * q + 2];
  for (int a = 0; a < 3; ++a) r[a] = l1 * T.v[0][a] + l2 * T.v[1][a] + l3 * T.v[2][a];
}

// Closed-form integrals over the flat triangle S for the observation point r:
//   I0 = int 1/R,  Irho = int (rho' - rho)/R,  gI = grad_r int 1/R = -int (r - r')/R^3
// (the normal, solid-angle part of gI is dropped on the triangle's own plane: principal value).
__device__ inline void static_potentials(const double* r, const Tri& S, double* I0, double* Irho,
                                         double* gI) {
  double t0[3];
  d_sub(r, S.v[0], t0);
  double d = d_dot(t0, S.n);
  double rho[3] = {r[0] - d * S.n[0], r[1] - d * S.n[1], r[2] - d * S.n[2]};
  double ad = fabs(d);
  double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
  if (ad <= 1e-10 * S.diam) { ad = 0.0; sg = 0.0; }
  double i0 = 0.0, om = 0.0;
  double ir[3] = {0, 0, 0}, g[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    const double* pa = S.v[i];
    const double* pb = S.v[(i + 1) % 3];
    double lv[3];
    d_sub(pb, pa, lv);
    double ll = sqrt(d_dot(lv, lv));
    double lh[3] = {lv[0] / ll, lv[1] / ll, lv[2] / ll};
    double uh[3];
    d_cross(lh, S.n, uh);
    double wp[3], wm[3];
    d_sub(pb, rho, wp);
    d_sub(pa, rho, wm);
    double lp = d_dot(wp, lh), lm = d_dot(wm, lh);
    double P0 = d_dot(wm, uh);
    double R0sq = P0 * P0 + ad * ad;
    double Rp = sqrt(lp * lp + R0sq), Rm = sqrt(lm * lm + R0sq);
    double f;
    if (lp + lm >= 0.0) f = log((Rp + lp) / (Rm + lm));
    else f = log((Rm - lm) / (Rp - lp));
    if (P0 == 0.0 && !isfinite(f)) f = 0.0;
    double dp = R0sq + ad * Rp, dm = R0sq + ad * Rm;
    double bp = dp > 0 ? atan(P0 * lp / dp) : 0.0;
    double bm = dm > 0 ? atan(P0 * lm / dm) : 0.0;
    i0 += P0 * f;
    om += bp - bm;
    double cf = 0.5 * (R0sq * f + lp * Rp - lm * Rm);
    for (int a = 0; a < 3; ++a) { ir[a] += cf * uh[a]; g[a] -= f * uh[a]; }
  }
  i0 -= ad * om;
  for (int a = 0; a < 3; ++a) g[a] -= sg * om * S.n[a];
  *I0 = i0;
  for (int a = 0; a < 3; ++a) { Irho[a] = ir[a]; gI[a] = g[a]; }
}

// exp(-j k R) for complex k = (kr, ki)
__device__ __forceinline__ double2 expjk(double kr, double ki, double R) {
  double s, c;
  sincos(kr * R, &s, &c);
  double m = exp(ki * R);
  return make_double2(m * c, -m * s);
}

// Moments of G(k) over the pair (t testing, s source):
//  L-type: M0 = int int G, M1 = int int r G, M1p = int int r' G, M2 = int int r . r' G
//  K-type: Vs = int_t V(r), U = int_t V(r) x r with V(r) = int_s grad_r G dS'
struct Moments {
  double2 M0, M2;
  double2 M1[3], M1p[3];
  double2 U[3], Vs[3];
};

__device__ inline void pair_moments(const Tri& T, const Tri& S, double kr, double ki, bool wantL,
                                    bool wantK, bool only_M0, Moments* out, int force = -1) {
  const double inv4pi = 1.0 / (4.0 * kPi);
  double dc[3];
  d_sub(T.c, S.c, dc);
  double dm = fmax(T.diam, S.diam);
  bool near = force >= 0 ? force == 1 : d_dot(dc, dc) < (kNearFactor * dm) * (kNearFactor * dm);
  const double* ri = near ? c_r28 : c_r7;
  const int nqi = near ? 28 : 7;
  double2 M0 = {0, 0}, M2 = {0, 0};
  double2 M1[3] = {{0, 0}, {0, 0}, {0, 0}}, M1p[3] = {{0, 0}, {0, 0}, {0, 0}};
  double2 U[3] = {{0, 0}, {0, 0}, {0, 0}}, Vs[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int p = 0; p < 7; ++p) {
    double r[3];
    rule_point(T, c_r7, p, r);
    const double wp = c_r7[4 * p + 3] * T.area;
    double2 S0 = {0, 0};
    double2 S1[3] = {{0, 0}, {0, 0}, {0, 0}};
    double2 V[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int q = 0; q < nqi; ++q) {
      double rq[3];
      rule_point(S, ri, q, rq);
      const double wq = ri[4 * q + 3] * S.area;
      double Rv[3];
      d_sub(r, rq, Rv);
      double R = sqrt(d_dot(Rv, Rv));
      double2 e = expjk(kr, ki, R);
      double2 gs;   // G (far) or the regular part g = G - 1/(4 pi R) (near)
      double2 gv;   // G'(R)/R (far) or gd = G'(R)/R + 1/(4 pi R^3) (near)
      if (!near) {
        double iR = 1.0 / R;
        gs = make_double2(e.x * iR * inv4pi, e.y * iR * inv4pi);
        if (wantK) {
          // -(1 + j k R) e / (4 pi R^3),  1 + j k R = (1 - ki R) + j kr R
          double ax = 1.0 - ki * R, ay = kr * R;
          double iR3 = iR * iR * iR * inv4pi;
          gv = make_double2(-(ax * e.x - ay * e.y) * iR3, -(ax * e.y + ay * e.x) * iR3);
        }
      } else {
        if (R > 0) {
          double iR = 1.0 / R;
          gs = make_double2((e.x - 1.0) * iR * inv4pi, e.y * iR * inv4pi);
          if (wantK) {
            double ax = 1.0 - ki * R, ay = kr * R;
            double iR3 = iR * iR * iR * inv4pi;
            gv = make_double2((1.0 - (ax * e.x - ay * e.y)) * iR3, -(ax * e.y + ay * e.x) * iR3);
          }
        } else {
          gs = make_double2(ki * inv4pi, -kr * inv4pi);  // limit -j k / (4 pi)
          gv = make_double2(0.0, 0.0);
        }
      }
      S0.x += wq * gs.x; S0.y += wq * gs.y;
      if (!only_M0) {
        for (int a = 0; a < 3; ++a) { S1[a].x += wq * rq[a] * gs.x; S1[a].y += wq * rq[a] * gs.y; }
        if (wantK)
          for (int a = 0; a < 3; ++a) { V[a].x += wq * Rv[a] * gv.x; V[a].y += wq * Rv[a] * gv.y; }
      }
    }
    if (near) {
      double I0, Irho[3], gI[3];
      static_potentials(r, S, &I0, Irho, gI);
      double t0[3];
      d_sub(r, S.v[0], t0);
      double d = d_dot(t0, S.n);
      S0.x += I0 * inv4pi;
      if (!only_M0) {
        for (int a = 0; a < 3; ++a) {
          double rho = r[a] - d * S.n[a];
          S1[a].x += (Irho[a] + rho * I0) * inv4pi;
        }
        if (wantK)
          for (int a = 0; a < 3; ++a) V[a].x += gI[a] * inv4pi;
      }
    }
    M0.x += wp * S0.x; M0.y += wp * S0.y;
    if (!only_M0) {
      if (wantL) {
        for (int a = 0; a < 3; ++a) {
          M1[a].x += wp * r[a] * S0.x; M1[a].y += wp * r[a] * S0.y;
          M1p[a].x += wp * S1[a].x; M1p[a].y += wp * S1[a].y;
          M2.x += wp * r[a] * S1[a].x; M2.y += wp * r[a] * S1[a].y;
        }
      }
      if (wantK) {
        // V x r
        double2 vx[3];
        vx[0] = make_double2(V[1].x * r[2] - V[2].x * r[1], V[1].y * r[2] - V[2].y * r[1]);
        vx[1] = make_double2(V[2].x * r[0] - V[0].x * r[2], V[2].y * r[0] - V[0].y * r[2]);
        vx[2] = make_double2(V[0].x * r[1] - V[1].x * r[0], V[0].y * r[1] - V[1].y * r[0]);
        for (int a = 0; a < 3; ++a) {
          Vs[a].x += wp * V[a].x; Vs[a].y += wp * V[a].y;
          U[a].x += wp * vx[a].x; U[a].y += wp * vx[a].y;
        }
      }
    }
  }
  out->M0 = M0;
  out->M2 = M2;
  for (int a = 0; a < 3; ++a) { out->M1[a] = M1[a]; out->M1p[a] = M1p[a]; out->U[a] = U[a]; out->Vs[a] = Vs[a]; }
}

// ---------------------------------------------------------------------------------------
// Near pairs at large |k| (Sec. II-B: specialised integration for highly conducting objects).
// Inside a good conductor G(k_i, R) decays over a skin depth far below the element size, so the
// static-part subtraction above stops working (G is negligible where 1/R is not). The library's
// reading, for pairs that are near and have |k| max(diam_t, diam_s) > kHighK:
//  * inner integrals at an observation point r over the source triangle S by the fan of S about
//    the projection rho of r on S's plane (height d, a = |d|): along each edge e (signed distance
//    P_e of rho to the edge line, outward in-plane normal u_e, foot parameters l-, l+,
//    R(t) = sqrt(P_e^2 + t^2 + a^2)) the radial integrals are closed forms, leaving
//      int_S G         = [Omega e^{-jka} - sum_e J1_e] / (4 pi j k)
//      int_S (r'-rho)G = -sum_e u_e J2_e / (4 pi j k)
//      int_S grad_r G  = -[sum_e u_e J3_e + n (sgn(d) Omega e^{-jka} - d sum_e J4_e)] / (4 pi)
//    J1 = int P e^{-jkR}/(P^2+t^2), J2 = int e^{-jkR}, J3 = int e^{-jkR}/R,
//    J4 = int P e^{-jkR}/((P^2+t^2) R) over [l-, l+]; Omega the plane angle S subtends at rho;
//    each J by 6-point Gauss-Legendre on a graded partition of |t| (the integrands are even):
//    breakpoints h0 2^j (h0 = min(|P|, 1/|k|)/2; w instead of |P| when P = 0) up to the first
//    above 2 dmax, then steps dmax = kDmaxFactor/|k|, cut where |Im k| (R - w) > kDecay; edges
//    with |Im k| (w - a) > kDecay skipped (w = sqrt(P^2 + a^2));
//  * outer integral: T split into four midpoint children, recursively, where a sub-triangle's
//    centroid c is closer to the set where the inner integrals vary fast (the edges of S when T
//    lies in S's plane, S itself otherwise) than its circumradius rad plus kSplitMargin times its
//    diameter and, for a lossy medium, |Im k| (dist - rad) < kSplitDecay, down to depth
//    min(kDepthMax, ceil(log2(|k| diam_T))); Radon's 7 points per leaf;
//  * near pairs whose testing triangle lies wholly beyond kDecay/|Im k| of the source (T's
//    centroid distance to S minus its circumradius) take the regular 7 x 7 rule.
// The set-up evaluates one outer rule point per thread (k_hk_points in setup.cu).
constexpr double kHighK = 0.5;
constexpr double kDecay = 18.0;
constexpr double kPZero = 1e-12;
constexpr double kSplitMargin = 0.25;
constexpr double kSplitDecay = 12.0;
constexpr double kDmaxFactor = 6.0;
constexpr int kDepthMax = 3;

// Gauss-Legendre on [0, 1] with kNgl points: c_glx[i] = node, c_glx[kNgl + i] = weight
constexpr int kNgl = 6;
__constant__ double c_glx[2 * kNgl];

struct EdgeJ {
  double2 J1, J2, J3, J4;
};

// J1..J4 over the |t| range [sa, sb] (the part below `cut`), graded breakpoints of the reading
__device__ inline void hk_piece(double P, double w2, double kr, double ki, double sa, double sb,
                                double h0, double dmax, double cut, bool wantK, EdgeJ* J) {
  const double se = fmin(sb, cut);
  if (!(se > sa)) return;
  double lo = sa;
  auto seg = [&](double hi) {
    const double L = hi - lo;
    if (L > 0) {
      for (int q = 0; q < kNgl; ++q) {
        const double t = lo + L * c_glx[q];
        const double wt = L * c_glx[kNgl + q];
        const double R = sqrt(w2 + t * t);
        double sn, cs;
        sincos(kr * R, &sn, &cs);
        const double m = exp(ki * R) * wt;
        const double ex = m * cs, ey = -m * sn;  // wt e^{-jkR}
        const double lor = P / (P * P + t * t);
        J->J1.x += lor * ex; J->J1.y += lor * ey;
        J->J2.x += ex; J->J2.y += ey;
        if (wantK) {
          const double iR = 1.0 / R;
          J->J3.x += ex * iR; J->J3.y += ey * iR;
          J->J4.x += lor * ex * iR; J->J4.y += lor * ey * iR;
        }
      }
    }
    lo = hi;
  };
  if (!(h0 > 0.0) || !(dmax > 0.0)) return;
  double g = h0, last = 0.0;
  bool done = false;
  for (int it = 0; it < 2200 && g <= 2.0 * dmax; ++it) {  // doubling points (bounded)
    last = g;
    if (g > lo) {
      if (g >= se) { seg(se); done = true; break; }
      seg(g);
    }
    g *= 2.0;
  }
  if (!done) {
    for (int i = 1; i < (1 << 20); ++i) {  // uniform steps after the last doubling point
      const double gi = __dadd_rn(last, __dmul_rn(dmax, (double)i));
      if (gi > lo) {
        if (gi >= se) { seg(se); break; }
        seg(gi);
      }
    }
  }
}

// inner integrals of the reading at r over S: S0 = int G, S1 = int r' G, V = int grad_r G
__device__ inline void hk_inner(const double* r, const Tri& S, double kr, double ki, bool wantK,
                                double2* S0, double2* S1, double2* V) {
  const double kabs = sqrt(kr * kr + ki * ki);
  const double kim = fabs(ki);
  const double x = 1.0 / kabs;
  const double dmax = kDmaxFactor * x;
  double t0[3];
  d_sub(r, S.v[0], t0);
  const double d = d_dot(t0, S.n);
  double a = fabs(d), sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
  if (a <= 1e-10 * S.diam) { a = 0.0; sg = 0.0; }
  const double rho[3] = {r[0] - d * S.n[0], r[1] - d * S.n[1], r[2] - d * S.n[2]};
  double Om = 0.0;
  double2 SJ1 = {0, 0}, SJ4 = {0, 0};
  double2 SJ2[3] = {{0, 0}, {0, 0}, {0, 0}}, SJ3[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int i = 0; i < 3; ++i) {
    const double* pa = S.v[i];
    const double* pb = S.v[(i + 1) % 3];
    double le[3];
    d_sub(pb, pa, le);
    const double ll = sqrt(d_dot(le, le));
    const double lh[3] = {le[0] / ll, le[1] / ll, le[2] / ll};
    double uh[3];
    d_cross(lh, S.n, uh);
    double wa[3], wb[3];
    d_sub(pa, rho, wa);
    d_sub(pb, rho, wb);
    double P = d_dot(wa, uh);
    const double lm = d_dot(wa, lh), lp = d_dot(wb, lh);
    const bool pz = fabs(P) <= kPZero * S.diam;
    if (pz) P = 0.0;
    const double w = fmax(sqrt(P * P + a * a), kPZero * S.diam);
    if (!pz) Om += atan(lp / P) - atan(lm / P);
    if (kim > 0 && kim * (w - a) > kDecay) continue;
    const double h0 = 0.5 * fmin(pz ? w : fabs(P), x);
    const double cut = kim > 0 ? sqrt(kDecay / kim * (2.0 * w + kDecay / kim)) : INFINITY;
    EdgeJ J = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    const double w2 = P * P + a * a;
    if (lm < 0 && lp > 0) {
      hk_piece(P, w2, kr, ki, 0.0, -lm, h0, dmax, cut, wantK, &J);
      hk_piece(P, w2, kr, ki, 0.0, lp, h0, dmax, cut, wantK, &J);
    } else {
      hk_piece(P, w2, kr, ki, fmin(fabs(lm), fabs(lp)), fmax(fabs(lm), fabs(lp)), h0, dmax, cut,
               wantK, &J);
    }
    SJ1.x += J.J1.x; SJ1.y += J.J1.y;
    SJ4.x += J.J4.x; SJ4.y += J.J4.y;
    for (int c = 0; c < 3; ++c) {
      SJ2[c].x += J.J2.x * uh[c]; SJ2[c].y += J.J2.y * uh[c];
      SJ3[c].x += J.J3.x * uh[c]; SJ3[c].y += J.J3.y * uh[c];
    }
  }
  // e^{-jka}
  double sn, cs;
  sincos(kr * a, &sn, &cs);
  const double m = exp(ki * a);
  const double2 ea = make_double2(m * cs, -m * sn);
  const double f4 = 4.0 * kPi;
  // 1/(4 pi j k) = -j / (4 pi k)
  const double2 ik = make_double2(kr / (kr * kr + ki * ki), -ki / (kr * kr + ki * ki));  // 1/k
  const double2 c4jk = make_double2(ik.y / f4, -ik.x / f4);                            // -j/(4 pi k)
  const double2 num = make_double2(Om * ea.x - SJ1.x, Om * ea.y - SJ1.y);
  *S0 = cmul(num, c4jk);
  for (int c = 0; c < 3; ++c) {
    const double2 t = cmul(SJ2[c], c4jk);
    S1[c] = make_double2(rho[c] * S0->x - t.x, rho[c] * S0->y - t.y);
  }
  if (wantK) {
    const double2 nn = make_double2(sg * Om * ea.x - d * SJ4.x, sg * Om * ea.y - d * SJ4.y);
    for (int c = 0; c < 3; ++c)
      V[c] = make_double2(-(SJ3[c].x + S.n[c] * nn.x) / f4, -(SJ3[c].y + S.n[c] * nn.y) / f4);
  }
}

__device__ inline double seg_dist(const double* c, const double* p, const double* q) {
  double v[3], cp[3];
  d_sub(q, p, v);
  d_sub(c, p, cp);
  double t = d_dot(cp, v) / d_dot(v, v);
  t = fmin(fmax(t, 0.0), 1.0);
  const double e[3] = {c[0] - (p[0] + t * v[0]), c[1] - (p[1] + t * v[1]), c[2] - (p[2] + t * v[2])};
  return sqrt(d_dot(e, e));
}

__device__ inline double tri_dist(const double* c, const Tri& S) {
  double t0[3];
  d_sub(c, S.v[0], t0);
  const double d = d_dot(t0, S.n);
  const double rho[3] = {c[0] - d * S.n[0], c[1] - d * S.n[1], c[2] - d * S.n[2]};
  bool inside = true;
  for (int i = 0; i < 3; ++i) {
    double e[3], q[3], x[3];
    d_sub(S.v[(i + 1) % 3], S.v[i], e);
    d_sub(rho, S.v[i], q);
    d_cross(e, q, x);
    if (d_dot(x, S.n) < 0) inside = false;
  }
  if (inside) return fabs(d);
  double m = seg_dist(c, S.v[0], S.v[1]);
  m = fmin(m, seg_dist(c, S.v[1], S.v[2]));
  return fmin(m, seg_dist(c, S.v[2], S.v[0]));
}

struct Sub {
  double v[3][3];
};

__device__ inline void sub_child(const Sub& t, int ch, Sub* o) {
  double m01[3], m12[3], m20[3];
  for (int a = 0; a < 3; ++a) {
    m01[a] = 0.5 * (t.v[0][a] + t.v[1][a]);
    m12[a] = 0.5 * (t.v[1][a] + t.v[2][a]);
    m20[a] = 0.5 * (t.v[2][a] + t.v[0][a]);
  }
  const double* src[4][3] = {{t.v[0], m01, m20}, {m01, t.v[1], m12}, {m20, m12, t.v[2]},
                             {m01, m12, m20}};
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) o->v[k][a] = src[ch][k][a];
}

__device__ inline double sub_diam(const Sub& t) {
  double e0[3], e1[3], e2[3];
  d_sub(t.v[1], t.v[0], e0);
  d_sub(t.v[2], t.v[1], e1);
  d_sub(t.v[0], t.v[2], e2);
  return fmax(fmax(sqrt(d_dot(e0, e0)), sqrt(d_dot(e1, e1))), sqrt(d_dot(e2, e2)));
}

// does the reading split this sub-triangle (given it is above the depth limit)?
__device__ inline bool hk_split(const Sub& t, const Tri& S, bool coplanar, double kim) {
  const double c[3] = {(t.v[0][0] + t.v[1][0] + t.v[2][0]) / 3.0,
                       (t.v[0][1] + t.v[1][1] + t.v[2][1]) / 3.0,
                       (t.v[0][2] + t.v[1][2] + t.v[2][2]) / 3.0};
  double rad = 0.0;
  for (int j = 0; j < 3; ++j) {
    double e[3];
    d_sub(t.v[j], c, e);
    rad = fmax(rad, sqrt(d_dot(e, e)));
  }
  const double dm = sub_diam(t);
  double dist;
  if (coplanar) {
    dist = seg_dist(c, S.v[0], S.v[1]);
    dist = fmin(dist, seg_dist(c, S.v[1], S.v[2]));
    dist = fmin(dist, seg_dist(c, S.v[2], S.v[0]));
  } else {
    dist = tri_dist(c, S);
  }
  return dist < rad + kSplitMargin * dm && (kim == 0.0 || kim * (dist - rad) < kSplitDecay);
}

__device__ inline int hk_depth(double kabs, double diamT) {
  const double q = kabs * diamT;
  if (!(q > 1.0)) return 0;
  return min(kDepthMax, max(0, (int)ceil(log2(q))));
}

__device__ inline bool hk_coplanar(const Tri& T, const Tri& S) {
  double e1[3], e2[3], nT[3];
  d_sub(T.v[1], T.v[0], e1);
  d_sub(T.v[2], T.v[0], e2);
  d_cross(e1, e2, nT);
  const double nn = sqrt(d_dot(nT, nT));
  const double cT[3] = {(T.v[0][0] + T.v[1][0] + T.v[2][0]) / 3.0,
                        (T.v[0][1] + T.v[1][1] + T.v[2][1]) / 3.0,
                        (T.v[0][2] + T.v[1][2] + T.v[2][2]) / 3.0};
  double q[3];
  d_sub(cT, S.v[0], q);
  return fabs(d_dot(nT, S.n)) / nn >= 1.0 - 1e-12 && fabs(d_dot(q, S.n)) <= 1e-10 * S.diam;
}

// one outer rule point r (weight wp): add its contributions to the 28 moment sums
// (M0, M2, M1[3], M1p[3], Vs[3], U[3] as re, im)
__device__ inline void hk_point(const double* r, double wp, const Tri& S, double kr, double ki,
                                bool wantK, double* acc) {
  double2 S0, S1[3], V[3];
  hk_inner(r, S, kr, ki, wantK, &S0, S1, V);
  acc[0] += wp * S0.x; acc[1] += wp * S0.y;
  for (int a = 0; a < 3; ++a) {
    acc[2] += wp * r[a] * S1[a].x; acc[3] += wp * r[a] * S1[a].y;
    acc[4 + 2 * a] += wp * r[a] * S0.x; acc[5 + 2 * a] += wp * r[a] * S0.y;
    acc[10 + 2 * a] += wp * S1[a].x; acc[11 + 2 * a] += wp * S1[a].y;
  }
  if (wantK) {
    const double2 vx[3] = {
        make_double2(V[1].x * r[2] - V[2].x * r[1], V[1].y * r[2] - V[2].y * r[1]),
        make_double2(V[2].x * r[0] - V[0].x * r[2], V[2].y * r[0] - V[0].y * r[2]),
        make_double2(V[0].x * r[1] - V[1].x * r[0], V[0].y * r[1] - V[1].y * r[0])};
    for (int a = 0; a < 3; ++a) {
      acc[16 + 2 * a] += wp * V[a].x; acc[17 + 2 * a] += wp * V[a].y;
      acc[22 + 2 * a] += wp * vx[a].x; acc[23 + 2 * a] += wp * vx[a].y;
    }
  }
}

// The outer rule points of a large-|k| pair as a flat list: a point is (finest sub-triangle index
// idx below the leaf that owns it, rule point q). hk_leaf walks from T to the leaf containing
// finest index idx and reports whether idx owns it (the first finest index below the leaf).
__device__ inline bool hk_leaf(const Tri& T, const Tri& S, int D, bool cop, double kim, int idx,
                               Sub* leaf) {
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) leaf->v[k][a] = T.v[k][a];
  for (int lev = 0; lev < D; ++lev) {
    if (!hk_split(*leaf, S, cop, kim)) return (idx & ((1 << (2 * (D - lev))) - 1)) == 0;
    Sub ch;
    sub_child(*leaf, (idx >> (2 * (D - 1 - lev))) & 3, &ch);
    *leaf = ch;
  }
  return true;
}

// number of outer rule points of the pair (7 per leaf)
__device__ inline int hk_count_points(const Tri& T, const Tri& S, double kr, double ki) {
  const int D = hk_depth(sqrt(kr * kr + ki * ki), T.diam);
  const bool cop = hk_coplanar(T, S);
  int n = 0;
  Sub leaf;
  for (int idx = 0; idx < (1 << (2 * D)); ++idx)
    if (hk_leaf(T, S, D, cop, fabs(ki), idx, &leaf)) n += 7;
  return n;
}

// classification of a pair for the reading: 0 regular 7 x 7, 1 near (small-|k| subtraction),
// 2 near at large |k| with T subdivided, 3 near at large |k| with T a single leaf
__device__ inline int pair_kind(const Tri& T, const Tri& S, double kr, double ki) {
  double dc[3];
  d_sub(T.c, S.c, dc);
  const double dm = fmax(T.diam, S.diam);
  const bool near = d_dot(dc, dc) < (kNearFactor * dm) * (kNearFactor * dm);
  if (!near) return 0;
  const double kabs = sqrt(kr * kr + ki * ki);
  if (!(kabs * dm > kHighK)) return 1;
  Sub t;
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) t.v[k][a] = T.v[k][a];
  const double c[3] = {(t.v[0][0] + t.v[1][0] + t.v[2][0]) / 3.0,
                       (t.v[0][1] + t.v[1][1] + t.v[2][1]) / 3.0,
                       (t.v[0][2] + t.v[1][2] + t.v[2][2]) / 3.0};
  if (ki != 0.0) {
    double rad = 0;
    for (int j = 0; j < 3; ++j) {
      double e[3];
      d_sub(t.v[j], c, e);
      rad = fmax(rad, sqrt(d_dot(e, e)));
    }
    if (fabs(ki) * (tri_dist(c, S) - rad) > kDecay) return 0;
  }
  if (hk_depth(kabs, T.diam) > 0 && hk_split(t, S, hk_coplanar(T, S), fabs(ki))) return 2;
  return 3;
}

}  // namespace bem

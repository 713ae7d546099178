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
                                    bool wantK, bool only_M0, Moments* out) {
  const double inv4pi = 1.0 / (4.0 * kPi);
  double dc[3];
  d_sub(T.c, S.c, dc);
  double dm = fmax(T.diam, S.diam);
  bool near = d_dot(dc, dc) < (kNearFactor * dm) * (kNearFactor * dm);
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

}  // namespace bem

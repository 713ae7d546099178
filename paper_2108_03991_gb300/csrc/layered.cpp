// Set-up of the AIM grid step inside one layer of a stratified background (the layered media
// of Table I: dielectric layers on a ground plane under air): the Toeplitz and Hankel tables of
// the layer's mixed-potential Green's functions on the grid's node offsets, for the grid step
// phi(a) = sum_b [G_T(rho_ab, z_a - z_b) + G_H(rho_ab, z_a + z_b)] sigma(b).
//
// Transmission-line form of the stratified medium's spectral fields (one line section per
// layer, TE and TM lines). In layer n (bottom z_b, top z_t, d = z_t - z_b) the bracket of the
// voltage due to a unit current source is
//   e^{-j kz |u|} + (G_b e1 + G_t e2 + G_b G_t (e3 + e4)) / D,
// and that of the current due to a unit voltage source has -G_b, -G_t in place of G_b, G_t,
// with u = z - z', e1 = e^{-j kz (z + z' - 2 z_b)}, e2 = e^{-j kz (2 z_t - z - z')},
// e3, e4 = e^{-j kz (2d +- u)}, D = 1 - G_b G_t e^{-2 j kz d}, G_b and G_t the line's reflection
// coefficients downward at z_b and upward at z_t. Kernels (each G(k_n, R) in a homogeneous
// medium): G^A_xx from the TE voltage bracket / (2 j kz), G^A_zz from the TM current bracket /
// (2 j kz), G^Phi from (j / (2 k_rho^2 kz)) (kz^2 v^e - k_n^2 v^h). The direct term is
// G(k_n, R) in closed form (zero at R = 0, the grid's convention); the doubly reflected terms
// (e3, e4) belong to the Toeplitz table, the singly reflected ones (e1, e2) to the Hankel one.
// The reflected terms are Sommerfeld integrals (1/2pi) int f(k) J0(k rho) k dk along a
// half-ellipse in the first quadrant (clear of the top half-space's branch point and of the
// surface-wave poles, on or below the real axis for exp(j w t)) and then the real axis, where
// they decay as e^{-k zeta} (zeta > 0 for nodes strictly inside the layer), in 16-point
// Gauss-Legendre panels; one path and one table of J0 values serve every row of a table.
#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <vector>

#include "common.cuh"

namespace bem {

typedef std::complex<double> cd;
static const cd kJ(0.0, 1.0);

// n-point Gauss-Legendre rule on [-1, 1]: Newton's method on the Legendre polynomial from the
// three-term recurrence, started at the Chebyshev-like guesses cos(pi (i + 3/4) / (n + 1/2))
static void gauss_legendre(int n, std::vector<double>* x, std::vector<double>* w) {
  x->assign(n, 0.0);
  w->assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    (*x)[i] = t;
    (*w)[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// J0 of a complex argument from its integral representation (1/pi) int_0^pi cos(z sin t) dt:
// the integrand is periodic and analytic, so the midpoint rule converges geometrically; real
// arguments use the library's cylindrical Bessel function
static cd bessel_j0(cd z) {
  if (z.imag() == 0.0) return cd(std::cyl_bessel_j(0.0, std::fabs(z.real())), 0.0);
  const int N = 40 + 2 * (int)std::ceil(std::abs(z));
  cd s = 0.0;
  for (int i = 0; i < N; ++i) s += std::cos(z * std::sin(M_PI * (i + 0.5) / N));
  return s / (double)N;
}

struct LayerStack {
  double k0 = 0;
  std::vector<double> d, z;   // thicknesses; interfaces z_0 = 0 .. z_N
  std::vector<cd> eps;
  cd top, bottom;
  bool ground = true;

  cd k(cd e) const {
    cd q = k0 * std::sqrt(e);
    return q.imag() > 0 ? -q : q;
  }
  static cd kz(cd k, cd kr) {
    cd q = std::sqrt(k * k - kr * kr);
    return q.imag() > 0 ? -q : q;
  }
  cd Z(cd e, cd kr, bool tm) const {  // line impedance / eta0
    const cd q = kz(k(e), kr);
    return tm ? q / (k0 * e) : k0 / q;
  }
  int layer_of(double zz) const {
    for (size_t l = 0; l + 1 < z.size(); ++l)
      if (z[l] < zz && zz < z[l + 1]) return (int)l;
    return -1;
  }
  // reflection coefficients of layer n's line: downward at its bottom, upward at its top
  void gammas(int n, cd kr, bool tm, cd* gb, cd* gt) const {
    cd g;
    if (ground) {
      g = -1.0;
    } else {
      const cd zb = Z(bottom, kr, tm), z0 = Z(eps[0], kr, tm);
      g = (zb - z0) / (zb + z0);
    }
    for (int l = 1; l <= n; ++l) {
      const cd gl = g * std::exp(-2.0 * kJ * kz(k(eps[l - 1]), kr) * d[l - 1]);
      const cd za = Z(eps[l - 1], kr, tm), zl = Z(eps[l], kr, tm);
      const cd r = (za - zl) / (za + zl);
      g = (r + gl) / (1.0 + r * gl);
    }
    *gb = g;
    const int N = (int)d.size();
    {
      const cd zt = Z(top, kr, tm), zn = Z(eps[N - 1], kr, tm);
      g = (zt - zn) / (zt + zn);
    }
    for (int l = N - 2; l >= n; --l) {
      const cd gl = g * std::exp(-2.0 * kJ * kz(k(eps[l + 1]), kr) * d[l + 1]);
      const cd zu = Z(eps[l + 1], kr, tm), zl = Z(eps[l], kr, tm);
      const cd r = (zu - zl) / (zu + zl);
      g = (r + gl) / (1.0 + r * gl);
    }
    *gt = g;
  }
  // reflected terms of a bracket: Toeplitz part (hankel = false, arg = u) or Hankel part (arg = v)
  cd bracket(int n, cd kr, bool tm, bool current, bool hankel, double arg, cd* kzn) const {
    const cd q = kz(k(eps[n]), kr);
    *kzn = q;
    cd gb, gt;
    gammas(n, kr, tm, &gb, &gt);
    const double dn = d[n], zb = z[n], zt = z[n + 1];
    const cd D = 1.0 - gb * gt * std::exp(-2.0 * kJ * q * dn);
    if (!hankel)
      return gb * gt * (std::exp(-kJ * q * (2 * dn + arg)) + std::exp(-kJ * q * (2 * dn - arg))) / D;
    const double s = current ? -1.0 : 1.0;
    return s * (gb * std::exp(-kJ * q * (arg - 2 * zb)) + gt * std::exp(-kJ * q * (2 * zt - arg))) / D;
  }
  // reflected spectral function of kind 0 (G^A_xx), 1 (G^A_zz), 2 (G^Phi)
  cd spectral(int n, cd kr, int kind, bool hankel, double arg) const {
    cd q;
    if (kind != 2) {  // the bracket sets q: evaluate it before dividing by q
      const cd b = kind == 0 ? bracket(n, kr, false, false, hankel, arg, &q)
                             : bracket(n, kr, true, true, hankel, arg, &q);
      return b / (2.0 * kJ * q);
    }
    const cd re = bracket(n, kr, true, false, hankel, arg, &q);
    const cd rh = bracket(n, kr, false, false, hankel, arg, &q);
    const cd kn = k(eps[n]);
    return kJ / (2.0 * kr * kr * q) * (q * q * re - kn * kn * rh);
  }
  double kmax() const {
    double m = std::fabs(k(top).real());
    for (const cd& e : eps) m = std::max(m, std::fabs(k(e).real()));
    if (!ground) m = std::max(m, std::fabs(k(bottom).real()));
    return m;
  }
  // integration path for rho <= rmax and decay e^{-k zeta}: nodes and weights (k dk included
  // through the caller)
  void path(double rmax, double zeta, std::vector<cd>* kk, std::vector<cd>* ww) const {
    static std::vector<double> gx, gw;
    if (gx.empty()) gauss_legendre(16, &gx, &gw);
    kk->clear();
    ww->clear();
    const double a = 2.0 * kmax();
    const double b = rmax > 0 ? std::min(a / 2.0, 1.0 / rmax) : a / 2.0;
    for (int p = 0; p < 64; ++p) {  // half-ellipse k(t) = a/2 (1 - cos t) + j b sin t
      const double t0 = M_PI * p / 64, t1 = M_PI * (p + 1) / 64;
      for (int i = 0; i < 16; ++i) {
        const double t = 0.5 * (t1 - t0) * gx[i] + 0.5 * (t1 + t0);
        kk->push_back(cd(0.5 * a * (1 - std::cos(t)), b * std::sin(t)));
        ww->push_back(cd(0.5 * a * std::sin(t), b * std::cos(t)) * (0.5 * (t1 - t0) * gw[i]));
      }
    }
    const double kend = a + 42.0 / zeta;
    const double cap = std::min(rmax > 0 ? 0.25 * M_PI / rmax : 1e300, 0.2 / zeta);
    for (double lo = a; lo < kend;) {
      const double hi = std::min(lo + std::min(cap, 0.2 * lo), kend);
      for (int i = 0; i < 16; ++i) {
        kk->push_back(cd(0.5 * (hi - lo) * gx[i] + 0.5 * (hi + lo), 0.0));
        ww->push_back(cd(0.5 * (hi - lo) * gw[i], 0.0));
      }
      lo = hi;
    }
  }
};

// rows[r][i] = (1/2pi) sum_p f_r(k_p) k_p w_p J0(k_p rho_i), one path for all rows
static void sommerfeld_rows(const LayerStack& st, const std::vector<double>& rho, double zeta,
                            int nrow, const std::function<cd(int, cd)>& f,
                            std::vector<std::vector<cd>>* rows) {
  const double rmax = *std::max_element(rho.begin(), rho.end());
  std::vector<cd> kk, ww;
  st.path(rmax, zeta, &kk, &ww);
  const size_t np = kk.size(), nr = rho.size();
  std::vector<cd> J(np * nr);
  for (size_t p = 0; p < np; ++p)
    for (size_t i = 0; i < nr; ++i) J[p * nr + i] = bessel_j0(kk[p] * rho[i]) * kk[p] * ww[p] / (2.0 * M_PI);
  rows->assign(nrow, std::vector<cd>(nr, 0.0));
  for (int r = 0; r < nrow; ++r) {
    std::vector<cd>& out = (*rows)[r];
    for (size_t p = 0; p < np; ++p) {
      const cd fp = f(r, kk[p]);
      for (size_t i = 0; i < nr; ++i) out[i] += fp * J[p * nr + i];
    }
  }
}

// the stack of the C description, checked
static int make_stack(const bem_stack* s, double freq_hz, const char* who, LayerStack* st) {
  if (!s || s->nlayer < 1 || !s->thickness || !s->eps || !(freq_hz > 0) || !std::isfinite(freq_hz)) {
    set_error("%s: bad arguments", who);
    return BEM_EINVAL;
  }
  st->k0 = k0_of(freq_hz);
  st->z.assign(1, 0.0);
  for (int l = 0; l < s->nlayer; ++l) {
    if (!(s->thickness[l] > 0) || !std::isfinite(s->eps[2 * l]) || !std::isfinite(s->eps[2 * l + 1])) {
      set_error("%s: bad layer %d", who, l);
      return BEM_EINVAL;
    }
    st->d.push_back(s->thickness[l]);
    st->z.push_back(st->z.back() + s->thickness[l]);
    st->eps.push_back(cd(s->eps[2 * l], s->eps[2 * l + 1]));
  }
  st->top = cd(s->top_eps[0], s->top_eps[1]);
  st->bottom = cd(s->bottom_eps[0], s->bottom_eps[1]);
  st->ground = s->ground != 0;
  return BEM_OK;
}

}  // namespace bem

using namespace bem;

extern "C" int bem_layered_grid_tables(const bem_stack* s, double freq_hz, const double* origin,
                                       const double* h, const int32_t* n, int kind, double* T,
                                       double* H) {
  if (!origin || !h || !n || !T || !H || kind < 0 || kind > 2) {
    set_error("bem_layered_grid_tables: bad arguments");
    return BEM_EINVAL;
  }
  LayerStack st;
  BEM_TRY(make_stack(s, freq_hz, "bem_layered_grid_tables", &st));
  const int nx = n[0], ny = n[1], nz = n[2];
  if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny > 65536 || !(h[0] > 0) || !(h[1] > 0) || !(h[2] > 0)) {
    set_error("bem_layered_grid_tables: bad grid (at most 65536 x-y offsets)");
    return BEM_EGRID;
  }
  const double z0 = origin[2], z1 = origin[2] + (nz - 1) * h[2];
  const int layer = st.layer_of(z0);
  if (layer < 0 || st.layer_of(z1) != layer) {
    set_error("bem_layered_grid_tables: the grid's node planes must lie strictly inside one layer");
    return BEM_EGRID;
  }
  std::vector<double> rho((size_t)nx * ny);
  for (int dy = 0; dy < ny; ++dy)
    for (int dx = 0; dx < nx; ++dx) rho[(size_t)dy * nx + dx] = std::hypot(dx * h[0], dy * h[1]);
  const double d = st.d[layer], zb = st.z[layer], zt = st.z[layer + 1];
  const int nrow = 2 * nz - 1;
  std::vector<std::vector<cd>> tr, hr;
  sommerfeld_rows(st, rho, 2 * d - (nz - 1) * h[2], nrow,
                  [&](int r, cd kr) { return st.spectral(layer, kr, kind, false, (r - (nz - 1)) * h[2]); }, &tr);
  const double v0 = 2 * z0, v1 = 2 * z0 + (nrow - 1) * h[2];
  sommerfeld_rows(st, rho, std::min(v0 - 2 * zb, 2 * zt - v1), nrow,
                  [&](int r, cd kr) { return st.spectral(layer, kr, kind, true, v0 + r * h[2]); }, &hr);
  const cd kn = st.k(st.eps[layer]);
  for (int r = 0; r < nrow; ++r) {
    const double u = (r - (nz - 1)) * h[2];
    for (size_t i = 0; i < rho.size(); ++i) {
      const double R = std::hypot(rho[i], u);
      cd t = tr[r][i];
      if (R > 0) t += std::exp(-kJ * kn * R) / (4.0 * M_PI * R);
      const size_t o = (size_t)r * rho.size() + i;
      T[2 * o] = t.real();
      T[2 * o + 1] = t.imag();
      H[2 * o] = hr[r][i].real();
      H[2 * o + 1] = hr[r][i].imag();
    }
  }
  return BEM_OK;
}

extern "C" int bem_layered_kernel_table(const bem_stack* s, double freq_hz, int layer, int kind,
                                        int part, int nrho, const double* rho, int narg,
                                        const double* arg, double* out) {
  if (!rho || !arg || !out || kind < 0 || kind > 2 || part < 0 || part > 1 || nrho < 1 ||
      narg < 1 || (int64_t)nrho * narg > (1 << 26)) {
    set_error("bem_layered_kernel_table: bad arguments");
    return BEM_EINVAL;
  }
  LayerStack st;
  BEM_TRY(make_stack(s, freq_hz, "bem_layered_kernel_table", &st));
  if (layer < 0 || layer >= (int)st.d.size()) {
    set_error("bem_layered_kernel_table: no layer %d", layer);
    return BEM_EINVAL;
  }
  const double d = st.d[layer], zb = st.z[layer], zt = st.z[layer + 1];
  double zeta = 1e300;
  for (int j = 0; j < narg; ++j) {  // the smallest decay among the rows sets the path
    const double a = arg[j];
    const double zj = part == 0 ? 2 * d - std::fabs(a) : std::min(a - 2 * zb, 2 * zt - a);
    const bool inside = part == 0 ? std::fabs(a) < d : zj > 0;
    if (!inside || !std::isfinite(a)) {
      set_error("bem_layered_kernel_table: argument %d outside the layer", j);
      return BEM_EINVAL;
    }
    zeta = std::min(zeta, zj);
  }
  std::vector<double> r(rho, rho + nrho);
  for (double v : r)
    if (!(v >= 0) || !std::isfinite(v)) {
      set_error("bem_layered_kernel_table: negative or non-finite rho");
      return BEM_EINVAL;
    }
  std::vector<std::vector<cd>> rows;
  sommerfeld_rows(st, r, zeta, narg,
                  [&](int j, cd kr) { return st.spectral(layer, kr, kind, part == 1, arg[j]); }, &rows);
  for (int j = 0; j < narg; ++j)
    for (int i = 0; i < nrho; ++i) {
      const size_t o = (size_t)j * nrho + i;
      out[2 * o] = rows[j][i].real();
      out[2 * o + 1] = rows[j][i].imag();
    }
  return BEM_OK;
}

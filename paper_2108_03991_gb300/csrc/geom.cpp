// Host-side set-up front-end: mesh validation, RWG / pulse data, AIM anchors, near-region
// sparsity, and the small sparse tables of the system matvec (I_x, F D).
//
// RWG functions (Sec. II, Rao-Wilton-Glisson): one per edge shared by two triangles; edges are
// ordered by object then by the sorted vertex pair (a < b); T+ is the triangle whose
// counter-clockwise boundary runs a -> b; f_n = +l/(2A+)(r - v+) on T+, -l/(2A-)(r - v-) on T-.
// Pulse functions (Sec. II-A): one per triangle, in input order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "common.cuh"

namespace bem {

static inline void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static inline void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline double norm3(const double* a) { return std::sqrt(dot3(a, a)); }

struct DirEdge {
  int64_t key;  // a * nv + b with a < b
  int32_t t, opp, dir;
};

int build_geometry(aim_ctx* c, const bem_mesh* m, const aim_grid* g) {
  if (!m || !g || !m->xyz || !m->tri || !m->obj_of_tri || !m->mat) {
    set_error("aim_setup: null mesh or grid pointer");
    return BEM_EINVAL;
  }
  if (m->nv < 3 || m->nt < 4 || m->nobj < 1) {
    set_error("aim_setup: empty mesh");
    return BEM_EINVAL;
  }
  if (g->order != 2) {
    set_error("aim_setup: only order-2 (3x3x3) stencils are implemented");
    return BEM_EINVAL;
  }
  if (g->r_near < 1 || g->r_near > 4) {
    set_error("aim_setup: r_near must be 1..4");
    return BEM_EINVAL;
  }
  for (int a = 0; a < 3; ++a) {
    if (!(g->h[a] > 0) || !std::isfinite(g->origin[a]) || g->n[a] < 3 || g->n[a] > 4096) {
      set_error("aim_setup: bad grid along axis %d", a);
      return BEM_EGRID;
    }
  }
  const int nv = m->nv, nt = m->nt;
  c->nv = nv;
  c->nt = nt;
  c->nobj = m->nobj;
  c->verts.assign(m->xyz, m->xyz + 3 * (size_t)nv);
  for (double v : c->verts)
    if (!std::isfinite(v)) {
      set_error("aim_setup: non-finite vertex coordinate");
      return BEM_EINVAL;
    }
  c->tris.assign(m->tri, m->tri + 3 * (size_t)nt);
  c->obj_t.assign(m->obj_of_tri, m->obj_of_tri + nt);
  c->mat.assign(m->mat, m->mat + m->nobj);
  for (int i = 0; i < m->nobj; ++i) {
    const bem_material& q = c->mat[i];
    if (!(q.sigma >= 0) || !(q.eps_r > 0) || !(q.mu_r > 0) || !std::isfinite(q.sigma)) {
      set_error("aim_setup: bad material of object %d", i);
      return BEM_EINVAL;
    }
  }
  for (int t = 0; t < nt; ++t) {
    for (int k = 0; k < 3; ++k)
      if (c->tris[3 * t + k] < 0 || c->tris[3 * t + k] >= nv) {
        set_error("aim_setup: triangle %d has a vertex index out of range", t);
        return BEM_EINVAL;
      }
    int o = c->obj_t[t];
    if (o < 0 || o >= m->nobj || (t > 0 && o < c->obj_t[t - 1])) {
      set_error("aim_setup: objects must be contiguous and non-decreasing in the triangle list");
      return BEM_EINVAL;
    }
  }
  // triangles
  c->area.resize(nt);
  c->normal.resize(3 * (size_t)nt);
  c->centroid.resize(3 * (size_t)nt);
  c->diam.resize(nt);
  for (int t = 0; t < nt; ++t) {
    const double* p0 = &c->verts[3 * c->tris[3 * t]];
    const double* p1 = &c->verts[3 * c->tris[3 * t + 1]];
    const double* p2 = &c->verts[3 * c->tris[3 * t + 2]];
    double u[3], v[3], w[3], cr[3];
    sub3(p1, p0, u);
    sub3(p2, p0, v);
    sub3(p2, p1, w);
    cross3(u, v, cr);
    double dbl = norm3(cr);
    if (!(dbl > 0)) {
      set_error("aim_setup: degenerate triangle %d", t);
      return BEM_EMESH;
    }
    c->area[t] = 0.5 * dbl;
    for (int a = 0; a < 3; ++a) {
      c->normal[3 * t + a] = cr[a] / dbl;
      c->centroid[3 * t + a] = (p0[a] + p1[a] + p2[a]) / 3.0;
    }
    c->diam[t] = std::max(norm3(u), std::max(norm3(v), norm3(w)));
  }
  // directed edges -> RWG functions
  std::vector<DirEdge> de(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k) {
      int a = c->tris[3 * t + k], b = c->tris[3 * t + (k + 1) % 3], opp = c->tris[3 * t + (k + 2) % 3];
      int lo = std::min(a, b), hi = std::max(a, b);
      de[3 * t + k] = DirEdge{(int64_t)lo * nv + hi, t, opp, a < b ? +1 : -1};
    }
  std::sort(de.begin(), de.end(), [](const DirEdge& x, const DirEdge& y) {
    return x.key != y.key ? x.key < y.key : x.dir > y.dir;
  });
  struct E { int32_t obj, a, b, tp, tm, vp, vm; };
  std::vector<E> edges;
  edges.reserve(de.size() / 2);
  for (size_t i = 0; i < de.size();) {
    size_t j = i;
    while (j < de.size() && de[j].key == de[i].key) ++j;
    if (j - i != 2) {
      set_error("aim_setup: edge (%lld,%lld) has %d triangles (open or non-manifold surface)",
                (long long)(de[i].key / nv), (long long)(de[i].key % nv), (int)(j - i));
      return BEM_EMESH;
    }
    const DirEdge& p = de[i];
    const DirEdge& q = de[i + 1];
    if (p.dir != +1 || q.dir != -1) {
      set_error("aim_setup: inconsistent triangle orientation at an edge");
      return BEM_EMESH;
    }
    if (c->obj_t[p.t] != c->obj_t[q.t]) {
      set_error("aim_setup: an edge joins two objects");
      return BEM_EMESH;
    }
    edges.push_back(E{c->obj_t[p.t], (int32_t)(p.key / nv), (int32_t)(p.key % nv), p.t, q.t, p.opp, q.opp});
    i = j;
  }
  std::stable_sort(edges.begin(), edges.end(), [](const E& x, const E& y) {
    if (x.obj != y.obj) return x.obj < y.obj;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
  });
  const int ne = (int)edges.size();
  if (2 * (int64_t)ne != 3 * (int64_t)nt) {
    set_error("aim_setup: 2 N_E != 3 N_T");
    return BEM_EMESH;
  }
  c->ne = ne;
  c->ev.resize(2 * (size_t)ne);
  c->et.resize(2 * (size_t)ne);
  c->eopp.resize(2 * (size_t)ne);
  c->obj_e.resize(ne);
  c->elen.resize(ne);
  c->t_edges.assign(3 * (size_t)nt, -1);
  c->t_esign.assign(3 * (size_t)nt, 0);
  c->t_evert.assign(3 * (size_t)nt, -1);
  std::vector<int> fill(nt, 0);
  for (int n = 0; n < ne; ++n) {
    const E& e = edges[n];
    c->ev[2 * n] = e.a; c->ev[2 * n + 1] = e.b;
    c->et[2 * n] = e.tp; c->et[2 * n + 1] = e.tm;
    c->eopp[2 * n] = e.vp; c->eopp[2 * n + 1] = e.vm;
    c->obj_e[n] = e.obj;
    double d[3];
    sub3(&c->verts[3 * e.b], &c->verts[3 * e.a], d);
    c->elen[n] = norm3(d);
    int ts[2] = {e.tp, e.tm}, vs[2] = {e.vp, e.vm}, sg[2] = {+1, -1};
    for (int s = 0; s < 2; ++s) {
      int t = ts[s], k = fill[t]++;
      c->t_edges[3 * t + k] = n;
      c->t_esign[3 * t + k] = sg[s];
      c->t_evert[3 * t + k] = vs[s];
    }
  }
  // object ranges
  c->e0.assign(c->nobj, 0); c->e1.assign(c->nobj, 0);
  c->t0.assign(c->nobj, 0); c->t1.assign(c->nobj, 0);
  for (int i = 0; i < c->nobj; ++i) { c->e0[i] = c->t0[i] = INT32_MAX; c->e1[i] = c->t1[i] = -1; }
  for (int n = 0; n < ne; ++n) { int o = c->obj_e[n]; c->e0[o] = std::min(c->e0[o], n); c->e1[o] = std::max(c->e1[o], n + 1); }
  for (int t = 0; t < nt; ++t) { int o = c->obj_t[t]; c->t0[o] = std::min(c->t0[o], t); c->t1[o] = std::max(c->t1[o], t + 1); }
  for (int i = 0; i < c->nobj; ++i)
    if (c->e1[i] < 0) {
      set_error("aim_setup: object %d has no triangles", i);
      return BEM_EINVAL;
    }
  // AIM grid and anchors (nearest node of the source centre)
  for (int a = 0; a < 3; ++a) { c->go[a] = g->origin[a]; c->gh[a] = g->h[a]; c->gn[a] = g->n[a]; }
  c->r_near = g->r_near;
  c->ng = (int64_t)c->gn[0] * c->gn[1] * c->gn[2];
  if (c->ng > (int64_t)1 << 31) {
    set_error("aim_setup: grid too large");
    return BEM_EGRID;
  }
  c->anc.resize(3 * (size_t)(ne + nt));
  for (int i = 0; i < ne + nt; ++i) {
    double ctr[3];
    if (i < ne) {
      for (int a = 0; a < 3; ++a)
        ctr[a] = 0.5 * (c->centroid[3 * c->et[2 * i] + a] + c->centroid[3 * c->et[2 * i + 1] + a]);
    } else {
      for (int a = 0; a < 3; ++a) ctr[a] = c->centroid[3 * (i - ne) + a];
    }
    for (int a = 0; a < 3; ++a) {
      int v = (int)std::floor((ctr[a] - c->go[a]) / c->gh[a] + 0.5);
      if (v < 1 || v > c->gn[a] - 2) {
        set_error("aim_setup: the stencil of source %d falls outside the grid (axis %d)", i, a);
        return BEM_EGRID;
      }
      c->anc[3 * (size_t)i + a] = v;
    }
  }
  for (int a = 0; a < 3; ++a) {
    c->gp[a] = smooth_length(2 * c->gn[a] - 1);
    if (!make_fft_plan(c->gp[a], &c->plan[a])) {
      set_error("aim_setup: no FFT plan for length %d", c->gp[a]);
      return BEM_EGRID;
    }
  }
  // near-region sparsity: pairs whose anchors differ by <= r_near in every axis
  // (row, col: the CSR; lst, cl: each row's offset into cl, which holds one column list per
  // anchor node: rows anchored at the same node have the same near columns)
  auto near_csr = [&](int first, int count, std::vector<int64_t>* row, std::vector<int32_t>* col,
                      std::vector<int64_t>* lst, std::vector<int32_t>* cl) {
    std::vector<int64_t> key(count);
    for (int i = 0; i < count; ++i) {
      const int32_t* q = &c->anc[3 * (size_t)(first + i)];
      key[i] = ((int64_t)q[2] * c->gn[1] + q[1]) * c->gn[0] + q[0];
    }
    std::vector<int32_t> ord(count);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return key[x] < key[y]; });
    std::vector<int64_t> sk(count);
    for (int i = 0; i < count; ++i) sk[i] = key[ord[i]];
    row->assign(count + 1, 0);
    col->clear();
    lst->assign(count, 0);
    cl->clear();
    std::unordered_map<int64_t, int64_t> list_of;  // anchor node -> offset of its list in cl
    const int R = c->r_near;
    std::vector<int32_t> buf;
    for (int i = 0; i < count; ++i) {
      const int32_t* q = &c->anc[3 * (size_t)(first + i)];
      buf.clear();
      for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
          for (int dx = -R; dx <= R; ++dx) {
            int x = q[0] + dx, y = q[1] + dy, z = q[2] + dz;
            if (x < 0 || y < 0 || z < 0 || x >= c->gn[0] || y >= c->gn[1] || z >= c->gn[2]) continue;
            int64_t k = ((int64_t)z * c->gn[1] + y) * c->gn[0] + x;
            auto lo = std::lower_bound(sk.begin(), sk.end(), k);
            for (auto it = lo; it != sk.end() && *it == k; ++it) buf.push_back(ord[it - sk.begin()]);
          }
      std::sort(buf.begin(), buf.end());
      col->insert(col->end(), buf.begin(), buf.end());
      (*row)[i + 1] = (int64_t)col->size();
      auto found = list_of.find(key[i]);
      if (found == list_of.end()) {
        found = list_of.emplace(key[i], (int64_t)cl->size()).first;
        cl->insert(cl->end(), buf.begin(), buf.end());
      }
      (*lst)[i] = found->second;
    }
  };
  near_csr(0, ne, &c->rowA, &c->colA, &c->lstA, &c->clA);
  near_csr(ne, nt, &c->rowP, &c->colP, &c->lstP, &c->clP);
  return BEM_OK;
}

// I_x,mn = int (n x f_m) . f_n over the triangles m and n share. On triangle t with
// f_m = s_m l_m/(2A)(r - v_a) and f_n = s_n l_n/(2A)(r - v_b):
// n . ((r - v_a) x (r - v_b)) = n . ((r - v_a) x (v_a - v_b)) is linear in r, so the integral
// is A n . ((c_t - v_a) x (v_a - v_b)) exactly.
void build_ix_fd(const aim_ctx* c, std::vector<int32_t>* ixcol, std::vector<double>* ixval,
                 std::vector<double>* fdE, std::vector<double>* fdT) {
  const int ne = c->ne, nt = c->nt;
  ixcol->assign(4 * (size_t)ne, 0);
  ixval->assign(4 * (size_t)ne, 0.0);
  std::vector<int> fill(ne, 0);
  for (int t = 0; t < nt; ++t) {
    const double* nrm = &c->normal[3 * t];
    const double* ct = &c->centroid[3 * t];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        if (i == j) continue;
        int m = c->t_edges[3 * t + i], n = c->t_edges[3 * t + j];
        const double* va = &c->verts[3 * c->t_evert[3 * t + i]];
        const double* vb = &c->verts[3 * c->t_evert[3 * t + j]];
        double u[3], w[3], cr[3];
        sub3(ct, va, u);
        sub3(va, vb, w);
        cross3(u, w, cr);
        double val = c->t_esign[3 * t + i] * c->t_esign[3 * t + j] * c->elen[m] * c->elen[n] /
                     (4.0 * c->area[t]) * dot3(nrm, cr);
        int k = fill[m]++;
        (*ixcol)[4 * (size_t)m + k] = n;
        (*ixval)[4 * (size_t)m + k] = val;
      }
  }
  fdE->resize(2 * (size_t)ne);
  for (int n = 0; n < ne; ++n) {
    (*fdE)[2 * n] = c->elen[n] / c->area[c->et[2 * n]];
    (*fdE)[2 * n + 1] = c->elen[n] / c->area[c->et[2 * n + 1]];
  }
  fdT->resize(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i)
      (*fdT)[3 * t + i] = c->t_esign[3 * t + i] * c->elen[c->t_edges[3 * t + i]] / c->area[t];
}

}  // namespace bem

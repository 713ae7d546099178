// Work lists for the uneven block-diagonal products (Sec. III-C): LPT (Alg. 1) and the
// modified Part_Schedule (Alg. 2), re-purposed from MPI processes to groups of CTAs.
//
// A task is one object's pair of dense blocks (Z_i, Y_i,eq) with workload W_i = N_E,i^2
// (Sec. III-C-2). A "processor" is one CTA slot of the persistent GEMV launch; P_i becomes the
// number of CTAs that split block i into row panels. Parallel tasks (P_i > 1) start together on
// dedicated slots; sequential tasks follow by LPT. Readings of Alg. 2: "P_i < P_cutoff" takes
// d = 1, otherwise d is the distance to the next approximate square (Q^2 or Q(Q+1)) above P_i;
// ties in tau or finish time go to the lowest index; an increment is undone, and the search
// ends, only when the new schedule is longer (the termination rule of Sec. III-C, which gives
// the two processes per conductor that Sec. IV-B reports for identical conductors).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.cuh"

namespace bem {

static bool approx_square(long n) {
  long q = (long)std::floor(std::sqrt((double)n));
  while (q * q > n) --q;
  while ((q + 1) * (q + 1) <= n) ++q;
  return q * q == n || q * (q + 1) == n;
}

static long next_approx_square(long n) {
  long m = n + 1;
  while (!approx_square(m)) ++m;
  return m;
}

// Mixed LPT: parallel tasks first on dedicated slots, then sequential tasks by LPT.
// Returns the finish times; slot lists in rows (task indices).
static double lpt_moldable(int ntask, const double* W, const int32_t* Pi, int P,
                           std::vector<std::vector<int>>* rows, std::vector<double>* F) {
  F->assign(P, 0.0);
  if (rows) rows->assign(P, {});
  int nxt = 0;
  for (int i = 0; i < ntask; ++i)
    if (Pi[i] > 1) {
      for (int p = nxt; p < nxt + Pi[i] && p < P; ++p) {
        (*F)[p] = W[i] / Pi[i];
        if (rows) (*rows)[p].push_back(i);
      }
      nxt += Pi[i];
    }
  std::vector<int> seq;
  for (int i = 0; i < ntask; ++i)
    if (Pi[i] == 1) seq.push_back(i);
  std::stable_sort(seq.begin(), seq.end(), [&](int a, int b) { return W[a] > W[b]; });
  for (int i : seq) {
    int p = (int)(std::min_element(F->begin(), F->end()) - F->begin());
    (*F)[p] += W[i];
    if (rows) (*rows)[p].push_back(i);
  }
  return *std::max_element(F->begin(), F->end());
}

double part_schedule(int ntask, const double* W, int P, int p_cutoff, int32_t* Pi) {
  for (int i = 0; i < ntask; ++i) Pi[i] = 1;
  std::vector<double> F;
  long a = P;
  double cmax = lpt_moldable(ntask, W, Pi, P, nullptr, &F);
  while (a > 0) {
    int im = 0;
    double h = -1;
    for (int i = 0; i < ntask; ++i) {
      double tau = W[i] / Pi[i];
      if (tau > h) { h = tau; im = i; }
    }
    long d = (p_cutoff <= 0 || Pi[im] < p_cutoff) ? 1 : next_approx_square(Pi[im]) - Pi[im];
    a = (Pi[im] == 1) ? a - d - 1 : a - d;
    if (cmax != h || a < 0) break;
    Pi[im] += (int32_t)d;
    double c2 = lpt_moldable(ntask, W, Pi, P, nullptr, &F);
    if (c2 > cmax) {  // a longer schedule ends the algorithm (Sec. III-C); a tie goes on
      Pi[im] -= (int32_t)d;
      break;
    }
    cmax = c2;
  }
  return cmax;
}

// Row-panel work list of the block GEMV. Slots = 4 CTAs per SM; each object becomes P_i row
// panels from the modified Part_Schedule; a panel is further cut into tasks of at most
// kRowsPerTask rows so one CTA (8 warps) processes one task.
void build_gemv_tasks(const std::vector<int32_t>& n, const std::vector<int64_t>& off,
                      const std::vector<int32_t>& xoff, const std::vector<int32_t>& ld, int nsm,
                      int rows_per_task, std::vector<GemvTask>* tasks) {
  const int nb = (int)n.size();
  std::vector<int> order(nb);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::vector<double> W(nb);
  for (int i = 0; i < nb; ++i) W[i] = (double)n[order[i]] * n[order[i]];
  std::vector<int32_t> Pi(nb, 1);
  const int P = std::max(1, 4 * nsm);
  part_schedule(nb, W.data(), P, 20, Pi.data());
  tasks->clear();
  const int kRowsPerTask = std::max(1, rows_per_task);
  for (int r = 0; r < nb; ++r) {
    int i = order[r];
    int panels = std::max(1, std::min<int>(Pi[r], n[i]));
    // panel p spans rows [bnd(p), bnd(p + 1)): the even split snapped to a whole number of
    // tasks, so only a block's last task can be short (a panel may come out empty)
    auto bnd = [&](int p) {
      if (p >= panels) return (int)n[i];
      const int64_t e = (int64_t)n[i] * p / panels;
      return (int)std::min<int64_t>(n[i], (e + kRowsPerTask / 2) / kRowsPerTask * kRowsPerTask);
    };
    for (int p = 0; p < panels; ++p) {
      const int a = bnd(p), b = bnd(p + 1);
      for (int r0 = a; r0 < b; r0 += kRowsPerTask) {
        GemvTask t;
        t.aoff = off[i];
        t.xoff = xoff[i];
        t.n = n[i];
        t.ld = ld[i];
        t.row0 = r0;
        t.nrows = std::min(kRowsPerTask, b - r0);
        t.sel = 0;
        tasks->push_back(t);
      }
    }
  }
}

// The persistent GEMV plan. On the GPU a task (one object's block) is moldable at the
// granularity of a single row, so the ideal schedule of Sec. III-C (total work spread evenly,
// C_max = C_ideal up to one row) is reachable directly: the rows of all blocks, in order, are
// cut into ncta contiguous ranges of equal matrix bytes, one per resident CTA, with no search
// over P_i. ratio reports the longest CTA's bytes over the mean.
void build_gemv_plan(const std::vector<int32_t>& n, const std::vector<int64_t>& off,
                     const std::vector<int32_t>& ld, int ncta, std::vector<RowInfo>* rows,
                     std::vector<int2>* segs, std::vector<int32_t>* cta_seg, double* ratio) {
  const int nb = (int)n.size();
  std::vector<int32_t> xoff(nb);
  int32_t tot = 0;
  double bytes = 0;
  for (int i = 0; i < nb; ++i) {
    xoff[i] = tot;
    tot += n[i];
    bytes += (double)n[i] * n[i];
  }
  rows->resize(tot);
  for (int i = 0; i < nb; ++i)
    for (int r = 0; r < n[i]; ++r) {
      RowInfo& ri = (*rows)[xoff[i] + r];
      ri.aoff = off[i] + (int64_t)r * ld[i];
      ri.n = n[i];
      ri.xoff = xoff[i];
    }
  segs->clear();
  cta_seg->assign(ncta + 1, 0);
  const double per = bytes / ncta;
  double acc = 0, worst = 0, cur = 0;
  int r0 = 0, p = 0;
  for (int m = 0; m < tot; ++m) {
    const double w = (*rows)[m].n;
    acc += w;
    cur += w;
    // close range p once the running total reaches its share (the last CTA takes the rest)
    if (p < ncta - 1 && acc >= per * (p + 1)) {
      segs->push_back(make_int2(r0, m + 1));
      worst = std::max(worst, cur);
      cur = 0;
      r0 = m + 1;
      ++p;
      (*cta_seg)[p] = (int32_t)segs->size();
    }
  }
  if (r0 < tot) {
    segs->push_back(make_int2(r0, tot));
    worst = std::max(worst, cur);
  }
  for (int q = p + 1; q <= ncta; ++q) (*cta_seg)[q] = (int32_t)segs->size();
  *ratio = per > 0 ? worst / per : 1.0;
}

}  // namespace bem

extern "C" double bem_part_schedule(int ntask, const double* W, int P, int p_cutoff, int32_t* Pi) {
  if (ntask <= 0 || !W || !Pi || P <= 0) {
    bem::set_error("bem_part_schedule: bad arguments");
    return -1.0;
  }
  for (int i = 1; i < ntask; ++i)
    if (W[i] > W[i - 1]) {
      bem::set_error("bem_part_schedule: W must be sorted in decreasing order");
      return -1.0;
    }
  return bem::part_schedule(ntask, W, P, p_cutoff, Pi);
}

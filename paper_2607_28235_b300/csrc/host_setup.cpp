// Host-side symbolic setup: R-tree bisection, block adjacency, fine-level windowed layout,
// GLL nodes and the tridiagonal eigenvalue of the Lanczos estimate.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace r3mg {

// ---------------------------------------------------------------- R-tree bisection
// Section 3 (R-tree of order (m, M)) and Section 4 (point-based agglomeration), read as a
// balanced bulk-loaded bisection: split at ceil(|S|/2) along the longest MBR extent, points
// ordered by (x_a, x_{a+1}, ..., caller index).  Only comparisons and min/max touch the
// coordinates, so the tree is bit-reproducible.

static int tree_depth(int64_t n, int leaf) {
  int t = 0;
  while (((n + ((int64_t)1 << t) - 1) >> t) > leaf) ++t;
  return t;
}

bool partition_points(int64_t n, int dim, const double* x, int leaf, int levels, HostPartition& P, Error& err) {
  if (n < 1 || (dim != 2 && dim != 3) || leaf < 2 || levels < 2) {
    // leaf_size 1 would allow empty leaves (n < 2^D); every box must own a point
    err = {R3MG_E_ARG, "partition: need n >= 1, dim in {2,3}, leaf_size >= 2, levels >= 2"};
    return false;
  }
  for (int64_t i = 0; i < n * dim; ++i)
    if (!std::isfinite(x[i])) { err = {R3MG_E_ARG, "partition: non-finite coordinate"}; return false; }
  const int D = tree_depth(n, leaf);
  if (D - dim * (levels - 2) < 0) {
    err = {R3MG_E_DEPTH, "partition: tree depth " + std::to_string(D) + " too shallow for " +
                             std::to_string(levels) + " levels"};
    return false;
  }
  P.n = n; P.dim = dim; P.depth = D; P.levels = levels;
  P.perm.resize(n);
  std::iota(P.perm.begin(), P.perm.end(), (int64_t)0);
  std::vector<int64_t> bounds{0, n};  // node boundaries at the current depth
  for (int t = 0; t < D; ++t) {
    const int64_t nn = (int64_t)bounds.size() - 1;
    std::vector<int64_t> next(2 * nn + 1);
    next[0] = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nn; ++k) {
      const int64_t s = bounds[k], e = bounds[k + 1];
      double mn[3], mx[3];
      for (int a = 0; a < dim; ++a) { mn[a] = x[P.perm[s] * dim + a]; mx[a] = mn[a]; }
      for (int64_t i = s; i < e; ++i)
        for (int a = 0; a < dim; ++a) {
          const double v = x[P.perm[i] * dim + a];
          mn[a] = std::min(mn[a], v); mx[a] = std::max(mx[a], v);
        }
      int ax = 0; double best = mx[0] - mn[0];
      for (int a = 1; a < dim; ++a)
        if (mx[a] - mn[a] > best) { best = mx[a] - mn[a]; ax = a; }
      std::sort(P.perm.begin() + s, P.perm.begin() + e, [&](int64_t u, int64_t v) {
        for (int k2 = 0; k2 < dim; ++k2) {
          const int a = (ax + k2) % dim;
          const double xu = x[u * dim + a], xv = x[v * dim + a];
          if (xu < xv) return true;
          if (xv < xu) return false;
        }
        return u < v;
      });
      const int64_t h = (e - s + 1) / 2;
      next[2 * k + 1] = s + h;
      next[2 * k + 2] = e;
    }
    bounds.swap(next);
  }
  P.leaf_off = bounds;
  P.iperm.resize(n);
  for (int64_t k = 0; k < n; ++k) P.iperm[P.perm[k]] = k;
  P.box_off.assign(levels, {});
  P.lo.assign(levels, {});
  P.hi.assign(levels, {});
  for (int l = 1; l < levels; ++l) {
    const int64_t stride = (int64_t)1 << (dim * (l - 1));
    std::vector<int64_t>& off = P.box_off[l];
    for (size_t k = 0; k < P.leaf_off.size(); k += stride) off.push_back(P.leaf_off[k]);
    const int64_t nb = (int64_t)off.size() - 1;
    P.lo[l].resize(nb * dim); P.hi[l].resize(nb * dim);
#pragma omp parallel for schedule(static)
    for (int64_t B = 0; B < nb; ++B) {
      for (int a = 0; a < dim; ++a) {
        double mn = x[P.perm[off[B]] * dim + a], mx = mn;
        for (int64_t k = off[B]; k < off[B + 1]; ++k) {
          const double v = x[P.perm[k] * dim + a];
          mn = std::min(mn, v); mx = std::max(mx, v);
        }
        P.lo[l][B * dim + a] = mn; P.hi[l][B * dim + a] = mx;
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------- cell-based agglomeration
// Section 4: an R-tree whose leaves are the cells' MBRs; the agglomerates, visited in their
// listed order, each take the support points of their cells that no earlier agglomerate took.
// Tree: the bisection above applied to cells (node MBR = union of cell MBRs, split key = the
// cell's MBR centre (m_a, m_{a+1}, ..., cell index), leaf_size counts cells).  Cell MBRs are
// taken over the cell's points that belong to the system (entries < 0 are eliminated points);
// cells with no such point take no part.  A point's level-l box is the level-l ancestor of its
// level-1 owner; points are listed by (level-1 owner, caller index); a box's MBR is the union
// of its cells' MBRs.
bool partition_cells(int64_t n, int dim, const double* x, int64_t ncells, const int64_t* cell_ptr,
                     const int64_t* cell_pts, int leaf, int levels, HostPartition& P, Error& err) {
  if (n < 1 || (dim != 2 && dim != 3) || leaf < 2 || levels < 2 || ncells < 1) {
    err = {R3MG_E_ARG, "partition_cells: need n >= 1, dim in {2,3}, ncells >= 1, leaf_size >= 2, levels >= 2"};
    return false;
  }
  if (cell_ptr[0] != 0) { err = {R3MG_E_ARG, "partition_cells: cell_ptr[0] != 0"}; return false; }
  for (int64_t c = 0; c < ncells; ++c)
    if (cell_ptr[c + 1] < cell_ptr[c]) { err = {R3MG_E_ARG, "partition_cells: cell_ptr not monotone"}; return false; }
  for (int64_t k = 0; k < cell_ptr[ncells]; ++k)
    if (cell_pts[k] >= n) { err = {R3MG_E_ARG, "partition_cells: point index out of range"}; return false; }
  for (int64_t i = 0; i < n * dim; ++i)
    if (!std::isfinite(x[i])) { err = {R3MG_E_ARG, "partition_cells: non-finite coordinate"}; return false; }
  std::vector<double> clo(ncells * dim), chi(ncells * dim), cen(ncells * dim);
  std::vector<int64_t> cells;
  for (int64_t c = 0; c < ncells; ++c) {
    bool any = false;
    for (int64_t k = cell_ptr[c]; k < cell_ptr[c + 1]; ++k) {
      const int64_t i = cell_pts[k];
      if (i < 0) continue;
      for (int a = 0; a < dim; ++a) {
        const double v = x[i * dim + a];
        if (!any) { clo[c * dim + a] = v; chi[c * dim + a] = v; }
        else { clo[c * dim + a] = std::min(clo[c * dim + a], v); chi[c * dim + a] = std::max(chi[c * dim + a], v); }
      }
      any = true;
    }
    if (any) {
      cells.push_back(c);
      for (int a = 0; a < dim; ++a) cen[c * dim + a] = 0.5 * (clo[c * dim + a] + chi[c * dim + a]);
    }
  }
  const int64_t ncv = (int64_t)cells.size();
  if (ncv < 1) { err = {R3MG_E_ARG, "partition_cells: no cell holds a point of the system"}; return false; }
  const int D = tree_depth(ncv, leaf);
  if (D - dim * (levels - 2) < 0) {
    err = {R3MG_E_DEPTH, "partition_cells: tree depth " + std::to_string(D) + " too shallow for " +
                             std::to_string(levels) + " levels"};
    return false;
  }
  std::vector<int64_t> bounds{0, ncv};
  for (int t = 0; t < D; ++t) {
    const int64_t nn = (int64_t)bounds.size() - 1;
    std::vector<int64_t> next(2 * nn + 1);
    next[0] = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nn; ++k) {
      const int64_t s = bounds[k], e = bounds[k + 1];
      double mn[3], mx[3];
      for (int a = 0; a < dim; ++a) { mn[a] = clo[cells[s] * dim + a]; mx[a] = chi[cells[s] * dim + a]; }
      for (int64_t i = s; i < e; ++i)
        for (int a = 0; a < dim; ++a) {
          mn[a] = std::min(mn[a], clo[cells[i] * dim + a]);
          mx[a] = std::max(mx[a], chi[cells[i] * dim + a]);
        }
      int ax = 0; double best = mx[0] - mn[0];
      for (int a = 1; a < dim; ++a)
        if (mx[a] - mn[a] > best) { best = mx[a] - mn[a]; ax = a; }
      std::sort(cells.begin() + s, cells.begin() + e, [&](int64_t u, int64_t v) {
        for (int k2 = 0; k2 < dim; ++k2) {
          const int a = (ax + k2) % dim;
          const double cu = cen[u * dim + a], cv = cen[v * dim + a];
          if (cu < cv) return true;
          if (cv < cu) return false;
        }
        return u < v;
      });
      const int64_t h = (e - s + 1) / 2;
      next[2 * k + 1] = s + h;
      next[2 * k + 2] = e;
    }
    bounds.swap(next);
  }
  // first-come ownership by the level-1 agglomerates (the nodes at depth D), in order
  const int64_t n1 = (int64_t)bounds.size() - 1;
  std::vector<int64_t> owner(n, -1);
  for (int64_t K = 0; K < n1; ++K)
    for (int64_t j = bounds[K]; j < bounds[K + 1]; ++j) {
      const int64_t c = cells[j];
      for (int64_t k = cell_ptr[c]; k < cell_ptr[c + 1]; ++k) {
        const int64_t i = cell_pts[k];
        if (i >= 0 && owner[i] < 0) owner[i] = K;
      }
    }
  for (int64_t i = 0; i < n; ++i)
    if (owner[i] < 0) { err = {R3MG_E_ARG, "partition_cells: point " + std::to_string(i) + " is in no cell"}; return false; }
  P.n = n; P.dim = dim; P.depth = D; P.levels = levels;
  std::vector<int64_t> cnt(n1 + 1, 0);
  for (int64_t i = 0; i < n; ++i) ++cnt[owner[i] + 1];
  for (int64_t K = 0; K < n1; ++K) cnt[K + 1] += cnt[K];
  P.leaf_off = cnt;
  P.perm.assign(n, 0);
  {
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < n; ++i) P.perm[fill[owner[i]]++] = i;   // ascending caller index within an owner
  }
  P.iperm.resize(n);
  for (int64_t k = 0; k < n; ++k) P.iperm[P.perm[k]] = k;
  P.box_off.assign(levels, {});
  P.lo.assign(levels, {});
  P.hi.assign(levels, {});
  for (int l = 1; l < levels; ++l) {
    const int shift = dim * (l - 1);
    const int64_t nb = n1 >> shift;
    std::vector<int64_t>& off = P.box_off[l];
    off.resize(nb + 1);
    for (int64_t B = 0; B <= nb; ++B) off[B] = cnt[B << shift];
    P.lo[l].resize(nb * dim); P.hi[l].resize(nb * dim);
    for (int64_t B = 0; B < nb; ++B) {
      const int64_t j0 = bounds[B << shift], j1 = bounds[(B + 1) << shift];
      for (int a = 0; a < dim; ++a) {
        double mn = clo[cells[j0] * dim + a], mx = chi[cells[j0] * dim + a];
        for (int64_t j = j0; j < j1; ++j) {
          mn = std::min(mn, clo[cells[j] * dim + a]);
          mx = std::max(mx, chi[cells[j] * dim + a]);
        }
        P.lo[l][B * dim + a] = mn; P.hi[l][B * dim + a] = mx;
      }
    }
  }
  return true;
}

bool validate_csr(int64_t n, const int64_t* rowptr, const int32_t* colidx, Error& err) {
  if (rowptr[0] != 0) { err = {R3MG_E_ARG, "CSR: rowptr[0] != 0"}; return false; }
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) { err = {R3MG_E_ARG, "CSR: rowptr not monotone"}; return false; }
    bool diag = false;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t c = colidx[k];
      if (c < 0 || c >= n) { err = {R3MG_E_ARG, "CSR: column index out of range"}; return false; }
      diag |= (c == i);
    }
    if (!diag) { err = {R3MG_E_ARG, "CSR: row " + std::to_string(i) + " stores no diagonal entry"}; return false; }
  }
  return true;
}

// Level-1 block adjacency: for each box B, the sorted boxes holding a column of a row of B.
void fine_pattern(const HostPartition& P, const int64_t* rowptr, const int32_t* colidx, HostPattern& pat) {
  const std::vector<int64_t>& off = P.box_off[1];
  const int64_t nb = P.nbox(1);
  std::vector<int64_t> box_of(P.n);
  for (int64_t B = 0; B < nb; ++B)
    for (int64_t k = off[B]; k < off[B + 1]; ++k) box_of[P.perm[k]] = B;  // caller index -> box
  std::vector<std::vector<int64_t>> lists(nb);
#pragma omp parallel
  {
    std::vector<int64_t> stamp(nb, -1);
#pragma omp for schedule(dynamic, 16)
    for (int64_t B = 0; B < nb; ++B) {
      std::vector<int64_t>& L = lists[B];
      for (int64_t k = off[B]; k < off[B + 1]; ++k) {
        const int64_t i = P.perm[k];
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
          const int64_t c = box_of[colidx[e]];
          if (stamp[c] != B) { stamp[c] = B; L.push_back(c); }
        }
      }
      std::sort(L.begin(), L.end());
    }
  }
  pat.ptr.assign(nb + 1, 0);
  for (int64_t B = 0; B < nb; ++B) pat.ptr[B + 1] = pat.ptr[B] + (int64_t)lists[B].size();
  pat.nbr.resize(pat.ptr[nb]);
  for (int64_t B = 0; B < nb; ++B) std::copy(lists[B].begin(), lists[B].end(), pat.nbr.begin() + pat.ptr[B]);
}

// Level l+1 adjacency from level l: a parent holds 2^d consecutive children; P~ is block
// diagonal by parent, so parents are adjacent iff some of their children are.
void coarse_pattern(const HostPattern& fine, int fan, int64_t nbox_coarse, HostPattern& out) {
  std::vector<std::vector<int64_t>> lists(nbox_coarse);
  for (int64_t B = 0; B < nbox_coarse; ++B) {
    std::vector<int64_t>& L = lists[B];
    for (int64_t c = B * fan; c < (B + 1) * fan; ++c)
      for (int64_t e = fine.ptr[c]; e < fine.ptr[c + 1]; ++e) L.push_back(fine.nbr[e] / fan);
    std::sort(L.begin(), L.end());
    L.erase(std::unique(L.begin(), L.end()), L.end());
  }
  out.ptr.assign(nbox_coarse + 1, 0);
  for (int64_t B = 0; B < nbox_coarse; ++B) out.ptr[B + 1] = out.ptr[B] + (int64_t)lists[B].size();
  out.nbr.resize(out.ptr[nbox_coarse]);
  for (int64_t B = 0; B < nbox_coarse; ++B) std::copy(lists[B].begin(), lists[B].end(), out.nbr.begin() + out.ptr[B]);
}

// Fine rows in tree order; each row's entries sorted by tree column (= window order); the
// window of box B is the concatenation of its neighbour boxes' points, so a column is
// addressed by a 16-bit window index.
bool fine_layout(const HostPartition& P, const HostPattern& pat, const int64_t* rowptr, const int32_t* colidx,
                 HostFineLayout& lay, Error& err) {
  const std::vector<int64_t>& off = P.box_off[1];
  const int64_t nb = P.nbox(1), n = P.n;
  std::vector<int64_t> box_of_tree(n);
  for (int64_t B = 0; B < nb; ++B)
    for (int64_t k = off[B]; k < off[B + 1]; ++k) box_of_tree[k] = B;
  // the window keeps, for each neighbour box, only the run of its points between the first and
  // the last one referenced by a row of the box (the rest would be staged for nothing)
  std::vector<int64_t> seg_lo(pat.nbr.size()), seg_hi(pat.nbr.size());
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t B = 0; B < nb; ++B) {
    const int64_t* nb0 = pat.nbr.data() + pat.ptr[B];
    const int64_t nn = pat.ptr[B + 1] - pat.ptr[B];
    for (int64_t e = pat.ptr[B]; e < pat.ptr[B + 1]; ++e) { seg_lo[e] = INT64_MAX; seg_hi[e] = -1; }
    for (int64_t k = off[B]; k < off[B + 1]; ++k) {
      const int64_t i = P.perm[k];
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int64_t t = P.iperm[colidx[e]], c = box_of_tree[t];
        const int64_t s2 = pat.ptr[B] + (std::lower_bound(nb0, nb0 + nn, c) - nb0);
        seg_lo[s2] = std::min(seg_lo[s2], t);
        seg_hi[s2] = std::max(seg_hi[s2], t + 1);
      }
    }
  }
  lay.win_off.resize(pat.nbr.size());
  lay.win_src.resize(pat.nbr.size());
  lay.win_size.resize(nb);
  int64_t wmax = 0;
  for (int64_t B = 0; B < nb; ++B) {
    int64_t w = 0;
    for (int64_t e = pat.ptr[B]; e < pat.ptr[B + 1]; ++e) {
      lay.win_off[e] = (int32_t)std::min<int64_t>(w, INT32_MAX);
      lay.win_src[e] = seg_lo[e];
      w += seg_hi[e] - seg_lo[e];
    }
    if (w > kMaxWindow) {
      err = {R3MG_E_LIMIT, "fine window of box " + std::to_string(B) + " has " + std::to_string(w) +
                               " points (> 65535): use a smaller leaf_size"};
      return false;
    }
    lay.win_size[B] = (int32_t)w;
    wmax = std::max(wmax, w);
  }
  lay.win_max = (int32_t)wmax;
  lay.row_ptr.assign(n + 1, 0);
  for (int64_t k = 0; k < n; ++k) {
    const int64_t i = P.perm[k];
    const int64_t len = rowptr[i + 1] - rowptr[i];
    lay.row_ptr[k + 1] = lay.row_ptr[k] + (len + kPad - 1) / kPad * kPad;
  }
  const int64_t tot = lay.row_ptr[n];
  lay.idx.assign(tot, 0);
  lay.src.assign(tot, -1);
  lay.diag_src.assign(n, -1);
  lay.nnz = rowptr[n];
#pragma omp parallel
  {
    std::vector<std::pair<int64_t, int64_t>> ent;
#pragma omp for schedule(dynamic, 256)
    for (int64_t k = 0; k < n; ++k) {
      const int64_t i = P.perm[k], B = box_of_tree[k];
      ent.clear();
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) ent.emplace_back(P.iperm[colidx[e]], e);
      std::sort(ent.begin(), ent.end());
      int64_t pos = lay.row_ptr[k];
      const int64_t* nb0 = pat.nbr.data() + pat.ptr[B];
      const int64_t nn = pat.ptr[B + 1] - pat.ptr[B];
      for (auto& pe : ent) {
        const int64_t c = box_of_tree[pe.first];
        const int64_t e2 = pat.ptr[B] + (std::lower_bound(nb0, nb0 + nn, c) - nb0);
        lay.idx[pos] = (uint16_t)(lay.win_off[e2] + (pe.first - lay.win_src[e2]));
        lay.src[pos] = pe.second;
        if (pe.first == k) lay.diag_src[k] = pe.second;
        ++pos;
      }
      // padding keeps the row sorted: repeat the last window index, value 0 (src = -1)
      const uint16_t last = pos > lay.row_ptr[k] ? lay.idx[pos - 1] : 0;
      for (; pos < lay.row_ptr[k + 1]; ++pos) lay.idx[pos] = last;
    }
  }
  return true;
}

// ---------------------------------------------------------------- small numerics
// GLL nodes on [0,1]: end points and the roots of P_p' (Newton on P_p' with the second
// derivative from Legendre's equation (1-t^2) P'' = 2 t P' - p(p+1) P).
static void legendre_pd(int p, double t, double& P, double& dP) {
  double p0 = 1.0, p1 = t;
  if (p == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 2; k <= p; ++k) { const double pk = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = pk; }
  P = p1;
  dP = p * (t * p1 - p0) / (t * t - 1.0);
}

void gll_nodes01(int p, double* z) {
  if (p == 0) { z[0] = 0.5; return; }
  z[0] = 0.0; z[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre_pd(p, t, P, dP);
      const double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      const double dt = dP / d2P;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    z[i] = 0.5 * (t + 1.0);
  }
  // symmetric pairs: enforce exact symmetry z_i + z_{p-i} = 1
  for (int i = 1; i < p - i; ++i) { const double a = 0.5 * (z[i] + (1.0 - z[p - i])); z[i] = a; z[p - i] = 1.0 - a; }
  if (p % 2 == 0) z[p / 2] = 0.5;
}

// Largest eigenvalue of a symmetric tridiagonal matrix by Sturm-sequence bisection.
// Largest distance between two support points coupled by a stored entry of A.  Two points
// share a stored entry exactly when they share an element, so this is the largest element
// diameter over the elements whose vertices are all unknowns of the system.
double max_coupled_distance(int64_t n, int dim, const double* coords, const int64_t* rowptr, const int32_t* colidx) {
  double m2 = 0.0;
#pragma omp parallel for schedule(static) reduction(max : m2)
  for (int64_t i = 0; i < n; ++i) {
    const double* xi = coords + i * dim;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const double* xj = coords + (int64_t)colidx[k] * dim;
      double s = 0.0;
      for (int a = 0; a < dim; ++a) s += (xi[a] - xj[a]) * (xi[a] - xj[a]);
      m2 = std::max(m2, s);
    }
  }
  return std::sqrt(m2);
}

double tridiag_max_eig(const std::vector<double>& d, const std::vector<double>& e) {
  return tridiag_kth_eig(d, e, (int)d.size() - 1);
}

// The j-th smallest eigenvalue (j = 0 .. k-1) of the symmetric tridiagonal matrix with diagonal
// d and off-diagonal e, by Sturm-sequence bisection on the Gershgorin interval.
double tridiag_kth_eig(const std::vector<double>& d, const std::vector<double>& e, int j) {
  const int k = (int)d.size();
  if (k == 0) return 0.0;
  double lo = d[0], hi = d[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r); hi = std::max(hi, d[i] + r);
  }
  auto count_below = [&](double s) {  // number of eigenvalues < s
    int cnt = 0; double q = 1.0;
    for (int i = 0; i < k; ++i) {
      const double e2 = (i > 0) ? e[i - 1] * e[i - 1] : 0.0;
      q = d[i] - s - (i > 0 ? e2 / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-16 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(mid) >= j + 1) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace r3mg

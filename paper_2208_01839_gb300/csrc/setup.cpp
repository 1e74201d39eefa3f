// Host-side setup: mesh validation, seeded recursive coordinate bisection,
// renumbering, the 5x5 BSR pattern, element gather lists, overlapping
// subdomains (Eq. RAS) with their ILU(0) patterns and level schedules, and the
// banded pattern of the coarse matrix Z^T J Z (Section 3.1).  Plain C++; runs
// once per context.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <exception>
#include <mutex>
#include <numeric>
#include <queue>
#include <random>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace seird {

namespace {

// Recursive coordinate bisection: the parts [pb, pe) share the nodes idx[lo, hi)
// in proportion to their weights; each cut is orthogonal to the longer side of
// the nodes' bounding box.
void rcb(const double* xy, std::vector<int32_t>& idx, int64_t lo, int64_t hi, int32_t pb, int32_t pe,
         const std::vector<double>& w, std::vector<int32_t>& owner) {
  if (pe - pb == 1) {
    for (int64_t k = lo; k < hi; ++k) owner[idx[k]] = pb;
    return;
  }
  const int32_t pm = pb + (pe - pb) / 2;
  double wl = 0, wt = 0;
  for (int32_t q = pb; q < pe; ++q) {
    wt += w[q];
    if (q < pm) wl += w[q];
  }
  const int64_t cnt = hi - lo;
  int64_t k = lo + (int64_t)std::llround((double)cnt * wl / wt);
  k = std::max<int64_t>(k, lo + (pm - pb));
  k = std::min<int64_t>(k, hi - (pe - pm));
  double mn[2] = {1e300, 1e300}, mx[2] = {-1e300, -1e300};
  for (int64_t q = lo; q < hi; ++q)
    for (int d = 0; d < 2; ++d) {
      mn[d] = std::min(mn[d], xy[2 * (int64_t)idx[q] + d]);
      mx[d] = std::max(mx[d], xy[2 * (int64_t)idx[q] + d]);
    }
  const int ax = (mx[0] - mn[0] >= mx[1] - mn[1]) ? 0 : 1;
  std::nth_element(idx.begin() + lo, idx.begin() + k, idx.begin() + hi, [&](int32_t a, int32_t b) {
    const double xa = xy[2 * (int64_t)a + ax], xb = xy[2 * (int64_t)b + ax];
    return xa < xb || (xa == xb && a < b);
  });
  rcb(xy, idx, lo, k, pb, pm, w, owner);
  rcb(xy, idx, k, hi, pm, pe, w, owner);
}

// Reverse Cuthill-McKee order of a small graph (adjacency lists).
std::vector<int32_t> rcm(const std::vector<std::vector<int32_t>>& adj) {
  const int32_t n = (int32_t)adj.size();
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<char> seen(n, 0);
  while ((int32_t)order.size() < n) {
    int32_t start = -1;
    for (int32_t v = 0; v < n; ++v)
      if (!seen[v] && (start < 0 || adj[v].size() < adj[start].size())) start = v;
    size_t head = order.size();
    order.push_back(start);
    seen[start] = 1;
    while (head < order.size()) {
      int32_t v = order[head++];
      std::vector<int32_t> nb;
      for (int32_t u : adj[v])
        if (!seen[u]) {
          seen[u] = 1;
          nb.push_back(u);
        }
      std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
        return adj[a].size() < adj[b].size() || (adj[a].size() == adj[b].size() && a < b);
      });
      order.insert(order.end(), nb.begin(), nb.end());
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

}  // namespace

int partition_nodes(const seird_mesh* mesh, const seird_options* opt, std::vector<int32_t>& owner_c, int32_t& P,
                    std::string& err) {
  const int64_t n = mesh->n_nodes;
  owner_c.assign(n, 0);
  if (opt->owner) {
    P = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (opt->owner[i] < 0) {
        err = "owner values must be >= 0";
        return SEIRD_EINVAL;
      }
      P = std::max(P, opt->owner[i] + 1);
    }
    std::vector<int64_t> cnt(P, 0);
    for (int64_t i = 0; i < n; ++i) cnt[opt->owner[i]]++;
    for (int32_t q = 0; q < P; ++q)
      if (!cnt[q]) {
        err = "subdomain " + std::to_string(q) + " owns no node";
        return SEIRD_EINVAL;
      }
    std::copy(opt->owner, opt->owner + n, owner_c.begin());
  } else {
    P = opt->n_subdomains;
    if (P < 1 || P > n) {
      err = "n_subdomains must be in [1, n_nodes]";
      return SEIRD_EINVAL;
    }
    std::mt19937_64 rng(opt->seed);
    std::uniform_real_distribution<double> U(0.75, 1.5);  // uneven parts, up to 2x apart
    std::vector<double> w(P);
    for (auto& x : w) x = U(rng);
    std::vector<int32_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    rcb(mesh->xy, idx, 0, n, 0, P, w, owner_c);
  }
  return SEIRD_OK;
}

// Worker threads for the per-subdomain parts of the set-up: the host's cores, at most 16.
static int setup_threads(int32_t units) {
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), 16, (int64_t)units}));
}

// f(i, worker) for i in [0, n): the calling thread is worker 0 and up to nth - 1
// helper threads take items from the same counter, so the loop completes (with
// fewer workers) even where a helper cannot be started.  An exception in any
// worker (a failed allocation) stops the hand-out and is rethrown to the caller
// once every worker has returned.
template <class F>
static void parallel_for(int32_t n, int nth, F&& f) {
  std::atomic<int32_t> next{0};
  std::exception_ptr first;
  std::mutex first_mu;
  auto work = [&](int t) {
    try {
      for (int32_t i = next.fetch_add(1); i < n; i = next.fetch_add(1)) f(i, t);
    } catch (...) {
      next.store(n);
      std::lock_guard<std::mutex> lk(first_mu);
      if (!first) first = std::current_exception();
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nth; ++t) {
    try {
      th.emplace_back(work, t);
    } catch (...) {
      break;
    }
  }
  work(0);
  for (auto& x : th) x.join();
  if (first) std::rethrow_exception(first);
}

// Symbolic block ILU(k) of one subdomain (level of fill; Saad, Iterative Methods for
// Sparse Linear Systems, Section 10.3.3), row by row in the local order: the row's
// own blocks have level 0; eliminating with pivot row m < i, in increasing m, offers
// every block (m, j), j > m, of row m's upper part the level lev(i, m) + lev(m, j) + 1,
// and a block joins row i when its level is at most k.  Replaces the local pattern
// (row ends, columns, J blocks with -1 for fill, diagonal positions) in place; rows
// stay sorted by column.
static void iluk_pattern(int k, int32_t nl, std::vector<int64_t>& rstart, std::vector<int64_t>& rowend,
                         std::vector<int32_t>& l_col, std::vector<int32_t>& l_gblk, std::vector<int64_t>& diag) {
  std::vector<int32_t> ncol, ngblk;
  ncol.reserve(l_col.size() * 2);
  ngblk.reserve(l_col.size() * 2);
  std::vector<int64_t> nend(nl), ndiag(nl);
  // the upper part of every finished row with its levels, for the rows below it
  std::vector<int64_t> uptr(nl + 1, 0);
  std::vector<int32_t> ucol;
  std::vector<int8_t> ulev;
  std::vector<int8_t> lev(nl, -1);  // level of each column in the current row (-1: absent)
  std::vector<int32_t> gb(nl, -1);  // J block of each column in the current row
  std::vector<int32_t> cols;
  std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>> pivots;
  for (int32_t i = 0; i < nl; ++i) {
    cols.clear();
    for (int64_t a = rstart[i]; a < rstart[i + 1]; ++a) {
      const int32_t c = l_col[a];
      lev[c] = 0;
      gb[c] = l_gblk[a];
      cols.push_back(c);
      if (c < i) pivots.push(c);
    }
    while (!pivots.empty()) {
      const int32_t m = pivots.top();
      pivots.pop();
      const int lim = lev[m];
      if (lim >= k) continue;  // every block it offers would have a level above k
      for (int64_t b = uptr[m]; b < uptr[m + 1]; ++b) {
        const int32_t j = ucol[b];
        const int l = lim + ulev[b] + 1;
        if (l > k) continue;
        if (lev[j] < 0) {
          lev[j] = (int8_t)l;
          gb[j] = -1;
          cols.push_back(j);
          if (j < i) pivots.push(j);  // j > m: popped after m
        } else if (l < lev[j]) {
          lev[j] = (int8_t)l;
        }
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t c : cols) {
      if (c == i) ndiag[i] = (int64_t)ncol.size();
      if (c > i) {
        ucol.push_back(c);
        ulev.push_back(lev[c]);
      }
      ncol.push_back(c);
      ngblk.push_back(gb[c]);
      lev[c] = -1;
      gb[c] = -1;
    }
    uptr[i + 1] = (int64_t)ucol.size();
    nend[i] = (int64_t)ncol.size();
  }
  l_col.swap(ncol);
  l_gblk.swap(ngblk);
  rowend.swap(nend);
  diag.swap(ndiag);
  rstart[0] = 0;
  for (int32_t i = 0; i < nl; ++i) rstart[i + 1] = rowend[i];
}

int build_setup(const seird_mesh* mesh, const seird_options* opt, HostSetup& hs, std::string& err) {
  const int64_t n = mesh->n_nodes, m = mesh->n_tris;
  if (n < 3 || m < 1 || !mesh->xy || !mesh->tri) {
    err = "mesh needs at least 3 nodes, 1 triangle and non-NULL arrays";
    return SEIRD_EINVAL;
  }
  if (n > (int64_t)INT32_MAX / 8 || m > (int64_t)INT32_MAX / 9) {
    err = "mesh too large for 32-bit element maps";
    return SEIRD_EINVAL;
  }
  for (int64_t t = 0; t < m; ++t) {
    const int32_t* v = mesh->tri + 3 * t;
    for (int a = 0; a < 3; ++a)
      if (v[a] < 0 || v[a] >= n) {
        err = "triangle " + std::to_string(t) + " has a node index out of range";
        return SEIRD_EINVAL;
      }
    const double* p0 = mesh->xy + 2 * (int64_t)v[0];
    const double* p1 = mesh->xy + 2 * (int64_t)v[1];
    const double* p2 = mesh->xy + 2 * (int64_t)v[2];
    const double twoA = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p2[0] - p0[0]) * (p1[1] - p0[1]);
    if (!(twoA > 0)) {
      err = "triangle " + std::to_string(t) + " is not counter-clockwise or is degenerate";
      return SEIRD_EINVAL;
    }
  }
  hs.n = n;
  hs.m = m;

  // ---- partition ---------------------------------------------------------
  std::vector<int32_t> owner_c;
  int32_t P;
  const int prc = partition_nodes(mesh, opt, owner_c, P, err);
  if (prc) return prc;
  hs.P = P;
  if (opt->ilu_fill < 0 || opt->ilu_fill > 8) {
    err = "ilu_fill must be 0-8";
    return SEIRD_EINVAL;
  }
  hs.ilu_fill = opt->ilu_fill;

  // ---- internal numbering: nodes sorted by (owner, caller index) ----------
  hs.own_ptr.assign(P + 1, 0);
  for (int64_t i = 0; i < n; ++i) hs.own_ptr[owner_c[i] + 1]++;
  for (int32_t q = 0; q < P; ++q) hs.own_ptr[q + 1] += hs.own_ptr[q];
  hs.perm.resize(n);
  hs.iperm.resize(n);
  hs.owner.resize(n);
  {
    std::vector<int32_t> fill(hs.own_ptr.begin(), hs.own_ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
      int32_t k = fill[owner_c[i]]++;
      hs.perm[k] = (int32_t)i;
      hs.iperm[i] = k;
      hs.owner[k] = owner_c[i];
    }
  }
  hs.xy.resize(2 * n);
  for (int64_t k = 0; k < n; ++k) {
    hs.xy[2 * k] = mesh->xy[2 * (int64_t)hs.perm[k]];
    hs.xy[2 * k + 1] = mesh->xy[2 * (int64_t)hs.perm[k] + 1];
  }
  // triangles renumbered, then ordered by their smallest node (stable)
  {
    std::vector<int32_t> tri(3 * m);
    std::vector<int32_t> key(m);
    for (int64_t t = 0; t < m; ++t) {
      for (int a = 0; a < 3; ++a) tri[3 * t + a] = hs.iperm[mesh->tri[3 * t + a]];
      key[t] = std::min(tri[3 * t], std::min(tri[3 * t + 1], tri[3 * t + 2]));
    }
    std::vector<int32_t> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    hs.tri.resize(3 * m);
    for (int64_t t = 0; t < m; ++t)
      for (int a = 0; a < 3; ++a) hs.tri[3 * t + a] = tri[3 * (int64_t)ord[t] + a];
  }

  // ---- element incidence and BSR pattern ---------------------------------
  // node -> (t*3 + a), ordered by triangle; a row's blocks are the vertices of
  // its incident triangles, sorted and deduplicated row by row
  hs.node_inc_ptr.assign(n + 1, 0);
  for (int64_t t = 0; t < m; ++t)
    for (int a = 0; a < 3; ++a) hs.node_inc_ptr[hs.tri[3 * t + a] + 1]++;
  for (int64_t i = 0; i < n; ++i) hs.node_inc_ptr[i + 1] += hs.node_inc_ptr[i];
  hs.node_inc.resize(3 * m);
  {
    std::vector<int32_t> fill(hs.node_inc_ptr.begin(), hs.node_inc_ptr.end() - 1);
    for (int64_t t = 0; t < m; ++t)
      for (int a = 0; a < 3; ++a) hs.node_inc[fill[hs.tri[3 * t + a]]++] = (int32_t)(3 * t + a);
  }
  {
    hs.row_ptr.assign(n + 1, 0);
    hs.col.clear();
    hs.col.reserve(8 * (size_t)n);
    std::vector<int32_t> cols;
    for (int64_t i = 0; i < n; ++i) {
      cols.clear();
      for (int32_t e = hs.node_inc_ptr[i]; e < hs.node_inc_ptr[i + 1]; ++e) {
        const int64_t t = hs.node_inc[e] / 3;
        for (int b = 0; b < 3; ++b) cols.push_back(hs.tri[3 * t + b]);
      }
      if (cols.empty()) {
        err = "node " + std::to_string(hs.perm[i]) + " belongs to no triangle";
        return SEIRD_EINVAL;
      }
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      hs.col.insert(hs.col.end(), cols.begin(), cols.end());
      hs.row_ptr[i + 1] = (int32_t)hs.col.size();
    }
  }
  const int64_t nnzb = hs.col.size();
  auto find_blk = [&](int32_t i, int32_t j) -> int32_t {
    const int32_t* b = hs.col.data() + hs.row_ptr[i];
    const int32_t* e = hs.col.data() + hs.row_ptr[i + 1];
    const int32_t* p = std::lower_bound(b, e, j);
    return (int32_t)(p - hs.col.data());
  };
  constexpr int64_t CHUNK = 1 << 16;  // rows or triangles per task of the parallel loops below
  hs.tpos.resize(nnzb);
  parallel_for((int32_t)((n + CHUNK - 1) / CHUNK), setup_threads(64), [&](int32_t ch, int) {
    const int64_t i1 = std::min<int64_t>(n, (ch + 1) * CHUNK);
    for (int64_t i = ch * CHUNK; i < i1; ++i)
      for (int32_t k = hs.row_ptr[i]; k < hs.row_ptr[i + 1]; ++k) hs.tpos[k] = find_blk(hs.col[k], (int32_t)i);
  });

  // ---- element gather lists (deterministic: ordered by triangle) ---------
  // (the node lists were built with the pattern above)
  hs.blk_inc_ptr.assign(nnzb + 1, 0);
  std::vector<int32_t> tblk(9 * m);
  parallel_for((int32_t)((m + CHUNK - 1) / CHUNK), setup_threads(64), [&](int32_t ch, int) {
    const int64_t t1 = std::min<int64_t>(m, (ch + 1) * CHUNK);
    for (int64_t t = ch * CHUNK; t < t1; ++t)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) tblk[9 * t + 3 * a + b] = find_blk(hs.tri[3 * t + a], hs.tri[3 * t + b]);
  });
  for (int64_t e = 0; e < 9 * m; ++e) hs.blk_inc_ptr[tblk[e] + 1]++;
  for (int64_t k = 0; k < nnzb; ++k) hs.blk_inc_ptr[k + 1] += hs.blk_inc_ptr[k];
  hs.blk_inc.resize(9 * m);
  {
    std::vector<int32_t> fill(hs.blk_inc_ptr.begin(), hs.blk_inc_ptr.end() - 1);
    for (int64_t t = 0; t < m; ++t)
      for (int ab = 0; ab < 9; ++ab) hs.blk_inc[fill[tblk[9 * t + ab]]++] = (int32_t)(9 * t + ab);
  }
  tblk.clear();
  tblk.shrink_to_fit();

  // ---- overlapping subdomains, local patterns, ILU(0) maps, levels --------
  // Subdomains are independent: each is built into its own buffers (threads over
  // the host's cores, one node-map per thread) and the buffers are concatenated in
  // subdomain order, so the result does not depend on the thread count.  Block
  // indices inside a part are relative to the subdomain's first block.
  const int delta = std::max(0, opt->overlap);
  struct SdPart {
    std::vector<int32_t> nodes;          // local rows: internal nodes, ascending
    std::vector<int64_t> rowend;         // end of each local row's blocks
    std::vector<int32_t> l_col, l_gblk;  // local column and J block of each local block
    std::vector<int64_t> diag;           // diagonal block of each row
    std::vector<int64_t> upd;            // ILU(0) update pairs (destination, source)
    std::vector<int64_t> updend;         // pairs issued up to and including each block
    std::vector<int32_t> order[2], lb[2];
  };
  std::vector<SdPart> parts(P);
  {
    const int nth = setup_threads(P);
    std::vector<std::vector<int32_t>> locs(nth);
    parallel_for(P, nth, [&](int32_t q, int th) {
      std::vector<int32_t>& loc = locs[th];  // internal node -> local row, -2 while found, -1 outside
      if (loc.empty()) loc.assign(n, -1);
      SdPart& S = parts[q];
      std::vector<int32_t>& nodes = S.nodes;
      std::vector<int32_t> front, next;
      for (int32_t i = hs.own_ptr[q]; i < hs.own_ptr[q + 1]; ++i) {
        nodes.push_back(i);
        front.push_back(i);
        loc[i] = -2;
      }
      for (int d = 0; d < delta; ++d) {
        next.clear();
        for (int32_t i : front)
          for (int32_t k = hs.row_ptr[i]; k < hs.row_ptr[i + 1]; ++k) {
            const int32_t j = hs.col[k];
            if (loc[j] == -1) {
              loc[j] = -2;
              next.push_back(j);
              nodes.push_back(j);
            }
          }
        front.swap(next);
      }
      std::sort(nodes.begin(), nodes.end());
      const int32_t nl = (int32_t)nodes.size();
      for (int32_t l = 0; l < nl; ++l) loc[nodes[l]] = l;
      // local BSR rows (restriction of J's rows to the subdomain keeps column order)
      int64_t pos = 0;
      std::vector<int64_t> rstart(nl + 1);
      S.rowend.resize(nl);
      for (int32_t l = 0; l < nl; ++l) {
        rstart[l] = pos;
        const int32_t g = nodes[l];
        for (int32_t k = hs.row_ptr[g]; k < hs.row_ptr[g + 1]; ++k) {
          const int32_t j = hs.col[k];
          if (loc[j] >= 0) {
            S.l_col.push_back(loc[j]);
            S.l_gblk.push_back(k);
            if (j == g) S.diag.push_back(pos);
            ++pos;
          }
        }
        S.rowend[l] = pos;
      }
      rstart[nl] = pos;
      if (opt->ilu_fill > 0) iluk_pattern(opt->ilu_fill, nl, rstart, S.rowend, S.l_col, S.l_gblk, S.diag);
      // update pairs of the factorisation: for lower block (i,k): every (k,j) with j > k and (i,j) present
      std::vector<int64_t> rowpos(nl, -1);  // local col -> block index in the current row
      S.updend.reserve(pos);
      for (int32_t i = 0; i < nl; ++i) {
        for (int64_t a = rstart[i]; a < rstart[i + 1]; ++a) rowpos[S.l_col[a]] = a;
        for (int64_t a = rstart[i]; a < rstart[i + 1]; ++a) {
          const int32_t k = S.l_col[a];
          if (k < i) {
            for (int64_t b = rstart[k]; b < rstart[k + 1]; ++b) {
              const int32_t j = S.l_col[b];
              if (j > k && rowpos[j] >= 0) {
                S.upd.push_back(rowpos[j]);
                S.upd.push_back(b);
              }
            }
          }
          S.updend.push_back((int64_t)S.upd.size() / 2);
        }
        for (int64_t a = rstart[i]; a < rstart[i + 1]; ++a) rowpos[S.l_col[a]] = -1;
      }
      // forward levels (lower triangle) and backward levels (upper triangle)
      std::vector<int32_t> lev(nl);
      for (int dir = 0; dir < 2; ++dir) {
        int32_t nlev = 0;
        if (dir == 0) {
          for (int32_t i = 0; i < nl; ++i) {
            int32_t lv = 0;
            for (int64_t a = rstart[i]; a < rstart[i + 1]; ++a)
              if (S.l_col[a] < i) lv = std::max(lv, lev[S.l_col[a]] + 1);
            lev[i] = lv;
            nlev = std::max(nlev, lv + 1);
          }
        } else {
          for (int32_t i = nl - 1; i >= 0; --i) {
            int32_t lv = 0;
            for (int64_t a = rstart[i]; a < rstart[i + 1]; ++a)
              if (S.l_col[a] > i) lv = std::max(lv, lev[S.l_col[a]] + 1);
            lev[i] = lv;
            nlev = std::max(nlev, lv + 1);
          }
        }
        std::vector<int32_t>& lb = S.lb[dir];
        lb.assign(nlev + 1, 0);
        for (int32_t i = 0; i < nl; ++i) lb[lev[i] + 1]++;
        for (int32_t v = 0; v < nlev; ++v) lb[v + 1] += lb[v];
        std::vector<int32_t>& order = S.order[dir];
        order.resize(nl);
        std::vector<int32_t> fill(lb.begin(), lb.end() - 1);
        if (dir == 0) {
          for (int32_t i = 0; i < nl; ++i) order[fill[lev[i]]++] = i;
        } else {
          for (int32_t i = nl - 1; i >= 0; --i) order[fill[lev[i]]++] = i;
        }
      }
      for (int32_t l = 0; l < nl; ++l) loc[nodes[l]] = -1;
    });
  }
  // concatenation: every part's slice is known from prefix sums, so the parts are
  // copied into place in parallel
  {
    std::vector<int64_t> roff(P + 1, 0), boff(P + 1, 0), uoff(P + 1, 0), loff[2];
    loff[0].assign(P + 1, 0);
    loff[1].assign(P + 1, 0);
    for (int32_t q = 0; q < P; ++q) {
      const SdPart& S = parts[q];
      roff[q + 1] = roff[q] + (int64_t)S.nodes.size();
      boff[q + 1] = boff[q] + (int64_t)S.l_col.size();
      uoff[q + 1] = uoff[q] + (int64_t)S.upd.size() / 2;
      for (int dir = 0; dir < 2; ++dir) {
        loff[dir][q + 1] = loff[dir][q] + (int64_t)S.lb[dir].size();
        hs.max_levels = std::max(hs.max_levels, (int32_t)S.lb[dir].size() - 1);
      }
      hs.max_sd_rows = std::max(hs.max_sd_rows, (int32_t)S.nodes.size());
    }
    const int64_t NLt = roff[P], NLBt = boff[P], NUt = uoff[P];
    if (NLt > INT32_MAX || NLBt > INT32_MAX) {
      err = "subdomains too large for 32-bit local maps";
      return SEIRD_EINVAL;
    }
    hs.sd_row0.resize(P + 1);
    for (int32_t q = 0; q <= P; ++q) hs.sd_row0[q] = (int32_t)roff[q];
    hs.sd_node.resize(NLt);
    hs.l_row_ptr.resize(NLt + 1);
    hs.l_row_ptr[0] = 0;
    hs.l_diag.resize(NLt);
    hs.l_col.resize(NLBt);
    hs.l_gblk.resize(NLBt);
    hs.upd_ptr.resize(NLBt + 1);
    hs.upd_ptr[0] = 0;
    hs.upd.resize(2 * NUt);
    hs.fwd_order.resize(NLt);
    hs.bwd_order.resize(NLt);
    hs.fwd_lev.resize(loff[0][P]);
    hs.bwd_lev.resize(loff[1][P]);
    hs.sd_fwd_lev0.resize(P + 1);
    hs.sd_bwd_lev0.resize(P + 1);
    for (int32_t q = 0; q <= P; ++q) {
      hs.sd_fwd_lev0[q] = (int32_t)loff[0][q];
      hs.sd_bwd_lev0[q] = (int32_t)loff[1][q];
    }
    bool diag_ok = true;
    for (int32_t q = 0; q < P; ++q) diag_ok &= parts[q].diag.size() == parts[q].nodes.size();
    if (!diag_ok) {
      err = "internal error: missing diagonal block in a subdomain";
      return SEIRD_EINVAL;
    }
    parallel_for(P, setup_threads(P), [&](int32_t q, int) {
      SdPart& S = parts[q];
      const int64_t r0 = roff[q], b0 = boff[q], u0 = uoff[q];
      const int64_t nl = (int64_t)S.nodes.size();
      std::copy(S.nodes.begin(), S.nodes.end(), hs.sd_node.begin() + r0);
      for (int64_t l = 0; l < nl; ++l) {
        hs.l_row_ptr[r0 + l + 1] = b0 + S.rowend[l];
        hs.l_diag[r0 + l] = b0 + S.diag[l];
      }
      std::copy(S.l_col.begin(), S.l_col.end(), hs.l_col.begin() + b0);
      std::copy(S.l_gblk.begin(), S.l_gblk.end(), hs.l_gblk.begin() + b0);
      for (size_t a = 0; a < S.updend.size(); ++a) hs.upd_ptr[b0 + a + 1] = u0 + S.updend[a];
      for (size_t k = 0; k < S.upd.size(); ++k) hs.upd[2 * u0 + k] = b0 + S.upd[k];
      for (int dir = 0; dir < 2; ++dir) {
        std::vector<int32_t>& order = dir == 0 ? hs.fwd_order : hs.bwd_order;
        std::vector<int32_t>& levs = dir == 0 ? hs.fwd_lev : hs.bwd_lev;
        std::copy(S.order[dir].begin(), S.order[dir].end(), order.begin() + r0);
        std::copy(S.lb[dir].begin(), S.lb[dir].end(), levs.begin() + loff[dir][q]);
      }
      S = SdPart();  // release the part
    });
    parts.clear();
    parts.shrink_to_fit();
  }

  // ---- ILU(0) solve plans ---------------------------------------------------
  // The solve numbers a subdomain's solution entries by their position in the
  // sweep (forward y and backward z each in their own order), so the column of
  // every factor block is the position of the entry it multiplies, and a row
  // record holds: forward (node, first block, block count, 0); backward (forward
  // position of the row, first block, block count, node if the subdomain owns it
  // else -1).
  // Built per subdomain in parallel (block indices relative to the subdomain's first
  // solve block), then concatenated in subdomain order.
  struct PlanPart {
    std::vector<int32_t> levpos, row, cnt, info, col;
    std::vector<int64_t> levblk, start, src;
  };
  for (int dir = 0; dir < 2; ++dir) {
    HostSetup::SolvePlan& sp = dir == 0 ? hs.sp_fwd : hs.sp_bwd;
    const std::vector<int32_t>& order = dir == 0 ? hs.fwd_order : hs.bwd_order;
    const std::vector<int32_t>& levs = dir == 0 ? hs.fwd_lev : hs.bwd_lev;
    const std::vector<int32_t>& lev0 = dir == 0 ? hs.sd_fwd_lev0 : hs.sd_bwd_lev0;
    std::vector<PlanPart> pp(P);
    parallel_for(P, setup_threads(P), [&](int32_t q, int) {
      PlanPart& T = pp[q];
      const int32_t r0 = hs.sd_row0[q];
      const int32_t nlq = hs.sd_row0[q + 1] - r0;
      std::vector<int32_t> posf(nlq, 0), posd(nlq, 0);
      for (int32_t k = 0; k < nlq; ++k) {
        posf[hs.fwd_order[r0 + k]] = k;
        posd[order[r0 + k]] = k;
      }
      const int32_t nlev = lev0[q + 1] - lev0[q] - 1;
      T.levpos.push_back(0);
      T.levblk.push_back(0);
      int32_t pos = 0, in_level = 0;
      for (int32_t v = 0; v < nlev; ++v) {
        for (int32_t k = levs[lev0[q] + v]; k < levs[lev0[q] + v + 1]; ++k) {
          const int32_t i = order[r0 + k];
          const int64_t R = (int64_t)r0 + i;
          int32_t nb = 0;
          if (dir == 0) {
            nb = (int32_t)(hs.l_diag[R] - hs.l_row_ptr[R]);
          } else {
            nb = 1 + (int32_t)(hs.l_row_ptr[R + 1] - hs.l_diag[R] - 1);
          }
          if ((in_level > 0 && in_level + nb > SOLVE_BUF_BLOCKS) ||
              pos - T.levpos.back() >= SOLVE_BUF_ROWS) {  // split: rows of a level are independent
            T.levpos.push_back(pos);
            T.levblk.push_back((int64_t)T.src.size());
            in_level = 0;
          }
          T.row.push_back(i);
          T.start.push_back((int64_t)T.src.size());
          T.cnt.push_back(nb);
          const int32_t node = hs.sd_node[R];
          const bool owned = node >= hs.own_ptr[q] && node < hs.own_ptr[q + 1];
          T.info.push_back(dir == 0 ? node : posf[i]);
          T.info.push_back((int32_t)((int64_t)T.src.size() - T.levblk.back()));
          T.info.push_back(nb);
          T.info.push_back(dir == 0 ? 0 : (owned ? node : -1));
          if (dir == 0) {
            for (int64_t a = hs.l_row_ptr[R]; a < hs.l_diag[R]; ++a) {
              T.src.push_back(a);
              T.col.push_back(posf[hs.l_col[a]]);
            }
          } else {
            T.src.push_back(-1 - R);
            T.col.push_back(posd[i]);
            for (int64_t a = hs.l_diag[R] + 1; a < hs.l_row_ptr[R + 1]; ++a) {
              T.src.push_back(a);
              T.col.push_back(posd[hs.l_col[a]]);
            }
          }
          in_level += nb;
          ++pos;
        }
        T.levpos.push_back(pos);
        T.levblk.push_back((int64_t)T.src.size());
        in_level = 0;
      }
    });
    // concatenation: slices from prefix sums, copied in parallel
    std::vector<int64_t> loff(P + 1, 0), roff(P + 1, 0), soff(P + 1, 0);
    for (int32_t q = 0; q < P; ++q) {
      loff[q + 1] = loff[q] + (int64_t)pp[q].levpos.size();
      roff[q + 1] = roff[q] + (int64_t)pp[q].row.size();
      soff[q + 1] = soff[q] + (int64_t)pp[q].src.size();
    }
    sp.sd_lev0.resize(P + 1);
    for (int32_t q = 0; q <= P; ++q) sp.sd_lev0[q] = (int32_t)loff[q];
    sp.levpos.resize(loff[P]);
    sp.levblk.resize(loff[P]);
    sp.row.resize(roff[P]);
    sp.start.resize(roff[P]);
    sp.cnt.resize(roff[P]);
    sp.info.resize(4 * roff[P]);
    sp.src.resize(soff[P]);
    sp.col.resize(soff[P]);
    parallel_for(P, setup_threads(P), [&](int32_t q, int) {
      PlanPart& T = pp[q];
      const int64_t l0 = loff[q], r0 = roff[q], s0 = soff[q];
      std::copy(T.levpos.begin(), T.levpos.end(), sp.levpos.begin() + l0);
      for (size_t k = 0; k < T.levblk.size(); ++k) sp.levblk[l0 + k] = s0 + T.levblk[k];
      std::copy(T.row.begin(), T.row.end(), sp.row.begin() + r0);
      for (size_t k = 0; k < T.start.size(); ++k) sp.start[r0 + k] = s0 + T.start[k];
      std::copy(T.cnt.begin(), T.cnt.end(), sp.cnt.begin() + r0);
      std::copy(T.info.begin(), T.info.end(), sp.info.begin() + 4 * r0);
      std::copy(T.src.begin(), T.src.end(), sp.src.begin() + s0);
      std::copy(T.col.begin(), T.col.end(), sp.col.begin() + s0);
      T = PlanPart();
    });
    for (int32_t q = 0; q < P; ++q)
      for (int32_t v = sp.sd_lev0[q]; v + 1 < sp.sd_lev0[q + 1]; ++v)
        sp.max_lev_blocks = std::max<int32_t>(sp.max_lev_blocks, (int32_t)(sp.levblk[v + 1] - sp.levblk[v]));
  }

  // ---- launch order of the subdomain CTAs ------------------------------------
  // Subdomains differ in size (2k-8k nodes at 4096 subdomains) and several waves of
  // CTAs share the SMs; launched longest first (a list schedule), the short ones fill
  // the tail instead of a long one starting last.
  {
    std::vector<int64_t> w(P);
    for (int32_t q = 0; q < P; ++q) w[q] = solve_work(hs, q);
    hs.sd_sched.resize(P);
    for (int32_t q = 0; q < P; ++q) hs.sd_sched[q] = q;
    std::stable_sort(hs.sd_sched.begin(), hs.sd_sched.end(), [&](int32_t a, int32_t b) { return w[a] > w[b]; });
  }

  // ---- coarse units: groups of consecutive subdomains -----------------------
  // The bisection numbers spatial neighbours consecutively, so a group of G
  // consecutive subdomains is a compact region.  G = options.coarse_group, or
  // with 0 the smallest G that keeps the explicit inverse of A_c affordable.
  {
    int32_t G = opt->coarse_group;
    if (G < 0) {
      err = "coarse_group must be >= 0";
      return SEIRD_EINVAL;
    }
    if (G == 0) {
      G = 1;
      while (5 * (int64_t)((P + G - 1) / G) > DENSE_COARSE_MAX || (P + G - 1) / G > COARSE_BLOCKCOL_MAX) ++G;
    }
    G = std::min(G, P);
    hs.cG = G;
    hs.Pc = (P + G - 1) / G;
    hs.cunit_ptr.resize(hs.Pc + 1);
    for (int32_t u = 0; u <= hs.Pc; ++u) hs.cunit_ptr[u] = hs.own_ptr[std::min<int64_t>((int64_t)u * G, P)];
    hs.cunit.resize(n);
    for (int64_t i = 0; i < n; ++i) hs.cunit[i] = hs.owner[i] / G;
  }

  // ---- A Z segments: per row, the blocks of each coarse unit --------------
  {
    hs.az_ptr.assign(n + 1, 0);
    hs.az_unit.clear();
    hs.az_blk.clear();
    for (int64_t i = 0; i < n; ++i) {
      for (int32_t k = hs.row_ptr[i]; k < hs.row_ptr[i + 1]; ++k) {
        const int32_t u = hs.cunit[hs.col[k]];
        if (k == hs.row_ptr[i] || u != hs.cunit[hs.col[k - 1]]) {
          hs.az_unit.push_back(u);
          hs.az_blk.push_back(k);
        }
      }
      hs.az_ptr[i + 1] = (int64_t)hs.az_unit.size();
    }
    hs.az_blk.push_back((int32_t)hs.col.size());
  }

  // ---- coarse pattern: unit graph, RCM order, band, segment sums ----------
  {
    const int32_t P = hs.Pc;  // the coarse matrix has one 5x5 block row per unit
    std::vector<std::vector<int32_t>> adj(P);
    std::vector<int64_t> pq;
    pq.reserve(nnzb);
    for (int64_t i = 0; i < n; ++i)
      for (int32_t k = hs.row_ptr[i]; k < hs.row_ptr[i + 1]; ++k) {
        int32_t a = hs.cunit[i], b = hs.cunit[hs.col[k]];
        if (a != b) pq.push_back((int64_t)a * P + b);
      }
    std::sort(pq.begin(), pq.end());
    pq.erase(std::unique(pq.begin(), pq.end()), pq.end());
    for (int64_t v : pq) adj[v / P].push_back((int32_t)(v % P));
    std::vector<int32_t> ord = rcm(adj);
    hs.cpos.assign(P, 0);
    for (int32_t k = 0; k < P; ++k) hs.cpos[ord[k]] = k;
    int32_t band = 0;
    for (int64_t v : pq) band = std::max(band, std::abs(hs.cpos[v / P] - hs.cpos[v % P]));
    hs.cband = band;
    const int64_t W = 2 * (int64_t)band + 1;
    // J blocks ordered by (cpos[owner(row)], cpos[owner(col)], block id)
    std::vector<int64_t> key(nnzb);
    std::vector<int32_t> rowof(nnzb);
    for (int64_t i = 0; i < n; ++i)
      for (int32_t k = hs.row_ptr[i]; k < hs.row_ptr[i + 1]; ++k) rowof[k] = (int32_t)i;
    for (int64_t k = 0; k < nnzb; ++k)
      key[k] = (int64_t)hs.cpos[hs.cunit[rowof[k]]] * P + hs.cpos[hs.cunit[hs.col[k]]];
    // stable counting sort on the key's banded slot p W + (q - p + band): the same order
    // as sorting by (p, q) and then by block id
    {
      std::vector<int64_t> cnt((size_t)P * W + 1, 0);
      auto slot = [&](int64_t kk) { return (kk / P) * W + (kk % P - kk / P + band); };
      for (int64_t k = 0; k < nnzb; ++k) cnt[slot(key[k]) + 1]++;
      for (size_t v = 1; v < cnt.size(); ++v) cnt[v] += cnt[v - 1];
      hs.cseg_blk.resize(nnzb);
      for (int64_t k = 0; k < nnzb; ++k) hs.cseg_blk[cnt[slot(key[k])]++] = (int32_t)k;
    }
    const int32_t CH = 256;  // blocks per chunk
    hs.cchunk_ptr.assign(1, 0);
    hs.cdst_ptr.assign(1, 0);
    int64_t s = 0;
    while (s < nnzb) {
      int64_t e = s;
      const int64_t kk = key[hs.cseg_blk[s]];
      while (e < nnzb && key[hs.cseg_blk[e]] == kk) ++e;
      for (int64_t c = s; c < e; c += CH) hs.cchunk_ptr.push_back((int32_t)std::min<int64_t>(e, c + CH));
      hs.cdst_ptr.push_back((int32_t)hs.cchunk_ptr.size() - 1);
      const int64_t pr = kk / P, qc = kk % P;
      hs.cdst_idx.push_back(pr * W + (qc - pr + band));
      s = e;
    }
  }
  return SEIRD_OK;
}

int64_t solve_work(const HostSetup& hs, int32_t q) {
  int64_t w = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const HostSetup::SolvePlan& sp = dir == 0 ? hs.sp_fwd : hs.sp_bwd;
    const int32_t v0 = sp.sd_lev0[q], v1 = sp.sd_lev0[q + 1] - 1;
    w += sp.levblk[v1] - sp.levblk[v0] + SOLVE_STAGE_WEIGHT * (int64_t)(v1 - v0);
  }
  return w;
}

// Invariants of a set-up that the kernels rely on without checking them (see
// seird_setup_check).  Returns the number of violations; `first` names the first.
int64_t check_setup(const HostSetup& hs, std::string& first) {
  int64_t bad = 0;
  auto fail = [&](bool ok, const std::string& what) {
    if (ok) return;
    if (!bad) first = what;
    ++bad;
  };
  const int64_t n = hs.n;
  const int32_t P = hs.P;
  // partition: owned ranges tile the internal numbering
  fail((int32_t)hs.own_ptr.size() == P + 1 && hs.own_ptr[0] == 0 && hs.own_ptr[P] == n, "owned ranges");
  for (int32_t q = 0; q < P && !bad; ++q) {
    fail(hs.own_ptr[q] <= hs.own_ptr[q + 1], "owned ranges not monotone");
    for (int32_t i = hs.own_ptr[q]; i < hs.own_ptr[q + 1]; ++i) fail(hs.owner[i] == q, "owner map");
  }
  // BSR pattern: sorted rows with their diagonal, structurally symmetric
  const int64_t nnzb = (int64_t)hs.col.size();
  fail((int64_t)hs.row_ptr.size() == n + 1 && hs.row_ptr[n] == nnzb, "row pointers");
  for (int64_t i = 0; i < n && !bad; ++i) {
    bool diag = false;
    for (int32_t k = hs.row_ptr[i]; k < hs.row_ptr[i + 1]; ++k) {
      if (k > hs.row_ptr[i]) fail(hs.col[k] > hs.col[k - 1], "columns not strictly increasing");
      diag |= hs.col[k] == i;
      const int32_t t = hs.tpos[k];
      fail(t >= 0 && t < nnzb && hs.col[t] == i && hs.row_ptr[hs.col[k]] <= t && t < hs.row_ptr[hs.col[k] + 1],
           "transpose map");
    }
    fail(diag, "missing diagonal block");
  }
  // assembly gather lists: each node lists its (triangle, corner) entries and each block
  // its (triangle, corner pair) entries exactly once, ascending in the triangle
  const int64_t m = hs.m;
  fail((int64_t)hs.node_inc.size() == 3 * m && hs.node_inc_ptr[n] == 3 * m, "node gather list sizes");
  for (int64_t i = 0; i < n && !bad; ++i)
    for (int32_t e = hs.node_inc_ptr[i]; e < hs.node_inc_ptr[i + 1]; ++e) {
      fail(hs.tri[hs.node_inc[e]] == i, "node gather entry of another node");
      if (e > hs.node_inc_ptr[i]) fail(hs.node_inc[e] > hs.node_inc[e - 1], "node gather order");
    }
  fail((int64_t)hs.blk_inc.size() == 9 * m && hs.blk_inc_ptr[nnzb] == 9 * m, "block gather list sizes");
  for (int64_t i = 0; i < n && !bad; ++i)
    for (int32_t k = hs.row_ptr[i]; k < hs.row_ptr[i + 1]; ++k)
      for (int32_t e = hs.blk_inc_ptr[k]; e < hs.blk_inc_ptr[k + 1]; ++e) {
        const int32_t v = hs.blk_inc[e], t = v / 9, a = (v % 9) / 3, b = v % 3;
        fail(hs.tri[3 * (int64_t)t + a] == i && hs.tri[3 * (int64_t)t + b] == hs.col[k], "block gather entry");
        if (e > hs.blk_inc_ptr[k]) fail(v > hs.blk_inc[e - 1], "block gather order");
      }
  // coarse space: units tile the nodes; the J Z segments of a row are the runs of its
  // blocks in one unit; the segment sums visit every J block once
  fail((int32_t)hs.cunit_ptr.size() == hs.Pc + 1 && hs.cunit_ptr[0] == 0 && hs.cunit_ptr[hs.Pc] == n, "coarse units");
  for (int32_t u = 0; u < hs.Pc && !bad; ++u)
    for (int32_t i = hs.cunit_ptr[u]; i < hs.cunit_ptr[u + 1]; ++i) fail(hs.cunit[i] == u, "coarse unit map");
  if (!hs.az_ptr.empty()) {
    for (int64_t i = 0; i < n && !bad; ++i)
      for (int64_t s = hs.az_ptr[i]; s < hs.az_ptr[i + 1]; ++s) {
        fail(hs.az_blk[s] >= hs.row_ptr[i] && hs.az_blk[s + 1] <= hs.row_ptr[i + 1] && hs.az_blk[s] < hs.az_blk[s + 1],
             "J Z segment outside its row");
        for (int32_t k = hs.az_blk[s]; k < hs.az_blk[s + 1]; ++k)
          fail(hs.cunit[hs.col[k]] == hs.az_unit[s], "J Z segment mixes coarse units");
      }
  }
  if (!hs.cseg_blk.empty()) {
    std::vector<uint8_t> hit(nnzb, 0);
    for (int32_t k : hs.cseg_blk) fail(k >= 0 && k < nnzb && hit[k]++ == 0, "coarse segment order not a permutation");
  }
  // subdomains: distinct rows covering the owned nodes, local diagonal in place
  const int64_t NL = (int64_t)hs.sd_node.size();
  fail((int32_t)hs.sd_row0.size() == P + 1 && hs.sd_row0[P] == NL, "subdomain row ranges");
  std::vector<int32_t> seen(n, -1);
  for (int32_t q = 0; q < P && !bad; ++q) {
    const int32_t r0 = hs.sd_row0[q], r1 = hs.sd_row0[q + 1];
    for (int32_t R = r0; R < r1; ++R) {
      const int32_t v = hs.sd_node[R];
      fail(v >= 0 && v < n && seen[v] != q, "subdomain rows not distinct");
      if (v >= 0 && v < n) seen[v] = q;
      const int64_t dg = hs.l_diag[R];
      fail(dg >= hs.l_row_ptr[R] && dg < hs.l_row_ptr[R + 1] && hs.l_col[dg] == R - r0, "local diagonal");
    }
    // factor pattern: rows sorted, structurally symmetric (the ILU(k) pattern of a symmetric
    // pattern is symmetric), every block of R_p J R_p^T present and naming its J block, and
    // only fill blocks (allowed with ilu_fill > 0) naming none
    for (int32_t R = r0; R < r1 && !bad; ++R) {
      const int32_t v = hs.sd_node[R];
      std::vector<int32_t> jcols;  // local columns of J's row v inside the subdomain
      for (int32_t k = hs.row_ptr[v]; k < hs.row_ptr[v + 1]; ++k) {
        const int32_t c = hs.col[k];
        if (seen[c] == q) jcols.push_back(c);
      }
      size_t found = 0;
      for (int64_t a = hs.l_row_ptr[R]; a < hs.l_row_ptr[R + 1]; ++a) {
        const int32_t lc = hs.l_col[a];
        fail(lc >= 0 && lc < r1 - r0 && (a == hs.l_row_ptr[R] || hs.l_col[a - 1] < lc), "factor row not sorted");
        if (bad) break;
        const int32_t g = hs.l_gblk[a];
        if (g >= 0) {
          fail(g >= hs.row_ptr[v] && g < hs.row_ptr[v + 1] && hs.col[g] == hs.sd_node[r0 + lc], "factor block names the wrong J block");
          ++found;
        } else {
          fail(hs.ilu_fill > 0, "fill block without ilu_fill");
        }
        // the transposed block (lc, R - r0)
        const int64_t t0 = hs.l_row_ptr[r0 + lc], t1 = hs.l_row_ptr[r0 + lc + 1];
        fail(std::binary_search(hs.l_col.begin() + t0, hs.l_col.begin() + t1, R - r0), "factor pattern not symmetric");
      }
      fail(found == jcols.size(), "a block of R_p J R_p^T is missing from the factor pattern");
    }
    for (int32_t i = hs.own_ptr[q]; i < hs.own_ptr[q + 1]; ++i) fail(seen[i] == q, "owned node outside its subdomain");
  }
  // solve plans: each stage fits the shared-memory rings, every dependency of a row
  // lies in an earlier stage, and the records number the entries by sweep position
  for (int dir = 0; dir < 2 && !bad; ++dir) {
    const HostSetup::SolvePlan& sp = dir == 0 ? hs.sp_fwd : hs.sp_bwd;
    const std::vector<int32_t>& order = dir == 0 ? hs.fwd_order : hs.bwd_order;
    for (int32_t q = 0; q < P && !bad; ++q) {
      const int32_t r0 = hs.sd_row0[q], nl = hs.sd_row0[q + 1] - r0;
      std::vector<int32_t> posf(nl, -1), hit(nl, 0);
      for (int32_t k = 0; k < nl; ++k) {
        const int32_t i = order[r0 + k];
        fail(i >= 0 && i < nl && hit[i]++ == 0, "sweep order is not a permutation");
        if (i >= 0 && i < nl) posf[i] = k;
      }
      const int32_t v0 = sp.sd_lev0[q], v1 = sp.sd_lev0[q + 1] - 1;
      fail(sp.levpos[v0] == 0 && sp.levpos[v1] == nl, "stage positions");
      int32_t owned = 0;
      for (int32_t v = v0; v < v1 && !bad; ++v) {
        const int32_t k0 = sp.levpos[v], k1 = sp.levpos[v + 1];
        const int64_t b0 = sp.levblk[v], nbs = sp.levblk[v + 1] - b0;
        fail(k1 >= k0 && k1 - k0 <= SOLVE_BUF_ROWS && nbs >= 0 && nbs <= SOLVE_BUF_BLOCKS, "stage exceeds the rings");
        for (int32_t k = k0; k < k1; ++k) {
          const int32_t* rec = &sp.info[4 * ((int64_t)r0 + k)];
          const int32_t i = order[r0 + k];
          const int64_t R = (int64_t)r0 + i;
          fail(rec[1] >= 0 && rec[2] >= 0 && rec[1] + rec[2] <= nbs, "row record outside its stage");
          int32_t expect = 0;
          if (dir == 0) {
            for (int64_t a = hs.l_row_ptr[R]; a < hs.l_diag[R]; ++a) ++expect;
            fail(rec[0] == hs.sd_node[R] && rec[3] == 0, "forward record");
          } else {
            expect = 1 + (int32_t)(hs.l_row_ptr[R + 1] - hs.l_diag[R] - 1);
            const int32_t node = hs.sd_node[R];
            const bool own = node >= hs.own_ptr[q] && node < hs.own_ptr[q + 1];
            fail(rec[0] >= 0 && rec[0] < nl && hs.fwd_order[r0 + rec[0]] == i, "backward record: forward position");
            fail(rec[3] == (own ? node : -1), "backward record: owned node");
            owned += own;
            fail(sp.src[b0 + rec[1]] == -1 - R && sp.col[b0 + rec[1]] == k, "backward pivot block");
          }
          fail(rec[2] == expect, "row block count");
          for (int32_t j = dir == 0 ? 0 : 1; j < rec[2]; ++j) {
            const int32_t pos = sp.col[b0 + rec[1] + j];
            fail(pos >= 0 && pos < k0, "dependency not in an earlier stage");
          }
        }
      }
      if (dir == 1) fail(owned == hs.own_ptr[q + 1] - hs.own_ptr[q], "owned rows written once");
    }
  }
  // launch order: every subdomain once (each CTA writes only the nodes its subdomain
  // owns), longest first
  fail((int32_t)hs.sd_sched.size() == P, "launch order size");
  if (!bad) {
    std::vector<int32_t> hit(P, 0);
    for (int32_t b = 0; b < P; ++b) {
      const int32_t q = hs.sd_sched[b];
      fail(q >= 0 && q < P && hit[q]++ == 0, "launch order is not a permutation");
      if (!bad && b > 0) fail(solve_work(hs, hs.sd_sched[b - 1]) >= solve_work(hs, q), "launch order not longest first");
    }
  }
  return bad;
}

}  // namespace seird

extern "C" int seird_setup_check(const seird_mesh* mesh, const seird_options* opt, int64_t* stats) {
  using namespace seird;
  seird_options o;
  if (opt) o = *opt;
  else seird_default_options(&o);
  HostSetup hs;
  std::string err;
  int64_t bad = 0;
  try {  // host exceptions (a failed allocation) end as an error code, as in every other entry point
    const int rc = build_setup(mesh, &o, hs, err);
    if (rc) {
      set_global_error(err);
      return rc;
    }
    bad = check_setup(hs, err);
  } catch (const std::exception& e) {
    const bool nomem = dynamic_cast<const std::bad_alloc*>(&e) || dynamic_cast<const std::length_error*>(&e);
    set_global_error(nomem ? "host allocation failed" : e.what());
    return nomem ? SEIRD_ENOMEM : SEIRD_EINVAL;
  }
  if (stats) {
    stats[0] = hs.n;
    stats[1] = hs.m;
    stats[2] = (int64_t)hs.col.size();
    stats[3] = hs.P;
    stats[4] = (int64_t)hs.sd_node.size();
    stats[5] = (int64_t)hs.sp_fwd.levpos.size() - hs.P;  // stages (each subdomain adds one boundary entry)
    stats[6] = (int64_t)hs.sp_bwd.levpos.size() - hs.P;
    stats[7] = bad;
  }
  if (bad) set_global_error("setup check: " + std::to_string(bad) + " violations, first: " + err);
  return bad ? SEIRD_EINVAL : SEIRD_OK;
}

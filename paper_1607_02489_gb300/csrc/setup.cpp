// Host setup of the EMIN-AMG hierarchy (Alg. 1 with Alg. 2-4 and Section 4.3).
//
// Built with -ffp-contract=off: the integer decisions taken from floating
// point (filtering, the packing heuristic, the mid-point test) must not
// depend on whether the compiler fuses a multiply and an add.
#include "setup.hpp"
#include "trace.hpp"

#include <algorithm>
#include <cmath>
#include <deque>
#include <limits>
#include <stdexcept>
#include <string>
#include <thread>

namespace emin {
namespace {

enum : signed char { UNMARKED = 0, CPT = 1, FPT = 2, EXCL = 3 };

struct Graph {
  int n = 0;
  std::vector<int64_t> ptr;
  std::vector<int> adj;  // ascending neighbours, no self loops
  int64_t begin(int v) const { return ptr[v]; }
  int64_t end(int v) const { return ptr[v + 1]; }
};

// eq. e:filtering: drop |z_ij| <= tau sqrt(|z_ii z_jj|), i != j, and add the
// dropped values to the diagonal (row sums kept).  The graph is the kept
// off-diagonal pattern, symmetrised by union.
void filter_lump(const Csr& Z, double tau, Csr& F, Graph& G) {
  const int n = Z.nrows;
  std::vector<double> d(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int64_t t = Z.row_begin(i); t < Z.row_end(i); ++t)
      if (Z.col[t] == i) d[i] = d[i] + Z.val[t];
  F.resize_rows(n, n);
  std::vector<std::vector<int>> nb(n);
  for (int i = 0; i < n; ++i) {
    double lump = 0.0;
    std::vector<std::pair<int, double>> kept;
    for (int64_t t = Z.row_begin(i); t < Z.row_end(i); ++t) {
      const int j = Z.col[t];
      if (j == i) continue;
      const double v = Z.val[t];
      const double thr = tau * std::sqrt(std::fabs(d[i] * d[j]));
      if (std::fabs(v) <= thr) {
        lump = lump + v;
      } else {
        kept.push_back({j, v});
        nb[i].push_back(j);
        nb[j].push_back(i);
      }
    }
    kept.push_back({i, d[i] + lump});
    std::sort(kept.begin(), kept.end());
    for (auto& kv : kept) {
      F.col.push_back(kv.first);
      F.val.push_back(kv.second);
    }
    F.rowptr[i + 1] = (int64_t)F.col.size();
  }
  G.n = n;
  G.ptr.assign(n + 1, 0);
  G.adj.clear();
  for (int i = 0; i < n; ++i) {
    auto& v = nb[i];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    G.adj.insert(G.adj.end(), v.begin(), v.end());
    G.ptr[i + 1] = (int64_t)G.adj.size();
  }
}

// Breadth-first search to distance maxd; `stamp` marks visited vertices.
struct Bfs {
  std::vector<int> stamp, dist;
  int epoch = 0;
  std::vector<int> out;  // visited vertices in BFS order
  explicit Bfs(int n) : stamp(n, -1), dist(n, 0) {}
  void run(const Graph& G, int src, int maxd) {
    ++epoch;
    out.clear();
    stamp[src] = epoch;
    dist[src] = 0;
    out.push_back(src);
    for (size_t h = 0; h < out.size(); ++h) {
      const int v = out[h];
      if (dist[v] == maxd) continue;
      for (int64_t t = G.begin(v); t < G.end(v); ++t) {
        const int w = G.adj[t];
        if (stamp[w] != epoch) {
          stamp[w] = epoch;
          dist[w] = dist[v] + 1;
          out.push_back(w);
        }
      }
    }
  }
};

double sqdist(const double* x, const double* y, int dim) {
  double s = 0.0;
  for (int k = 0; k < dim; ++k) {
    const double t = x[k] - y[k];
    s = s + t * t;
  }
  return s;
}

double seg_sqdist(const double* x, const double* a, const double* b, int dim) {
  double ab[3], ax[3];
  double L2 = 0.0, dot = 0.0;
  for (int k = 0; k < dim; ++k) {
    ab[k] = b[k] - a[k];
    ax[k] = x[k] - a[k];
  }
  for (int k = 0; k < dim; ++k) {
    L2 = L2 + ab[k] * ab[k];
    dot = dot + ax[k] * ab[k];
  }
  double t = L2 > 0.0 ? dot / L2 : 0.0;
  t = std::min(std::max(t, 0.0), 1.0);
  double s = 0.0;
  for (int k = 0; k < dim; ++k) {
    const double e = ax[k] - t * ab[k];
    s = s + e * e;
  }
  return s;
}

struct CoarsePressures {
  std::vector<signed char> state;
  std::vector<std::vector<std::pair<int, int>>> S;  // (C-point, graph distance <= 3)
};

// Alg. 3 main loop (find_coarse_pressures) with update_heuristics taken as the
// smallest Euclidean distance to a C-point within graph distance 4; the next
// C-point is the lowest-index candidate whose squared distance is within a
// relative 1e-9 of the smallest one, or the lowest-index unmarked vertex.
CoarsePressures find_coarse_pressures(const Graph& G, const double* X, int dim, int excluded) {
  const int n = G.n;
  CoarsePressures cp;
  cp.state.assign(n, UNMARKED);
  cp.S.assign(n, {});
  if (excluded >= 0) cp.state[excluded] = EXCL;
  std::vector<double> h1sq(n, std::numeric_limits<double>::infinity());
  std::vector<char> in_cand(n, 0);
  std::vector<int> cand;
  Bfs bfs(n);
  int next_unmarked = 0;
  auto lowest_unmarked = [&]() {
    while (next_unmarked < n && cp.state[next_unmarked] != UNMARKED) ++next_unmarked;
    return next_unmarked < n ? next_unmarked : -1;
  };
  int k = lowest_unmarked();
  while (k >= 0) {
    bfs.run(G, k, 4);
    for (int j : bfs.out)
      if (bfs.dist[j] <= 3) cp.S[j].push_back({k, bfs.dist[j]});
    cp.state[k] = CPT;
    for (int j : bfs.out)
      if (bfs.dist[j] <= 3 && j != k && cp.state[j] == UNMARKED) cp.state[j] = FPT;
    for (int j : bfs.out)
      if (bfs.dist[j] == 4 && !in_cand[j]) {
        in_cand[j] = 1;
        cand.push_back(j);
      }
    size_t w = 0;
    for (size_t t = 0; t < cand.size(); ++t) {
      if (cp.state[cand[t]] == UNMARKED)
        cand[w++] = cand[t];
      else
        in_cand[cand[t]] = 0;
    }
    cand.resize(w);
    for (int j : bfs.out)
      if (j != k) h1sq[j] = std::min(h1sq[j], sqdist(X + (size_t)j * dim, X + (size_t)k * dim, dim));
    if (!cand.empty()) {
      double m = std::numeric_limits<double>::infinity();
      for (int j : cand) m = std::min(m, h1sq[j]);
      const double lim = m * (1.0 + 1e-9);
      int best = -1;
      for (int j : cand)
        if (h1sq[j] <= lim && (best < 0 || j < best)) best = j;
      k = best;
    } else {
      k = lowest_unmarked();
    }
  }
  return cp;
}

// find_extra_dist3_Cpoints: in index order convert F-points with |S_j| = 1 at
// graph distance 3, or |S_j| = 2 at distance 3 from both C-points and farther
// than a quarter of their separation from the segment joining them.
std::vector<int> find_extra_dist3_cpoints(const Graph& G, const double* X, int dim, CoarsePressures& cp) {
  std::vector<int> added;
  Bfs bfs(G.n);
  for (int j = 0; j < G.n; ++j) {
    if (cp.state[j] != FPT) continue;
    auto s = cp.S[j];
    std::sort(s.begin(), s.end());
    bool convert = false;
    if (s.size() == 1) {
      convert = s[0].second == 3;
    } else if (s.size() == 2) {
      const int a = s[0].first, b = s[1].first;
      if (s[0].second == 3 && s[1].second == 3) {
        const double L2 = sqdist(X + (size_t)a * dim, X + (size_t)b * dim, dim);
        convert = seg_sqdist(X + (size_t)j * dim, X + (size_t)a * dim, X + (size_t)b * dim, dim) > 0.0625 * L2;
      }
    }
    if (convert) {
      cp.state[j] = CPT;
      added.push_back(j);
      bfs.run(G, j, 3);
      for (int v : bfs.out) cp.S[v].push_back({j, bfs.dist[v]});
    }
  }
  return added;
}

std::vector<int> sorted_keys(const std::vector<std::pair<int, int>>& s) {
  std::vector<int> k;
  k.reserve(s.size());
  for (auto& e : s) k.push_back(e.first);
  std::sort(k.begin(), k.end());
  return k;
}

// Alg. 4 (find_velocity_Cpoints): pressure mid-points, processed by descending
// |S_i| then index; t_i^2 is the squared diagonal of B_i's bounding box and the
// test is min squared distance >= tau2^2 t_i^2 (+inf when B_i has no C-bar point).
std::vector<char> find_velocity_cpoints(const CoarsePressures& cp, const double* X, int dim, double tau2sq) {
  const int n = (int)cp.state.size();
  std::vector<int> F;
  for (int i = 0; i < n; ++i)
    if (cp.state[i] == FPT) F.push_back(i);
  std::vector<std::vector<int>> keys(n);
  std::vector<std::vector<int>> users(n);
  for (int j : F) {
    keys[j] = sorted_keys(cp.S[j]);
    for (int c : keys[j]) users[c].push_back(j);
  }
  std::vector<char> Cbar(n, 0);
  for (int i = 0; i < n; ++i)
    if (cp.state[i] == CPT) Cbar[i] = 1;
  std::vector<int> order = F;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (keys[a].size() != keys[b].size()) return keys[a].size() > keys[b].size();
    return a < b;
  });
  std::vector<int> Bi;
  for (int i : order) {
    const auto& s = keys[i];
    double Xi[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
      double acc = 0.0;
      for (int c : s) acc = acc + X[(size_t)c * dim + k];
      Xi[k] = acc / (double)s.size();
    }
    Bi.clear();
    for (int j : users[s[0]]) {
      if (cp.state[j] != FPT) continue;
      const auto& kj = keys[j];
      if (std::includes(kj.begin(), kj.end(), s.begin(), s.end())) Bi.push_back(j);
    }
    std::sort(Bi.begin(), Bi.end());
    double t2 = 0.0;
    for (int k = 0; k < dim; ++k) {
      double mx = -std::numeric_limits<double>::infinity(), mn = std::numeric_limits<double>::infinity();
      for (int j : Bi) {
        mx = std::max(mx, X[(size_t)j * dim + k]);
        mn = std::min(mn, X[(size_t)j * dim + k]);
      }
      const double e = mx - mn;
      t2 = t2 + e * e;
    }
    int m = -1;
    double best = 0.0;
    for (int j : Bi) {
      const double dj = sqdist(X + (size_t)j * dim, Xi, dim);
      if (m < 0 || dj < best) {
        best = dj;
        m = j;
      }
    }
    double dmin = std::numeric_limits<double>::infinity();
    for (int j : Bi)
      if (Cbar[j]) dmin = std::min(dmin, sqdist(X + (size_t)j * dim, X + (size_t)m * dim, dim));
    if (dmin >= tau2sq * t2) Cbar[m] = 1;
  }
  return Cbar;
}

// Velocity pattern: C^(v) nodes within distance 3 in the filtered velocity
// graph; extra C-points for non-Dirichlet nodes left without one (index order);
// C rows injection, Dirichlet rows empty.  Returns rows of coarse indices.
std::vector<std::vector<int>> velocity_pattern(const Graph& G, std::vector<char>& isC,
                                               const std::vector<unsigned char>& dirichlet,
                                               std::vector<int>& Cv) {
  const int n = G.n;
  std::vector<std::vector<int>> rows(n);
  Bfs bfs(n);
  for (int c = 0; c < n; ++c) {
    if (!isC[c]) continue;
    bfs.run(G, c, 3);
    for (int v : bfs.out) rows[v].push_back(c);
  }
  for (int i = 0; i < n; ++i) {
    if (dirichlet[i] || isC[i] || !rows[i].empty()) continue;
    isC[i] = 1;
    bfs.run(G, i, 3);
    for (int v : bfs.out) rows[v].push_back(i);
  }
  Cv.clear();
  std::vector<int> cidx(n, -1);
  for (int i = 0; i < n; ++i)
    if (isC[i]) {
      cidx[i] = (int)Cv.size();
      Cv.push_back(i);
    }
  std::vector<std::vector<int>> out(n);
  for (int i = 0; i < n; ++i) {
    if (dirichlet[i]) continue;
    if (isC[i]) {
      out[i] = {cidx[i]};
      continue;
    }
    for (int c : rows[i]) out[i].push_back(cidx[c]);
    std::sort(out[i].begin(), out[i].end());
    out[i].erase(std::unique(out[i].begin(), out[i].end()), out[i].end());
  }
  return out;
}

Csr pattern_csr(const std::vector<std::vector<int>>& rows, int ncols) {
  Csr N;
  N.resize_rows((int)rows.size(), ncols);
  for (size_t i = 0; i < rows.size(); ++i) {
    for (int c : rows[i]) {
      N.col.push_back(c);
      N.val.push_back(1.0);
    }
    N.rowptr[i + 1] = (int64_t)N.col.size();
  }
  return N;
}

// Orthogonal projection onto {pattern of N, zero row sums}: G sampled on the
// pattern minus each row's mean over the pattern.
Csr project(const Csr& G, const Csr& N) {
  Csr Q = N;
  for (int i = 0; i < N.nrows; ++i) {
    const int64_t b = N.row_begin(i), e = N.row_end(i);
    if (b == e) continue;
    double sum = 0.0;
    int64_t g = G.row_begin(i);
    for (int64_t t = b; t < e; ++t) {
      while (g < G.row_end(i) && G.col[g] < N.col[t]) ++g;
      Q.val[t] = (g < G.row_end(i) && G.col[g] == N.col[t]) ? G.val[g] : 0.0;
      sum = sum + Q.val[t];
    }
    const double mean = sum / (double)(e - b);
    for (int64_t t = b; t < e; ++t) Q.val[t] = Q.val[t] - mean;
  }
  return Q;
}

// One EMIN step (eq. min_problem): P0 = pattern / row count,
// R0 = -Proj(At P0); CG: alpha = <R0,R0> / <R0, At R0>; GMRES: Q = Proj(At R0),
// alpha = <R0,Q> / <Q,Q>; P = P0 + alpha R0 on the pattern.
Csr emin_step(const Csr& At, const std::vector<std::vector<int>>& rows, int ncols, bool cg) {
  Csr P = pattern_csr(rows, ncols);
  for (int i = 0; i < P.nrows; ++i) {
    const int64_t cnt = P.row_end(i) - P.row_begin(i);
    for (int64_t t = P.row_begin(i); t < P.row_end(i); ++t) P.val[t] = 1.0 / (double)cnt;
  }
  Csr R0 = project(spgemm(At, P), P);
  for (auto& v : R0.val) v = -v;
  double num = 0.0, den = 0.0;
  if (cg) {
    for (double v : R0.val) num += v * v;
    Csr AR = spgemm(At, R0);
    for (int i = 0; i < R0.nrows; ++i)
      for (int64_t t = R0.row_begin(i); t < R0.row_end(i); ++t) den += R0.val[t] * lookup(AR, i, R0.col[t]);
  } else {
    Csr Q = project(spgemm(At, R0), P);
    for (size_t t = 0; t < R0.val.size(); ++t) {
      num += R0.val[t] * Q.val[t];
      den += Q.val[t] * Q.val[t];
    }
  }
  const double alpha = den != 0.0 ? num / den : 0.0;
  for (size_t t = 0; t < P.val.size(); ++t) P.val[t] = P.val[t] + alpha * R0.val[t];
  return P;
}

// Braess-Sarazin data (Section 5.2): D = |A| row sums (Dirichlet rows 1/c), the
// explicit Schur complement S = B D^-1 Bt (pinned row = identity), the strip
// length of the Gauss-Seidel ordering and a greedy coloring of each strip's
// subgraph of S's graph (vertices in index order, smallest free color).
void form_relaxation(HostLevel& L, const SetupParams& prm) {
  L.D.assign(L.n_v, 0.0);
  for (int i = 0; i < L.n_v; ++i) {
    double s = 0.0;
    for (int64_t t = L.A.row_begin(i); t < L.A.row_end(i); ++t) s += std::fabs(L.A.val[t]);
    L.D[i] = L.dirichlet[i] ? 1.0 / prm.c : s;
  }
  Csr BD = L.B;
  for (int64_t t = 0; t < BD.nnz(); ++t) BD.val[t] = BD.val[t] * (1.0 / L.D[BD.col[t] % L.n_v]);
  L.S = spgemm(BD, L.Bt);
  if (L.pinned >= 0) {
    Csr S2;
    S2.resize_rows(L.S.nrows, L.S.ncols);
    for (int i = 0; i < L.S.nrows; ++i) {
      bool done = false;
      for (int64_t t = L.S.row_begin(i); t < L.S.row_end(i); ++t) {
        const int j = L.S.col[t];
        if (i == L.pinned && !done && j > i) {
          S2.col.push_back(i);
          S2.val.push_back(1.0);
          done = true;
        }
        S2.col.push_back(j);
        S2.val.push_back((i == L.pinned && j == i) ? 1.0 : L.S.val[t]);
        if (i == L.pinned && j == i) done = true;
      }
      if (i == L.pinned && !done) {
        S2.col.push_back(i);
        S2.val.push_back(1.0);
      }
      S2.rowptr[i + 1] = (int64_t)S2.col.size();
    }
    L.S = std::move(S2);
  }
  // Gauss-Seidel ordering: strips of T consecutive rows, T the smallest length
  // >= bandwidth/2 for which every entry couples the same or adjacent strips (so
  // strips two apart never interact); rows go by (strip parity, color, index)
  int bw = 0;
  for (int i = 0; i < L.n_p; ++i)
    for (int64_t t = L.S.row_begin(i); t < L.S.row_end(i); ++t)
      if (L.S.col[t] != i) bw = std::max(bw, std::abs(L.S.col[t] - i));
  L.gs_strip = std::max(bw, 1);
  for (int T = std::max(1, (bw + 1) / 2); T < bw; ++T) {
    bool ok = true;
    for (int i = 0; i < L.n_p && ok; ++i)
      for (int64_t t = L.S.row_begin(i); t < L.S.row_end(i); ++t) {
        const int j = L.S.col[t];
        if (j != i && std::abs(j / T - i / T) > 1) {
          ok = false;
          break;
        }
      }
    if (ok) {
      L.gs_strip = T;
      break;
    }
  }
  // greedy coloring of each strip's own subgraph (index order, smallest free color)
  L.colors.assign(L.n_p, -1);
  L.n_colors = 0;
  std::vector<int> used_stamp(64, -1);
  for (int i = 0; i < L.n_p; ++i) {
    for (int64_t t = L.S.row_begin(i); t < L.S.row_end(i); ++t) {
      const int j = L.S.col[t];
      if (j != i && j / L.gs_strip == i / L.gs_strip && L.colors[j] >= 0) {
        if (L.colors[j] >= (int)used_stamp.size()) used_stamp.resize(2 * L.colors[j] + 2, -1);
        used_stamp[L.colors[j]] = i;
      }
    }
    int c = 0;
    while (c < (int)used_stamp.size() && used_stamp[c] == i) ++c;
    if (c >= (int)used_stamp.size()) used_stamp.resize(2 * c + 2, -1);
    L.colors[i] = c;
    L.n_colors = std::max(L.n_colors, c + 1);
  }
}

// Dense block matrix of a level, row-major N x N.
std::vector<double> dense_level(const HostLevel& L) {
  const int N = L.N(), nu = L.dim * L.n_v;
  std::vector<double> M((size_t)N * N, 0.0);
  for (int c = 0; c < L.dim; ++c)
    for (int i = 0; i < L.n_v; ++i)
      for (int64_t t = L.A.row_begin(i); t < L.A.row_end(i); ++t)
        M[(size_t)(c * L.n_v + i) * N + c * L.n_v + L.A.col[t]] += L.A.val[t];
  for (int r = 0; r < nu; ++r)
    for (int64_t t = L.Bt.row_begin(r); t < L.Bt.row_end(r); ++t) M[(size_t)r * N + nu + L.Bt.col[t]] += L.Bt.val[t];
  for (int k = 0; k < L.n_p; ++k)
    for (int64_t t = L.B.row_begin(k); t < L.B.row_end(k); ++t) M[(size_t)(nu + k) * N + L.B.col[t]] += L.B.val[t];
  if (L.pinned >= 0) M[(size_t)(nu + L.pinned) * N + nu + L.pinned] += 1.0;
  return M;
}

// Pseudo-inverse by the one-sided Jacobi SVD (Hestenes 1958): rotate column
// pairs of M until they are orthogonal; then M = U S V^T with the column norms
// as singular values; singular values below rcond * max are dropped.
std::vector<double> pseudo_inverse(const std::vector<double>& M, int n, double rcond) {
  std::vector<double> U((size_t)n * n), V((size_t)n * n, 0.0);  // column j at [j*n, j*n+n)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) U[(size_t)j * n + i] = M[(size_t)i * n + j];
  for (int j = 0; j < n; ++j) V[(size_t)j * n + j] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double* up = &U[(size_t)p * n];
        double* uq = &U[(size_t)q * n];
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = 0; i < n; ++i) {
          a += up[i] * up[i];
          b += uq[i] * uq[i];
          g += up[i] * uq[i];
        }
        if (a == 0.0 || b == 0.0) continue;
        const double rel = std::fabs(g) / std::sqrt(a * b);
        if (rel <= 1e-15) continue;
        off = std::max(off, rel);
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        double* vp = &V[(size_t)p * n];
        double* vq = &V[(size_t)q * n];
        for (int i = 0; i < n; ++i) {
          const double x = up[i], y = uq[i];
          up[i] = c * x - s * y;
          uq[i] = s * x + c * y;
          const double xv = vp[i], yv = vq[i];
          vp[i] = c * xv - s * yv;
          vq[i] = s * xv + c * yv;
        }
      }
    if (off <= 1e-15) break;
  }
  std::vector<double> s(n);
  double smax = 0.0;
  for (int j = 0; j < n; ++j) {
    double a = 0.0;
    for (int i = 0; i < n; ++i) a += U[(size_t)j * n + i] * U[(size_t)j * n + i];
    s[j] = std::sqrt(a);
    smax = std::max(smax, s[j]);
  }
  std::vector<double> Pinv((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    if (!(s[j] > rcond * smax)) continue;
    const double inv2 = 1.0 / (s[j] * s[j]);
    const double* u = &U[(size_t)j * n];
    const double* v = &V[(size_t)j * n];
    for (int i = 0; i < n; ++i) {
      const double vi = v[i] * inv2;
      double* row = &Pinv[(size_t)i * n];
      for (int k = 0; k < n; ++k) row[k] += vi * u[k];
    }
  }
  return Pinv;
}

// Refinement of a pseudo-inverse X of the dense n x n matrix M (Newton-Schulz
// step X <- X + X (I - M X), twice): the residual I - M X is formed with
// compensated dot products (the sum and the products carried as value + error
// term, Ogita, Rump and Oishi 2005), so it is accurate to about twice the
// working precision, and each step removes the part of X's error that an SVD
// leaves in the directions of small singular values (about cond(M) times the
// unit roundoff).  The refined X agrees with the exact pseudo-inverse to a few
// units of roundoff of ||X||.  Directions dropped from X stay dropped: X R lies
// in X's row space.  Rows of the residual are split over the host's threads.
// Coarsest levels above kRefineMaxDofs (only reached when max_coarse or
// max_levels stop coarsening early) keep the SVD's X.
constexpr int kRefineMaxDofs = 512;
void refine_pseudo_inverse(const std::vector<double>& M, std::vector<double>& X, int n) {
  if (n > kRefineMaxDofs) return;
  std::vector<double> R((size_t)n * n), Y((size_t)n * n);
  auto residual_rows = [&](int i0, int i1) {
    for (int i = i0; i < i1; ++i)
      for (int j = 0; j < n; ++j) {
        double s = i == j ? 1.0 : 0.0, c = 0.0;  // s + c carries the running sum
        for (int k = 0; k < n; ++k) {
          const double a = -M[(size_t)i * n + k], b = X[(size_t)k * n + j];
          const double p = a * b;
          const double pe = std::fma(a, b, -p);  // exact error of the product
          const double t = s + p;
          const double bb = t - s;
          const double se = (s - (t - bb)) + (p - bb);  // exact error of the sum
          s = t;
          c = c + (se + pe);
        }
        R[(size_t)i * n + j] = s + c;
      }
  };
  auto update_rows = [&](int i0, int i1) {
    for (int i = i0; i < i1; ++i)
      for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = acc + X[(size_t)i * n + k] * R[(size_t)k * n + j];
        Y[(size_t)i * n + j] = X[(size_t)i * n + j] + acc;
      }
  };
  const int nt = std::max(1, std::min<int>({(int)std::thread::hardware_concurrency(), 16, (n + 31) / 32}));
  auto parallel = [&](auto&& f) {
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(f, (int)((int64_t)n * t / nt), (int)((int64_t)n * (t + 1) / nt));
    for (auto& th : pool) th.join();
  };
  for (int step = 0; step < 2; ++step) {
    parallel(residual_rows);
    parallel(update_rows);
    X.swap(Y);
  }
}

// Alg. 2 + form_restriction + the Petrov-Galerkin product; false when the
// coarsening makes no progress.
void finish_interpolation(HostLevel& L, HostLevel& Lc, const SetupParams& prm, const Csr& Ap, const Csr& Av,
                          const std::vector<std::vector<int>>& rows_p, const std::vector<std::vector<int>>& rows_v);

bool form_interpolation(HostLevel& L, HostLevel& Lc, const SetupParams& prm) {
  const int d = L.dim;
  trace_push("graph phase: filtering, Alg. 3, Alg. 4, patterns");
  // form_aux_block_diagonal
  Csr Zp = spgemm(L.B, transpose(L.B));
  Csr Ap, Av;
  Graph Gp, Gv;
  filter_lump(Zp, prm.tau1_for(L.dim), Ap, Gp);
  filter_lump(L.A, prm.tau1_for(L.dim), Av, Gv);
  // Alg. 3
  CoarsePressures cp = find_coarse_pressures(Gp, L.pX.data(), d, L.pinned);
  find_extra_dist3_cpoints(Gp, L.pX.data(), d, cp);
  L.Cp.clear();
  std::vector<int> cidx(L.n_p, -1);
  for (int i = 0; i < L.n_p; ++i)
    if (cp.state[i] == CPT) {
      cidx[i] = (int)L.Cp.size();
      L.Cp.push_back(i);
    }
  if ((int)L.Cp.size() >= L.n_p) {
    trace_pop();
    return false;
  }
  // pressure pattern: S_i for F-points, injection for C-points, empty if excluded
  std::vector<std::vector<int>> rows_p(L.n_p);
  for (int i = 0; i < L.n_p; ++i) {
    if (cp.state[i] == CPT) {
      rows_p[i] = {cidx[i]};
    } else if (cp.state[i] == FPT) {
      for (auto& e : cp.S[i]) rows_p[i].push_back(cidx[e.first]);
      std::sort(rows_p[i].begin(), rows_p[i].end());
    }
  }
  // Alg. 4 and co-located velocities
  std::vector<char> Cbar = find_velocity_cpoints(cp, L.pX.data(), d, prm.tau2sq);
  std::vector<char> isCv(L.n_v, 0);
  for (int k = 0; k < L.n_p; ++k)
    if (Cbar[k]) {
      const int v = L.p2v[k];
      if (v >= 0 && !L.dirichlet[v]) isCv[v] = 1;
    }
  std::vector<std::vector<int>> rows_v = velocity_pattern(Gv, isCv, L.dirichlet, L.Cv);
  trace_pop();
  finish_interpolation(L, Lc, prm, Ap, Av, rows_p, rows_v);
  return true;
}

// The coarse points and sparsity patterns of a previous hierarchy's level (same
// matrix structure), with EMIN and the Petrov-Galerkin product redone on this
// level's values: the graph phase is done once per nonlinear sequence (Section
// 6.1), the rest per matrix.
void form_interpolation_reuse(HostLevel& L, HostLevel& Lc, const SetupParams& prm, const HostLevel& prev) {
  if (prev.Pp.nrows != L.n_p || prev.P.nrows != L.n_v || prev.dim != L.dim)
    throw std::runtime_error("reused hierarchy does not match the problem's structure");
  Csr Zp = spgemm(L.B, transpose(L.B));
  Csr Ap, Av;
  Graph Gp, Gv;
  filter_lump(Zp, prm.tau1_for(L.dim), Ap, Gp);
  filter_lump(L.A, prm.tau1_for(L.dim), Av, Gv);
  L.Cp = prev.Cp;
  L.Cv = prev.Cv;
  auto rows_of = [](const Csr& M) {
    std::vector<std::vector<int>> rows(M.nrows);
    for (int i = 0; i < M.nrows; ++i) rows[i].assign(M.col.begin() + M.row_begin(i), M.col.begin() + M.row_end(i));
    return rows;
  };
  finish_interpolation(L, Lc, prm, Ap, Av, rows_of(prev.Pp), rows_of(prev.P));
}

// EMIN on the patterns, restriction and the Petrov-Galerkin product (Alg. 1-2,
// Section 4.3), given the filtered matrices, the coarse points (L.Cp, L.Cv) and
// the patterns.
void finish_interpolation(HostLevel& L, HostLevel& Lc, const SetupParams& prm, const Csr& Ap, const Csr& Av,
                          const std::vector<std::vector<int>>& rows_p, const std::vector<std::vector<int>>& rows_v) {
  TraceRange range("EMIN steps, restriction, Galerkin products");
  const int d = L.dim;
  const bool cg = prm.symmetric;
  L.Pp = emin_step(Ap, rows_p, (int)L.Cp.size(), cg);
  L.P = emin_step(Av, rows_v, (int)L.Cv.size(), cg);
  // form_restriction (Section 4.3)
  if (cg) {
    L.R = transpose(L.P);
    L.Rp = transpose(L.Pp);
  } else {
    L.R = transpose(emin_step(transpose(Av), rows_v, (int)L.Cv.size(), false));
    L.Rp = transpose(emin_step(transpose(Ap), rows_p, (int)L.Cp.size(), false));
  }
  // Petrov-Galerkin product A_{l+1} = R A P, block by block
  Csr Pv = kron_identity(d, L.P), Rv = kron_identity(d, L.R);
  Lc.dim = d;
  Lc.n_v = (int)L.Cv.size();
  Lc.n_p = (int)L.Cp.size();
  Lc.pinned = -1;
  Lc.A = spgemm(spgemm(L.R, L.A), L.P);
  Lc.B = spgemm(spgemm(L.Rp, L.B), Pv);
  Lc.Bt = spgemm(spgemm(Rv, L.Bt), L.Pp);
  // project_coordinates: injection; co-location restricted to the coarse points
  Lc.vX.resize((size_t)Lc.n_v * d);
  Lc.pX.resize((size_t)Lc.n_p * d);
  for (int t = 0; t < Lc.n_v; ++t)
    for (int k = 0; k < d; ++k) Lc.vX[(size_t)t * d + k] = L.vX[(size_t)L.Cv[t] * d + k];
  for (int t = 0; t < Lc.n_p; ++t)
    for (int k = 0; k < d; ++k) Lc.pX[(size_t)t * d + k] = L.pX[(size_t)L.Cp[t] * d + k];
  std::vector<int> vpos(L.n_v, -1);
  for (int t = 0; t < Lc.n_v; ++t) vpos[L.Cv[t]] = t;
  Lc.p2v.resize(Lc.n_p);
  for (int t = 0; t < Lc.n_p; ++t) {
    const int v = L.p2v[L.Cp[t]];
    Lc.p2v[t] = v >= 0 ? vpos[v] : -1;
  }
  Lc.dirichlet.assign(Lc.n_v, 0);
}


// ---------------------------------------------------------------------------
// Dense form of a small level's Gauss-Seidel call: the iterations from dp = 0 are
// the linear map dp = M g.  Rows are relaxed in the order (strip parity, color,
// index); row i of M becomes (e_i - sum_{j != i} S_ij M_j) / S_ii when row i is
// relaxed.  The columns of M are independent, so host threads split them.
void form_dense_gs(HostLevel& L, int iters) {
  const int n = L.n_p, T = L.gs_strip, ncol = L.n_colors;
  const int nstrips = std::max(1, (n + T - 1) / T);
  std::vector<int> order;  // rows in relaxation order for one iteration
  order.reserve(n);
  for (int par = 0; par < 2; ++par)
    for (int c = 0; c < ncol; ++c)
      for (int st = par; st < nstrips; st += 2)
        for (int i = st * T; i < std::min(n, (st + 1) * T); ++i)
          if (L.colors[i] == c) order.push_back(i);
  L.gs_dense.assign((size_t)n * n, 0.0);
  double* M = L.gs_dense.data();
  auto work = [&](int q0, int q1) {
    std::vector<double> row(q1 - q0);
    for (int it = 0; it < iters; ++it)
      for (int i : order) {
        double diag = 0.0;
        std::fill(row.begin(), row.end(), 0.0);
        if (i >= q0 && i < q1) row[i - q0] = 1.0;
        for (int64_t t = L.S.row_begin(i); t < L.S.row_end(i); ++t) {
          const int j = L.S.col[t];
          if (j == i) {
            diag += L.S.val[t];
            continue;
          }
          const double v = L.S.val[t];
          const double* Mj = M + (size_t)j * n + q0;
          for (int q = 0; q < q1 - q0; ++q) row[q] -= v * Mj[q];
        }
        const double dinv = diag != 0.0 ? 1.0 / diag : 0.0;
        double* Mi = M + (size_t)i * n + q0;
        for (int q = 0; q < q1 - q0; ++q) Mi[q] = row[q] * dinv;
      }
  };
  const int nt = std::max(1, std::min<int>({(int)std::thread::hardware_concurrency(), 16, (n + 63) / 64}));
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(work, (int)((int64_t)n * t / nt), (int)((int64_t)n * (t + 1) / nt));
  for (auto& th : pool) th.join();
}

// ---------------------------------------------------------------------------
// Vanka blocks (Section 5.1): block i = the columns of row i of B plus pressure i;
// a non-Dirichlet dof in no block is a block of its own; Dirichlet velocity dofs
// (zero columns of B, identity rows of A) are relaxed exactly instead.  Order of
// relaxation: (color, index), a greedy coloring (index order, smallest free
// color) of the graph in which two blocks are adjacent when a row of the block
// matrix in one has an entry in a column of the other (or they share a dof).

// Columns and values of row q of the block matrix [I_d (x) A, Bt; B, C].
template <typename F>
void block_matrix_row(const HostLevel& L, int q, F&& f) {
  const int nu = L.dim * L.n_v;
  if (q < nu) {
    const int c = q / L.n_v, i = q % L.n_v;
    for (int64_t t = L.A.row_begin(i); t < L.A.row_end(i); ++t) f(c * L.n_v + L.A.col[t], L.A.val[t]);
    for (int64_t t = L.Bt.row_begin(q); t < L.Bt.row_end(q); ++t) f(nu + L.Bt.col[t], L.Bt.val[t]);
  } else {
    const int i = q - nu;
    for (int64_t t = L.B.row_begin(i); t < L.B.row_end(i); ++t) f(L.B.col[t], L.B.val[t]);
    if (i == L.pinned) f(q, 1.0);
  }
}

// In-place inverse of a dense n x n row-major matrix by Gauss-Jordan elimination
// with partial pivoting; false if the matrix is numerically singular: a pivot at
// most n * eps times the largest entry of the matrix.
bool invert_dense(std::vector<double>& a, int n) {
  double amax = 0.0;
  for (double v : a) amax = std::max(amax, std::fabs(v));
  const double tiny = n * std::numeric_limits<double>::epsilon() * amax;
  std::vector<int> piv(n);
  for (int i = 0; i < n; ++i) piv[i] = i;
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int best = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)best * n + col])) best = r;
    if (!(std::fabs(a[(size_t)best * n + col]) > tiny)) return false;
    if (best != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)best * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)best * n + k], inv[(size_t)col * n + k]);
      }
    const double d = 1.0 / a[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      a[(size_t)col * n + k] *= d;
      inv[(size_t)col * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

void form_vanka(HostLevel& L, const SetupParams& prm) {
  const int nu = L.dim * L.n_v, N = L.N();
  std::vector<char> covered(N, 0);
  L.vk_ptr.assign(1, 0);
  L.vk_dofs.clear();
  for (int i = 0; i < L.n_p; ++i) {
    std::vector<int> cols(L.B.col.begin() + L.B.row_begin(i), L.B.col.begin() + L.B.row_end(i));
    std::sort(cols.begin(), cols.end());
    for (int v : cols) {
      L.vk_dofs.push_back(v);
      covered[v] = 1;
    }
    L.vk_dofs.push_back(nu + i);
    covered[nu + i] = 1;
    L.vk_ptr.push_back((int)L.vk_dofs.size());
  }
  L.vk_dirichlet.clear();
  for (int c = 0; c < L.dim; ++c)
    for (int i = 0; i < L.n_v; ++i)
      if (L.dirichlet[i]) {
        L.vk_dirichlet.push_back(c * L.n_v + i);
        covered[c * L.n_v + i] = 1;
      }
  for (int q = 0; q < N; ++q)
    if (!covered[q]) {
      L.vk_dofs.push_back(q);
      L.vk_ptr.push_back((int)L.vk_dofs.size());
    }
  const int nb = (int)L.vk_ptr.size() - 1;
  // dof -> blocks holding it
  std::vector<int> dptr(N + 1, 0), dblk(L.vk_dofs.size());
  for (int v : L.vk_dofs) ++dptr[v + 1];
  for (int q = 0; q < N; ++q) dptr[q + 1] += dptr[q];
  {
    std::vector<int> pos(dptr.begin(), dptr.end() - 1);
    for (int b = 0; b < nb; ++b)
      for (int t = L.vk_ptr[b]; t < L.vk_ptr[b + 1]; ++t) dblk[pos[L.vk_dofs[t]]++] = b;
  }
  // interaction graph (symmetrised) and greedy coloring
  std::vector<std::vector<int>> adj(nb);
  std::vector<int> stamp(nb, -1);
  for (int b = 0; b < nb; ++b) {
    auto touch = [&](int v) {
      for (int t = dptr[v]; t < dptr[v + 1]; ++t) {
        const int o = dblk[t];
        if (o != b && stamp[o] != b) {
          stamp[o] = b;
          adj[b].push_back(o);
        }
      }
    };
    for (int t = L.vk_ptr[b]; t < L.vk_ptr[b + 1]; ++t) {
      const int q = L.vk_dofs[t];
      touch(q);
      block_matrix_row(L, q, [&](int v, double) { touch(v); });
    }
  }
  for (int b = 0; b < nb; ++b)
    for (int o : adj[b])
      if (std::find(adj[o].begin(), adj[o].end(), b) == adj[o].end()) adj[o].push_back(b);
  L.vk_colors.assign(nb, -1);
  L.vk_ncolors = 0;
  std::vector<int> mark;
  for (int b = 0; b < nb; ++b) {
    mark.assign(mark.size(), 0);
    for (int o : adj[b])
      if (L.vk_colors[o] >= 0) {
        if ((int)mark.size() <= L.vk_colors[o]) mark.resize(L.vk_colors[o] + 1, 0);
        mark[L.vk_colors[o]] = 1;
      }
    int c = 0;
    while (c < (int)mark.size() && mark[c]) ++c;
    L.vk_colors[b] = c;
    L.vk_ncolors = std::max(L.vk_ncolors, c + 1);
  }
  // local matrices and their inverses, blocks split over the host's threads
  L.vk_inv_off.assign(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    const int64_t m = L.vk_ptr[b + 1] - L.vk_ptr[b];
    L.vk_inv_off[b + 1] = L.vk_inv_off[b] + m * m;
  }
  if ((size_t)L.vk_inv_off[nb] * sizeof(double) > prm.vanka_max_bytes)
    throw std::runtime_error("Vanka block inverses of a level need " +
                             std::to_string((size_t)L.vk_inv_off[nb] * sizeof(double) >> 20) +
                             " MiB, more than the limit (blocks too large, e.g. in 3D)");
  L.vk_inv.assign((size_t)L.vk_inv_off[nb], 0.0);
  std::string failure;
  auto work = [&](int b0, int b1) {
    std::vector<int> loc(N, -1);
    std::vector<double> a;
    for (int b = b0; b < b1; ++b) {
      const int p0 = L.vk_ptr[b], m = L.vk_ptr[b + 1] - p0;
      for (int j = 0; j < m; ++j) loc[L.vk_dofs[p0 + j]] = j;
      a.assign((size_t)m * m, 0.0);
      for (int j = 0; j < m; ++j)
        block_matrix_row(L, L.vk_dofs[p0 + j], [&](int v, double val) {
          if (loc[v] >= 0) a[(size_t)j * m + loc[v]] += val;
        });
      if (!invert_dense(a, m))
        failure = "a Vanka block matrix is singular (a level whose pressures carry no coupling, such as a "
                  "coarsest level that keeps only the constant pressure, has no Vanka step)";
      std::copy(a.begin(), a.end(), L.vk_inv.begin() + L.vk_inv_off[b]);
      for (int j = 0; j < m; ++j) loc[L.vk_dofs[p0 + j]] = -1;
    }
  };
  const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), 16));
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(work, (int)((int64_t)nb * t / nt), (int)((int64_t)nb * (t + 1) / nt));
  for (auto& th : pool) th.join();
  if (!failure.empty()) throw std::runtime_error(failure);
}

// ILU(1) relaxation (Section 5): x <- x + (L U)^-1 (b - A x) with incomplete factors
// of the whole block matrix M, whose diagonal (the zero block's too) is kept in the
// pattern so that fill can reach it.  Level of fill one: position (i, j) of the
// factors exists when M has it or i == j (level 0), or when some m < min(i, j) has
// (i, m) and (m, j) at level 0 (level 1: a path through a level-1 entry has level 2
// and is dropped); the elimination then runs in IKJ order over that pattern.  A
// pivot that no elimination step reaches and whose entry of M is zero (a row of the
// zero block ordered before all its neighbours) becomes -sum_j M_ij M_ji / M_jj over
// its row: the Schur-complement diagonal of its neighbours with their block taken
// as diagonal.

// Reverse Cuthill-McKee on the graph of M + M^T without self loops: start at the
// unvisited vertex of smallest degree (lowest index on ties), visit each vertex's
// unvisited neighbours by increasing (degree, index), start again for every new
// component, reverse the visiting order.  Result: position -> index.
std::vector<int> rcm_order(const Csr& M) {
  const int n = M.nrows;
  std::vector<std::vector<int>> nb(n);
  for (int i = 0; i < n; ++i)
    for (int64_t t = M.row_begin(i); t < M.row_end(i); ++t) {
      const int j = M.col[t];
      if (j == i || M.val[t] == 0.0) continue;
      nb[i].push_back(j);
      nb[j].push_back(i);
    }
  std::vector<int> deg(n);
  for (int i = 0; i < n; ++i) {
    std::sort(nb[i].begin(), nb[i].end());
    nb[i].erase(std::unique(nb[i].begin(), nb[i].end()), nb[i].end());
    deg[i] = (int)nb[i].size();
  }
  auto before = [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; };
  std::vector<int> by_degree(n);
  for (int i = 0; i < n; ++i) by_degree[i] = i;
  std::sort(by_degree.begin(), by_degree.end(), before);
  std::vector<char> seen(n, 0);
  std::vector<int> order;
  order.reserve(n);
  std::vector<int> next;
  for (int start : by_degree) {
    if (seen[start]) continue;
    seen[start] = 1;
    size_t head = order.size();
    order.push_back(start);
    while (head < order.size()) {
      const int v = order[head++];
      next.clear();
      for (int u : nb[v])
        if (!seen[u]) next.push_back(u);
      std::sort(next.begin(), next.end(), before);
      for (int u : next) {
        seen[u] = 1;
        order.push_back(u);
      }
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

// Rows of a triangular factor by (dependency level, position): a row's level is one
// more than the largest level among the rows its entries refer to.
void schedule(const Csr& T, bool lower, std::vector<int>& sched, int& depth) {
  const int n = T.nrows;
  std::vector<int> lev(n, 0);
  depth = 0;
  for (int s = 0; s < n; ++s) {
    const int i = lower ? s : n - 1 - s;
    int l = 0;
    for (int64_t t = T.row_begin(i); t < T.row_end(i); ++t) l = std::max(l, lev[T.col[t]] + 1);
    lev[i] = l;
    depth = std::max(depth, l + 1);
  }
  std::vector<int> cnt(depth + 1, 0);
  for (int i = 0; i < n; ++i) cnt[lev[i] + 1]++;
  for (int l = 0; l < depth; ++l) cnt[l + 1] += cnt[l];
  sched.assign(n, 0);
  for (int i = 0; i < n; ++i) sched[cnt[lev[i]]++] = i;
}

// Location order: dofs sorted by their node's coordinates (last coordinate slowest:
// lexicographic from the lower-left corner), the dofs of one node as u_x, u_y (, u_z),
// p; a pressure takes its co-located velocity node's coordinates (exact ties).
std::vector<int> location_order(const HostLevel& L) {
  const int n = L.N(), nu = L.dim * L.n_v, d = L.dim;
  auto coord = [&](int q) -> const double* {
    if (q < nu) return &L.vX[(size_t)(q % L.n_v) * d];
    const int i = q - nu;
    const int v = L.p2v.empty() ? -1 : L.p2v[i];
    return v >= 0 ? &L.vX[(size_t)v * d] : &L.pX[(size_t)i * d];
  };
  std::vector<int> order(n);
  for (int q = 0; q < n; ++q) order[q] = q;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const double* xa = coord(a);
    const double* xb = coord(b);
    for (int k = d - 1; k >= 0; --k)
      if (xa[k] != xb[k]) return xa[k] < xb[k];
    return a < b;  // u_x, u_y (, u_z), p: the block order at one node
  });
  return order;
}

void form_ilu(HostLevel& L, bool symmetric, int ilu_order) {
  const int n = L.N();
  Csr M;  // natural order
  M.resize_rows(n, n);
  for (int q = 0; q < n; ++q) {
    const size_t b = M.col.size();
    block_matrix_row(L, q, [&](int v, double val) {
      M.col.push_back(v);
      M.val.push_back(val);
    });
    std::vector<std::pair<int, double>> row;
    for (size_t t = b; t < M.col.size(); ++t) row.emplace_back(M.col[t], M.val[t]);
    std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    for (size_t t = 0; t < row.size(); ++t) {
      M.col[b + t] = row[t].first;
      M.val[b + t] = row[t].second;
    }
    M.rowptr[q + 1] = (int64_t)M.col.size();
  }
  std::vector<int> perm(n);
  if (!symmetric)
    perm = rcm_order(M);
  else if (ilu_order == 1)
    perm = location_order(L);
  else
    for (int i = 0; i < n; ++i) perm[i] = i;
  std::vector<int> pos(n);
  for (int i = 0; i < n; ++i) pos[perm[i]] = i;
  // the permuted matrix (rows and columns in positions), rows ascending
  Csr Mp;
  Mp.resize_rows(n, n);
  {
    std::vector<std::pair<int, double>> row;
    for (int i = 0; i < n; ++i) {
      row.clear();
      const int q = perm[i];
      for (int64_t t = M.row_begin(q); t < M.row_end(q); ++t) row.emplace_back(pos[M.col[t]], M.val[t]);
      std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      for (const auto& e : row) {
        Mp.col.push_back(e.first);
        Mp.val.push_back(e.second);
      }
      Mp.rowptr[i + 1] = (int64_t)Mp.col.size();
    }
  }
  // symbolic: level-0 pattern (M's plus the diagonal) and the level-1 fill
  std::vector<int64_t> fptr(n + 1, 0);
  std::vector<int> fcol;
  {
    std::vector<int> mark(n, -1), row;
    for (int i = 0; i < n; ++i) {
      row.clear();
      auto add = [&](int j) {
        if (mark[j] != i) {
          mark[j] = i;
          row.push_back(j);
        }
      };
      add(i);
      for (int64_t t = Mp.row_begin(i); t < Mp.row_end(i); ++t) add(Mp.col[t]);
      for (int64_t t = Mp.row_begin(i); t < Mp.row_end(i); ++t) {
        const int m = Mp.col[t];
        if (m >= i) continue;
        for (int64_t u = Mp.row_begin(m); u < Mp.row_end(m); ++u)
          if (Mp.col[u] > m) add(Mp.col[u]);
      }
      std::sort(row.begin(), row.end());
      fcol.insert(fcol.end(), row.begin(), row.end());
      fptr[i + 1] = (int64_t)fcol.size();
    }
  }
  // numeric: IKJ over the fixed pattern
  Csr& Lf = L.il_L;
  Csr& Uf = L.il_U;
  Lf.resize_rows(n, n);
  Uf.resize_rows(n, n);
  L.il_diag.assign(n, 0.0);
  std::vector<double> w(n, 0.0);
  std::vector<int> in(n, -1);
  for (int i = 0; i < n; ++i) {
    for (int64_t t = fptr[i]; t < fptr[i + 1]; ++t) {
      in[fcol[t]] = i;
      w[fcol[t]] = 0.0;
    }
    for (int64_t t = Mp.row_begin(i); t < Mp.row_end(i); ++t) w[Mp.col[t]] += Mp.val[t];
    bool reached = false;
    for (int64_t t = fptr[i]; t < fptr[i + 1] && fcol[t] < i; ++t) {
      const int m = fcol[t];
      const double f = w[m] / L.il_diag[m];
      w[m] = f;
      for (int64_t u = Uf.row_begin(m); u < Uf.row_end(m); ++u) {
        const int j = Uf.col[u];
        if (in[j] == i) w[j] -= f * Uf.val[u];
      }
      // the step reaches the pivot when (m, i) is in row m's upper part
      if (std::binary_search(Uf.col.begin() + Uf.row_begin(m), Uf.col.begin() + Uf.row_end(m), i)) reached = true;
    }
    if (!reached && w[i] == 0.0) {
      double sdiag = 0.0;
      for (int64_t t = Mp.row_begin(i); t < Mp.row_end(i); ++t) {
        const int j = Mp.col[t];
        if (j == i) continue;
        const double mjj = lookup(Mp, j, j);
        if (mjj != 0.0) sdiag -= Mp.val[t] * lookup(Mp, j, i) / mjj;
      }
      w[i] = sdiag;
    }
    for (int64_t t = fptr[i]; t < fptr[i + 1]; ++t) {
      const int j = fcol[t];
      if (j < i) {
        Lf.col.push_back(j);
        Lf.val.push_back(w[j]);
      } else if (j > i) {
        Uf.col.push_back(j);
        Uf.val.push_back(w[j]);
      }
    }
    L.il_diag[i] = w[i];
    Lf.rowptr[i + 1] = Lf.nnz();
    Uf.rowptr[i + 1] = Uf.nnz();
  }
  L.il_perm = std::move(perm);
  schedule(Lf, true, L.il_schedL, L.il_depthL);
  schedule(Uf, false, L.il_schedU, L.il_depthU);
}

}  // namespace

std::vector<HostLevel> build_hierarchy(HostLevel fine, const SetupParams& prm) {
  std::vector<HostLevel> levels;
  levels.push_back(std::move(fine));
  const std::vector<HostLevel>* prev = prm.reuse;
  while (true) {
    HostLevel& L = levels.back();
    TraceRange level_range("setup: level %d", (int)levels.size() - 1);
    {
      TraceRange r("Braess-Sarazin data (D, S, strips, colors)");
      form_relaxation(L, prm);
    }
    if (prev) {
      // the previous hierarchy decides the levels
      if (levels.size() >= prev->size()) break;
      HostLevel Lc;
      form_interpolation_reuse(L, Lc, prm, (*prev)[levels.size() - 1]);
      levels.push_back(std::move(Lc));
      continue;
    }
    if (L.N() <= prm.max_coarse || (int)levels.size() == prm.max_levels) break;
    HostLevel Lc;
    // with the coarsest level relaxed by Vanka, a level keeping only one pressure (the
    // constant, whose B vanishes) has no Vanka step: the current level stays the coarsest
    if (!form_interpolation(L, Lc, prm) || Lc.N() >= L.N() || (prm.vanka_coarse && Lc.n_p <= 1)) {
      L.P = L.Pp = L.R = L.Rp = Csr();
      L.Cp.clear();
      L.Cv.clear();
      break;
    }
    levels.push_back(std::move(Lc));
  }
  complete_hierarchy(levels, prm, false);
  return levels;
}

void complete_hierarchy(std::vector<HostLevel>& levels, const SetupParams& prm, bool relaxation) {
  if (levels.empty()) throw std::runtime_error("a hierarchy needs at least one level");
  if (relaxation) {
    TraceRange r("setup: Braess-Sarazin data of every level");
    for (HostLevel& L : levels) form_relaxation(L, prm);
  }
  HostLevel& C = levels.back();
  if (C.N() > 4096) throw std::runtime_error("coarsest level too large for the dense solve: " + std::to_string(C.N()));
  {
    TraceRange r("setup: coarsest pseudo-inverse");
    const std::vector<double> M = dense_level(C);
    C.pinv = pseudo_inverse(M, C.N(), 1e-12);
    refine_pseudo_inverse(M, C.pinv, C.N());
  }
  if (prm.vanka || prm.vanka_coarse) {
    TraceRange r("setup: Vanka blocks");
    if (prm.vanka)
      for (size_t l = 0; l + 1 < levels.size(); ++l) form_vanka(levels[l], prm);
    if (prm.vanka_coarse) form_vanka(levels.back(), prm);
  }
  if (prm.ilu) {
    TraceRange r("setup: ILU(1) factors");
    for (size_t l = 0; l + 1 < levels.size(); ++l) form_ilu(levels[l], prm.symmetric, prm.ilu_order);
  }
  if (prm.dense_gs) {
    TraceRange r("setup: dense Gauss-Seidel maps (host)");
    for (size_t l = 0; l + 1 < levels.size(); ++l)
      if (levels[l].n_p <= kGsDenseMaxRows) form_dense_gs(levels[l], prm.gs_iters);
  }
}

}  // namespace emin

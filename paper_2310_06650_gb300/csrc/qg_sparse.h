// Host-side sparse factorizations of the reduced DC Laplacian Yhat = E_hat^T Y_x E_hat
// (Sec. II-E), with a minimum-degree elimination order.
//   SparseLDL  full LDL^T; builds columns of Yhat^-1 at set-up (dense inverse for small grids).
//   TailLDL    LDL^T with a dense tail for large grids: the gather lists and the tail inverse
//              that the device solves use, and u_k = Yhat^-1 a_k for the line-outage block.
#pragma once

#include <cstdint>
#include <map>
#include <set>
#include <utility>
#include <vector>
#include <algorithm>
#include <cmath>
#include <thread>

namespace qg {

class SparseLDL {
 public:
  // A: symmetric matrix of size n given as adjacency maps (off-diagonal) plus diagonal.
  // Returns false if a pivot is not positive (the grid is disconnected or not positive definite).
  bool factor(int n, std::vector<std::map<int, double>> off, std::vector<double> diag) {
    n_ = n;
    order_.clear();
    order_.reserve(n);
    colp_.assign(1, 0);
    rows_.clear();
    vals_.clear();
    D_.clear();
    std::set<std::pair<int, int>> heap;  // (degree, node)
    std::vector<char> gone(n, 0);
    for (int i = 0; i < n; ++i) heap.insert({(int)off[i].size(), i});
    for (int step = 0; step < n; ++step) {
      const int k = heap.begin()->second;
      heap.erase(heap.begin());
      gone[k] = 1;
      const double dk = diag[k];
      if (!(dk > 0.0)) return false;
      order_.push_back(k);
      D_.push_back(dk);
      // neighbours of k in the current (filled) graph
      std::vector<std::pair<int, double>> nb(off[k].begin(), off[k].end());
      for (auto &e : nb) {
        rows_.push_back(e.first);
        vals_.push_back(e.second / dk);
      }
      colp_.push_back((int64_t)rows_.size());
      // Schur complement update on the neighbours, with fill
      for (size_t a = 0; a < nb.size(); ++a) {
        const int i = nb[a].first;
        heap.erase({(int)off[i].size(), i});
        off[i].erase(k);
      }
      for (size_t a = 0; a < nb.size(); ++a) {
        const int i = nb[a].first;
        const double aik = nb[a].second;
        diag[i] -= aik * aik / dk;
        for (size_t b = 0; b < nb.size(); ++b) {
          if (b == a) continue;
          const int j = nb[b].first;
          off[i][j] -= aik * nb[b].second / dk;
        }
      }
      for (size_t a = 0; a < nb.size(); ++a) {
        const int i = nb[a].first;
        heap.insert({(int)off[i].size(), i});
      }
    }
    return true;
  }

  // In-place solve A x = b (b has n entries in the original numbering).
  void solve(double *b) const {
    for (int s = 0; s < n_; ++s) {
      const int k = order_[s];
      const double bk = b[k];
      for (int64_t e = colp_[s]; e < colp_[s + 1]; ++e) b[rows_[e]] -= vals_[e] * bk;
    }
    for (int s = 0; s < n_; ++s) b[order_[s]] /= D_[s];
    for (int s = n_ - 1; s >= 0; --s) {
      const int k = order_[s];
      double acc = b[k];
      for (int64_t e = colp_[s]; e < colp_[s + 1]; ++e) acc -= vals_[e] * b[rows_[e]];
      b[k] = acc;
    }
  }

  int64_t nnz() const { return (int64_t)rows_.size(); }
  int size() const { return n_; }

 private:
  int n_ = 0;
  std::vector<int> order_;
  std::vector<int64_t> colp_;
  std::vector<int> rows_;
  std::vector<double> vals_;
  std::vector<double> D_;
};

}  // namespace qg

namespace qg {

// Run f(i) for i in [0, count) on all hardware threads, interleaved for load balance.
template <typename F>
void parallel_for(int count, F f) {
  const int nth = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
  if (count < 64 || nth == 1) {
    for (int i = 0; i < count; ++i) f(i);
    return;
  }
  std::vector<std::thread> pool;
  for (int w = 0; w < nth; ++w)
    pool.emplace_back([&, w]() {
      for (int i = w; i < count; i += nth) f(i);
    });
  for (auto &t : pool) t.join();
}

// LDL^T of the reduced DC Laplacian for large grids: minimum-degree elimination while the
// eliminated node has at most `dmax` neighbours, then a dense Schur complement S on the remaining
// "tail" nodes, stored through its explicit inverse: Yhat = L diag(D_S, S) L^T.  `levels` is the
// height of the elimination forest of the eliminated nodes (one more than the longest chain of
// dependencies), which bounds the length of every reach column below.
class TailLDL {
 public:
  struct Col {
    int node;
    std::vector<std::pair<int, double>> l;  // (row node, l_ik) for rows eliminated later
    double d;
    int level;
  };

  int n = 0;                 // reduced size
  std::vector<Col> cols;     // eliminated (sparse) nodes in elimination order
  std::vector<int> tail;     // tail nodes
  std::vector<int> tail_pos; // node -> position in tail, -1 for sparse nodes
  std::vector<double> Sinv;  // tail x tail, row-major
  int levels = 0;

  bool factor(int nn, std::vector<std::map<int, double>> off, std::vector<double> diag, int dmax) {
    n = nn;
    cols.clear();
    tail.clear();
    std::vector<int> level(n, 0);
    std::set<std::pair<int, int>> heap;
    std::vector<char> gone(n, 0);
    for (int i = 0; i < n; ++i) heap.insert({(int)off[i].size(), i});
    while (!heap.empty()) {
      const int k = heap.begin()->second;
      if ((int)off[k].size() > dmax) break;
      heap.erase(heap.begin());
      gone[k] = 1;
      const double dk = diag[k];
      if (!(dk > 0.0)) return false;
      Col c;
      c.node = k;
      c.d = dk;
      c.level = level[k];
      std::vector<std::pair<int, double>> nb(off[k].begin(), off[k].end());
      for (auto &e : nb) c.l.push_back({e.first, e.second / dk});
      for (auto &e : nb) {
        heap.erase({(int)off[e.first].size(), e.first});
        off[e.first].erase(k);
        level[e.first] = std::max(level[e.first], level[k] + 1);
      }
      for (size_t a = 0; a < nb.size(); ++a) {
        const int i = nb[a].first;
        const double aik = nb[a].second;
        diag[i] -= aik * aik / dk;
        for (size_t b = 0; b < nb.size(); ++b)
          if (b != a) off[i][nb[b].first] -= aik * nb[b].second / dk;
      }
      for (auto &e : nb) heap.insert({(int)off[e.first].size(), e.first});
      levels = std::max(levels, c.level + 1);
      cols.push_back(std::move(c));
    }
    tail_pos.assign(n, -1);
    for (int i = 0; i < n; ++i)
      if (!gone[i]) {
        tail_pos[i] = (int)tail.size();
        tail.push_back(i);
      }
    const int m = (int)tail.size();
    std::vector<double> S((size_t)m * m, 0.0);
    for (int a = 0; a < m; ++a) {
      const int i = tail[a];
      S[(size_t)a * m + a] = diag[i];
      for (auto &e : off[i]) S[(size_t)a * m + tail_pos[e.first]] = e.second;
    }
    return invert_spd(S, m);
  }

  // Node positions: eliminated nodes first, in elimination order, then the tail nodes.
  int n_sparse() const { return (int)cols.size(); }
  std::vector<int> positions() const {
    std::vector<int> pos(n, -1);
    for (size_t c = 0; c < cols.size(); ++c) pos[cols[c].node] = (int)c;
    for (size_t a = 0; a < tail.size(); ++a) pos[tail[a]] = (int)(cols.size() + a);
    return pos;
  }

  // Columns of the explicit factor inverse, in positions: for every eliminated node q the
  // nonzeros of L^-1 e_q (its reach: q itself with value 1, then the eliminated ancestors, rows of
  // M1 = L_SS^-1, and the tail nodes they touch, rows of M2 = -L_TS L_SS^-1).  With these,
  //   forward   z_S = M1 b_S,  z_T = b_T + M2 b_S,
  //   backward  x_T = S^-1 z_T,  x_S = M1^T (D_S^-1 z_S) + M2^T x_T
  // solve Yhat x = b with two gathers and one dense product.  Parallel over columns.
  void reach_columns(std::vector<std::vector<std::pair<int, double>>> &out) const {
    const int nS = n_sparse();
    const std::vector<int> pos = positions();
    std::vector<std::vector<std::pair<int, double>>> lp(nS);
    for (int c = 0; c < nS; ++c) {
      for (auto &e : cols[c].l) lp[c].push_back({pos[e.first], e.second});
      std::sort(lp[c].begin(), lp[c].end());
    }
    out.assign(nS, {});
    const unsigned nth = std::max(1u, std::thread::hardware_concurrency());
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nth; ++w)
      pool.emplace_back([&, w]() {
        std::map<int, double> reach;
        for (int q = (int)w; q < nS; q += (int)nth) {
          reach.clear();
          reach[q] = 1.0;
          for (auto it = reach.begin(); it != reach.end() && it->first < nS; ++it) {
            const double v = it->second;
            for (auto &e : lp[it->first]) reach[e.first] -= e.second * v;
          }
          out[q].assign(reach.begin(), reach.end());
        }
      });
    for (auto &t : pool) t.join();
  }

  // In-place solve Yhat x = b for one right-hand side (reduced numbering).
  void solve(double *b) const {
    for (const Col &c : cols)
      for (auto &e : c.l) b[e.first] -= e.second * b[c.node];
    const int m = (int)tail.size();
    std::vector<double> t(m, 0.0);
    for (int a = 0; a < m; ++a) {
      double s = 0.0;
      const double *row = &Sinv[(size_t)a * m];
      for (int q = 0; q < m; ++q) s += row[q] * b[tail[q]];
      t[a] = s;
    }
    for (int a = 0; a < m; ++a) b[tail[a]] = t[a];
    for (auto it = cols.rbegin(); it != cols.rend(); ++it) {
      double acc = b[it->node] / it->d;
      for (auto &e : it->l) acc -= e.second * b[e.first];
      b[it->node] = acc;
    }
  }

 private:
  // Explicit inverse of a symmetric positive definite matrix: blocked right-looking Cholesky
  // S = C C^T (lower triangle of S, in place), then the columns of C^-1 by forward substitution,
  // then S^-1 = C^-T C^-1.  Every inner loop runs over contiguous memory.
  bool invert_spd(std::vector<double> &S, int m) {
    Sinv.assign((size_t)m * m, 0.0);
    if (m == 0) return true;
    double *A = S.data();
    constexpr int NB = 64;
    bool ok = true;
    for (int J = 0; J < m && ok; J += NB) {
      const int je = std::min(m, J + NB);
      for (int j = J; j < je && ok; ++j) {  // diagonal block, unblocked
        double *aj = A + (size_t)j * m;
        double d = aj[j];
        for (int k = J; k < j; ++k) d -= aj[k] * aj[k];
        if (!(d > 0.0)) {
          ok = false;
          break;
        }
        aj[j] = std::sqrt(d);
        for (int i = j + 1; i < je; ++i) {
          double *ai = A + (size_t)i * m;
          double v = ai[j];
          for (int k = J; k < j; ++k) v -= ai[k] * aj[k];
          ai[j] = v / aj[j];
        }
      }
      if (!ok) break;
      parallel_for(m - je, [&](int r) {  // panel rows below the block, then their trailing update
        const int i = je + r;
        double *ai = A + (size_t)i * m;
        for (int j = J; j < je; ++j) {
          const double *aj = A + (size_t)j * m;
          double v = ai[j];
          for (int k = J; k < j; ++k) v -= ai[k] * aj[k];
          ai[j] = v / aj[j];
        }
      });
      parallel_for(m - je, [&](int r) {
        const int i = je + r;
        double *ai = A + (size_t)i * m;
        for (int k = je; k <= i; ++k) {
          const double *ak = A + (size_t)k * m;
          double v = 0.0;
          for (int c = J; c < je; ++c) v += ai[c] * ak[c];
          ai[k] -= v;
        }
      });
    }
    if (!ok) return false;
    // W[c][i] = (C^-1)[i][c] for i >= c
    std::vector<double> W((size_t)m * m, 0.0);
    parallel_for(m, [&](int c) {
      double *w = W.data() + (size_t)c * m;
      for (int i = c; i < m; ++i) {
        const double *ai = A + (size_t)i * m;
        double v = (i == c) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) v -= ai[k] * w[k];
        w[i] = v / ai[i];
      }
    });
    parallel_for(m, [&](int a) {
      const double *wa = W.data() + (size_t)a * m;
      for (int b = 0; b <= a; ++b) {
        const double *wb = W.data() + (size_t)b * m;
        double v = 0.0;
        for (int k = a; k < m; ++k) v += wa[k] * wb[k];
        Sinv[(size_t)a * m + b] = v;
        Sinv[(size_t)b * m + a] = v;
      }
    });
    return true;
  }
};

}  // namespace qg

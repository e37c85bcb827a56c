// Host-side sparse LDL^T factorization of the reduced DC Laplacian
// Yhat = E_hat^T Y_x E_hat (Sec. II-E), with a minimum-degree elimination order.
// Used at set-up to build columns of Yhat^-1 (the dense inverse for small grids and
// u_k = Yhat^-1 a_k for the line-outage block).
#pragma once

#include <cstdint>
#include <map>
#include <set>
#include <utility>
#include <vector>

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

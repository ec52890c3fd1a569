// setup.cpp -- host construction of the classical AMG hierarchy that the GPU
// solve phase runs on (paper Sec. 2.3: the MultiGrid setup(), done once; the
// solve phase then treats its output as frozen input).
//
// Steps, per level, in this order (classical Ruge-Stueben AMG, Trottenberg et
// al. App. A, which the paper's Sec. 1 and 2.1 name):
//   1. strength of connection with threshold theta: j is a strong dependency
//      of i when -a_ij >= theta * max_{k != i}(-a_ik) and that maximum is > 0;
//   2. C/F splitting, first pass: the undecided point with the largest
//      measure lambda_i = |S_i^T cap U| + 2 |S_i^T cap F| (ties: smallest
//      index) becomes C and its undecided strong dependents become F; points
//      without strong dependencies start as F;
//   3. second pass: for F points in index order, each strong F neighbour k
//      (column order) must depend strongly on a point of C_i, else k becomes C;
//   4. classical interpolation (weak connections lumped into the diagonal,
//      strong F connections spread over C_i through the entries of row k whose
//      sign is opposite to a_kk; a zero spread lumps into the diagonal);
//   5. R = P^T and the Galerkin product A_c = R A P, accumulated per coarse row
//      in the order (k in R_I, l in A_k, J in P_l) with every structural entry
//      kept;
//   6. stop at n <= max_coarse, at max_levels, or when more than 0.9 n points
//      would stay coarse;
//   7. Chebyshev interval of D^-1 A per level: b = min(hi_safety * lambda_hat,
//      Gershgorin bound), a = lo_frac * b, lambda_hat from power iterations
//      started at the SplitMix64 vector of seed 0;
//   8. dense LU with partial pivoting of the coarsest operator.
// The floating-point expressions are evaluated exactly in the order written
// (the file is compiled without contraction), so the hierarchy is a
// deterministic function of A and the parameters for any thread count.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>

#include "hier_host.h"

namespace xamg {
namespace {

int thread_count(int req) {
  if (req > 0) return req;
  unsigned h = std::thread::hardware_concurrency();
  return h ? (int)std::min(h, 64u) : 1;
}

// Runs f(begin, end, tid) over [0, n) in contiguous chunks.  Returns false if
// any chunk ran out of memory.
template <class F>
bool parallel_rows(int n, int nt, F &&f) {
  std::atomic<bool> ok{true};
  auto run = [&](int b, int e, int t) {
    try {
      f(b, e, t);
    } catch (const std::bad_alloc &) {
      ok = false;
    }
  };
  if (nt <= 1 || n < 8192) {
    run(0, n, 0);
    return ok;
  }
  std::vector<std::thread> th;
  int chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back(run, b, e, t);
  }
  for (auto &x : th) x.join();
  return ok;
}

int chunks_for(int n, int nt) { return (nt <= 1 || n < 8192) ? 1 : nt; }

// ---- step 1 ----
void strength(const HostCsr &A, double theta, HostCsr &S, int nt) {
  const int n = A.n;
  S.n = S.ncols = n;
  S.rowptr.assign((size_t)n + 1, 0);
  auto row_max = [&](int i) {
    double mx = 0.0;
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
      if (A.col[p] != i && -A.val[p] > mx) mx = -A.val[p];
    return mx;
  };
  parallel_rows(n, nt, [&](int b, int e, int) {
    for (int i = b; i < e; ++i) {
      double mx = row_max(i);
      int c = 0;
      if (mx > 0.0)
        for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
          if (A.col[p] != i && -A.val[p] >= theta * mx) ++c;
      S.rowptr[i + 1] = c;
    }
  });
  for (int i = 0; i < n; ++i) S.rowptr[i + 1] += S.rowptr[i];
  S.col.resize((size_t)S.rowptr[n]);
  parallel_rows(n, nt, [&](int b, int e, int) {
    for (int i = b; i < e; ++i) {
      double mx = row_max(i);
      int q = S.rowptr[i];
      if (mx > 0.0)
        for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
          if (A.col[p] != i && -A.val[p] >= theta * mx) S.col[q++] = A.col[p];
    }
  });
}

// CSR transpose by counting sort; rows of the result have ascending columns.
void transpose(const HostCsr &A, HostCsr &T, bool values) {
  T.n = A.ncols;
  T.ncols = A.n;
  T.rowptr.assign((size_t)T.n + 1, 0);
  const int64_t nnz = A.nnz();
  for (int64_t p = 0; p < nnz; ++p) T.rowptr[A.col[p] + 1]++;
  for (int i = 0; i < T.n; ++i) T.rowptr[i + 1] += T.rowptr[i];
  T.col.resize((size_t)nnz);
  if (values) T.val.resize((size_t)nnz);
  std::vector<int32_t> next(T.rowptr.begin(), T.rowptr.end() - 1);
  for (int i = 0; i < A.n; ++i)
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
      int q = next[A.col[p]]++;
      T.col[q] = i;
      if (values) T.val[q] = A.val[p];
    }
}

// Arg-max tree over the undecided points: the root holds the point with the
// largest measure, the smallest index among equal measures.
class ArgMaxTree {
 public:
  ArgMaxTree(const std::vector<int32_t> &key, const std::vector<char> &live) : key_(key), live_(live) {
    size_ = 1;
    while (size_ < (int)key.size()) size_ <<= 1;
    node_.assign(2 * (size_t)size_, -1);
    for (int i = 0; i < (int)key.size(); ++i) node_[size_ + i] = live[i] ? i : -1;
    for (int p = size_ - 1; p >= 1; --p) node_[p] = pick(node_[2 * p], node_[2 * p + 1]);
  }
  int top() const { return node_[1]; }
  void refresh(int i) {
    int p = size_ + i;
    node_[p] = live_[i] ? i : -1;
    for (p >>= 1; p >= 1; p >>= 1) node_[p] = pick(node_[2 * p], node_[2 * p + 1]);
  }

 private:
  int pick(int a, int b) const {
    if (a < 0) return b;
    if (b < 0) return a;
    if (key_[a] != key_[b]) return key_[a] > key_[b] ? a : b;
    return a < b ? a : b;
  }
  const std::vector<int32_t> &key_;
  const std::vector<char> &live_;
  int size_;
  std::vector<int32_t> node_;
};

// ---- steps 2 and 3 ----
void split(const HostCsr &S, const HostCsr &ST, std::vector<int32_t> &cf) {
  const int n = S.n;
  enum : char { U = 0, C = 1, F = 2 };
  std::vector<char> st((size_t)n);
  std::vector<char> live((size_t)n);
  std::vector<int32_t> lam((size_t)n);
  for (int i = 0; i < n; ++i) {
    lam[i] = ST.rowptr[i + 1] - ST.rowptr[i];
    st[i] = (S.rowptr[i + 1] == S.rowptr[i]) ? F : U;
    live[i] = st[i] == U;
  }
  ArgMaxTree tree(lam, live);
  for (int i = tree.top(); i >= 0; i = tree.top()) {
    st[i] = C;
    live[i] = 0;
    tree.refresh(i);
    for (int p = ST.rowptr[i]; p < ST.rowptr[i + 1]; ++p) {
      const int j = ST.col[p];
      if (st[j] != U) continue;
      st[j] = F;
      live[j] = 0;
      tree.refresh(j);
      for (int q = S.rowptr[j]; q < S.rowptr[j + 1]; ++q) {
        const int k = S.col[q];
        if (st[k] == U) {
          lam[k] += 1;
          tree.refresh(k);
        }
      }
    }
    for (int p = S.rowptr[i]; p < S.rowptr[i + 1]; ++p) {
      const int k = S.col[p];
      if (st[k] == U) {
        lam[k] -= 1;
        tree.refresh(k);
      }
    }
  }
  // second pass
  std::vector<int32_t> mark((size_t)n, -1);
  for (int i = 0; i < n; ++i) {
    if (st[i] != F || S.rowptr[i + 1] == S.rowptr[i]) continue;
    for (int p = S.rowptr[i]; p < S.rowptr[i + 1]; ++p)
      if (st[S.col[p]] == C) mark[S.col[p]] = i;
    for (int p = S.rowptr[i]; p < S.rowptr[i + 1]; ++p) {
      const int k = S.col[p];
      if (st[k] != F) continue;
      bool shared = false;
      for (int q = S.rowptr[k]; q < S.rowptr[k + 1] && !shared; ++q) shared = mark[S.col[q]] == i;
      if (!shared) {
        st[k] = C;
        mark[k] = i;
      }
    }
  }
  cf.resize((size_t)n);
  for (int i = 0; i < n; ++i) cf[i] = st[i] == C ? 1 : 0;
}

double diag_of(const HostCsr &A, int i) {
  double d = 0.0;
  for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
    if (A.col[p] == i) d = A.val[p];
  return d;
}

// ---- step 4 ----
int interpolation(const HostCsr &A, const HostCsr &S, const std::vector<int32_t> &cf, HostCsr &P,
                  int nt) {
  const int n = A.n;
  std::vector<int32_t> cidx((size_t)n);
  int nc = 0;
  for (int i = 0; i < n; ++i) cidx[i] = cf[i] ? nc++ : -1;
  P.n = n;
  P.ncols = nc;
  P.rowptr.assign((size_t)n + 1, 0);
  parallel_rows(n, nt, [&](int b, int e, int) {
    for (int i = b; i < e; ++i) {
      int c = 0;
      if (cf[i]) c = 1;
      else
        for (int p = S.rowptr[i]; p < S.rowptr[i + 1]; ++p) c += cf[S.col[p]];
      P.rowptr[i + 1] = c;
    }
  });
  for (int i = 0; i < n; ++i) P.rowptr[i + 1] += P.rowptr[i];
  P.col.resize((size_t)P.rowptr[n]);
  P.val.resize((size_t)P.rowptr[n]);
  std::atomic<int> bad{0};
  const int nchunks = chunks_for(n, nt);
  std::vector<std::vector<int32_t>> smark_t(nchunks), cmark_t(nchunks);
  std::vector<std::vector<double>> num_t(nchunks);
  bool ok = parallel_rows(n, nt, [&](int b, int e, int t) {
    std::vector<int32_t> &smark = smark_t[t], &cmark = cmark_t[t];
    std::vector<double> &num = num_t[t];
    smark.assign((size_t)n, -1);
    cmark.assign((size_t)n, -1);
    num.assign((size_t)n, 0.0);
    for (int i = b; i < e; ++i) {
      int q = P.rowptr[i];
      if (cf[i]) {
        P.col[q] = cidx[i];
        P.val[q] = 1.0;
        continue;
      }
      if (S.rowptr[i + 1] == S.rowptr[i]) continue;
      for (int p = S.rowptr[i]; p < S.rowptr[i + 1]; ++p) {
        const int j = S.col[p];
        smark[j] = i;
        if (cf[j]) {
          cmark[j] = i;
          num[j] = 0.0;
        }
      }
      double diag = diag_of(A, i);
      for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
        const int j = A.col[p];
        if (j == i) continue;
        if (smark[j] != i) diag = diag + A.val[p];
        else if (cf[j]) num[j] = num[j] + A.val[p];
      }
      for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
        const int k = A.col[p];
        if (k == i || smark[k] != i || cf[k]) continue;
        const double aik = A.val[p];
        const double akk = diag_of(A, k);
        double sum = 0.0;
        for (int r = A.rowptr[k]; r < A.rowptr[k + 1]; ++r)
          if (cmark[A.col[r]] == i && A.val[r] * akk < 0.0) sum = sum + A.val[r];
        if (sum == 0.0) {
          diag = diag + aik;
        } else {
          for (int r = A.rowptr[k]; r < A.rowptr[k + 1]; ++r) {
            const int l = A.col[r];
            if (cmark[l] == i && A.val[r] * akk < 0.0) num[l] = num[l] + aik * A.val[r] / sum;
          }
        }
      }
      if (diag == 0.0) {
        bad = 1;
        continue;
      }
      for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
        const int j = A.col[p];
        if (j != i && cmark[j] == i) {
          P.col[q] = cidx[j];
          P.val[q] = -num[j] / diag;
          ++q;
        }
      }
    }
    std::vector<int32_t>().swap(smark);
    std::vector<int32_t>().swap(cmark);
    std::vector<double>().swap(num);
  });
  if (!ok) return XAMG_ERR_OOM;
  return bad ? XAMG_ERR_SETUP : XAMG_OK;
}

// ---- step 5 ----
int galerkin(const HostCsr &R, const HostCsr &A, const HostCsr &P, HostCsr &Ac, int nt) {
  const int nc = R.n;
  const int nchunks = chunks_for(nc, nt);
  std::vector<std::vector<int32_t>> cols_t(nchunks), len_t(nchunks);
  std::vector<std::vector<double>> vals_t(nchunks);
  std::vector<int> first_row(nchunks, 0);
  bool ok = parallel_rows(nc, nt, [&](int b, int e, int t) {
    std::vector<int32_t> pos((size_t)P.ncols, -1), list;
    std::vector<double> acc((size_t)P.ncols, 0.0);
    std::vector<int32_t> &cols = cols_t[t], &lens = len_t[t];
    std::vector<double> &vals = vals_t[t];
    first_row[t] = b;
    for (int I = b; I < e; ++I) {
      list.clear();
      for (int p = R.rowptr[I]; p < R.rowptr[I + 1]; ++p) {
        const int k = R.col[p];
        const double rik = R.val[p];
        for (int q = A.rowptr[k]; q < A.rowptr[k + 1]; ++q) {
          const int l = A.col[q];
          const double t2 = rik * A.val[q];
          for (int s = P.rowptr[l]; s < P.rowptr[l + 1]; ++s) {
            const int J = P.col[s];
            if (pos[J] < 0) {
              pos[J] = (int32_t)list.size();
              list.push_back(J);
              acc[J] = 0.0;
            }
            acc[J] = acc[J] + t2 * P.val[s];
          }
        }
      }
      std::sort(list.begin(), list.end());
      for (int J : list) {
        cols.push_back(J);
        vals.push_back(acc[J]);
        pos[J] = -1;
      }
      lens.push_back((int32_t)list.size());
    }
  });
  if (!ok) return XAMG_ERR_OOM;
  Ac.n = nc;
  Ac.ncols = P.ncols;
  Ac.rowptr.assign((size_t)nc + 1, 0);
  int64_t total = 0;
  for (int t = 0; t < nchunks; ++t) total += (int64_t)cols_t[t].size();
  if (total >= INT32_MAX) return XAMG_ERR_SETUP;
  Ac.col.resize((size_t)total);
  Ac.val.resize((size_t)total);
  int64_t off = 0;
  for (int t = 0; t < nchunks; ++t) {
    int row = first_row[t];
    for (size_t r = 0; r < len_t[t].size(); ++r, ++row) Ac.rowptr[row + 1] = len_t[t][r];
    std::memcpy(Ac.col.data() + off, cols_t[t].data(), cols_t[t].size() * sizeof(int32_t));
    std::memcpy(Ac.val.data() + off, vals_t[t].data(), vals_t[t].size() * sizeof(double));
    off += (int64_t)cols_t[t].size();
  }
  for (int I = 0; I < nc; ++I) Ac.rowptr[I + 1] += Ac.rowptr[I];
  return XAMG_OK;
}

// SplitMix64 (Steele, Lea, Flood 2014), output number i of the generator
// seeded with 0, mapped to [-1, 1).
double counter_uniform(uint64_t i) {
  uint64_t z = (i + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// ---- step 7 ----
void chebyshev_interval(HostLevel &L, int power_iters, double hi_safety, double lo_frac, int nt) {
  const HostCsr &A = L.A;
  const int n = A.n;
  double g = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) s = s + std::fabs(A.val[p]);
    s = s * std::fabs(L.dinv[i]);
    if (s > g) g = s;
  }
  std::vector<double> v((size_t)n), w((size_t)n);
  for (int i = 0; i < n; ++i) v[i] = counter_uniform((uint64_t)i);
  double lam = 0.0;
  for (int it = 0; it < power_iters; ++it) {
    parallel_rows(n, nt, [&](int b, int e, int) {
      for (int i = b; i < e; ++i) {
        double y = 0.0;
        for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) y = y + A.val[p] * v[A.col[p]];
        w[i] = L.dinv[i] * y;
      }
    });
    double nv = 0.0, nw = 0.0;
    for (int i = 0; i < n; ++i) nv = nv + v[i] * v[i];
    for (int i = 0; i < n; ++i) nw = nw + w[i] * w[i];
    nv = std::sqrt(nv);
    nw = std::sqrt(nw);
    if (nw == 0.0 || nv == 0.0) break;
    lam = nw / nv;
    for (int i = 0; i < n; ++i) v[i] = w[i] / nw;
  }
  L.lam = lam;
  L.gersh = g;
  L.hi = hi_safety * lam;
  if (L.hi > g || lam == 0.0) L.hi = g;
  L.lo = lo_frac * L.hi;
}

// ---- step 8 ----
int dense_lu(int n, std::vector<double> &a, std::vector<int32_t> &piv) {
  piv.resize((size_t)n);
  for (int k = 0; k < n; ++k) {
    int pr = k;
    double best = std::fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      const double v = std::fabs(a[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        pr = i;
      }
    }
    piv[k] = pr;
    if (best == 0.0) return XAMG_ERR_SETUP;
    if (pr != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)pr * n + j]);
    for (int i = k + 1; i < n; ++i) {
      const double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] = a[(size_t)i * n + j] - l * a[(size_t)k * n + j];
    }
  }
  return XAMG_OK;
}

int validate(const xamg_csr &A) {
  if (A.n < 1 || !A.rowptr || !A.col || !A.val) return XAMG_ERR_INVALID_ARG;
  if (A.rowptr[0] != 0 || A.rowptr[A.n] != A.nnz || A.nnz >= INT32_MAX) return XAMG_ERR_INVALID_ARG;
  for (int i = 0; i < A.n; ++i) {
    if (A.rowptr[i + 1] < A.rowptr[i]) return XAMG_ERR_INVALID_ARG;
    bool diag = false;
    for (int p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
      if (A.col[p] < 0 || A.col[p] >= A.n) return XAMG_ERR_INVALID_ARG;
      if (p > A.rowptr[i] && A.col[p] <= A.col[p - 1]) return XAMG_ERR_INVALID_ARG;
      if (!std::isfinite(A.val[p])) return XAMG_ERR_NONFINITE;
      if (A.col[p] == i && A.val[p] != 0.0) diag = true;
    }
    if (!diag) return XAMG_ERR_INVALID_ARG;
  }
  return XAMG_OK;
}

}  // namespace

int build_hierarchy(const xamg_csr &Ain, const xamg_amg_params &prm, HostHier &h) {
  int rc = validate(Ain);
  if (rc != XAMG_OK) return rc;
  if (prm.max_levels < 1 || prm.max_levels > 40 || prm.cheb_steps < 1 || prm.cheb_steps > 4 ||
      prm.power_iters < 0 || !(prm.theta >= 0.0) || prm.max_dense < 1)
    return XAMG_ERR_INVALID_ARG;
  const int nt = thread_count(prm.nthreads);
  try {
    h.lv.clear();
    h.cheb_steps = prm.cheb_steps;
    h.lv.emplace_back();
    {
      HostCsr &A0 = h.lv[0].A;
      A0.n = A0.ncols = Ain.n;
      A0.rowptr.assign(Ain.rowptr, Ain.rowptr + Ain.n + 1);
      A0.col.assign(Ain.col, Ain.col + Ain.nnz);
      A0.val.assign(Ain.val, Ain.val + Ain.nnz);
    }
    for (int l = 0;; ++l) {
      HostLevel &L = h.lv[l];
      const int n = L.A.n;
      L.dinv.resize((size_t)n);
      for (int i = 0; i < n; ++i) {
        const double d = diag_of(L.A, i);
        if (d == 0.0) return XAMG_ERR_SETUP;
        L.dinv[i] = 1.0 / d;
      }
      if (n <= prm.max_coarse || l == prm.max_levels - 1) break;
      HostCsr S, ST;
      strength(L.A, prm.theta, S, nt);
      transpose(S, ST, false);
      split(S, ST, L.cf);
      ST = HostCsr();
      int nc = 0;
      for (int i = 0; i < n; ++i) nc += L.cf[i];
      if (nc == 0 || (double)nc > 0.9 * (double)n) {
        L.cf.clear();
        break;
      }
      if ((rc = interpolation(L.A, S, L.cf, L.P, nt)) != XAMG_OK) return rc;
      S = HostCsr();
      transpose(L.P, L.R, true);
      HostCsr Ac;
      if ((rc = galerkin(L.R, L.A, L.P, Ac, nt)) != XAMG_OK) return rc;
      h.lv.emplace_back();
      h.lv.back().A = std::move(Ac);
    }
    for (size_t l = 0; l + 1 < h.lv.size(); ++l)
      chebyshev_interval(h.lv[l], prm.power_iters, prm.cheb_hi_safety, prm.cheb_lo_frac, nt);
    const HostCsr &Ac = h.lv.back().A;
    h.nc = Ac.n;
    if (Ac.n > prm.max_dense) return XAMG_ERR_SETUP;
    h.lu.assign((size_t)Ac.n * Ac.n, 0.0);
    for (int i = 0; i < Ac.n; ++i)
      for (int p = Ac.rowptr[i]; p < Ac.rowptr[i + 1]; ++p) h.lu[(size_t)i * Ac.n + Ac.col[p]] = Ac.val[p];
    return dense_lu(Ac.n, h.lu, h.piv);
  } catch (const std::bad_alloc &) {
    return XAMG_ERR_OOM;
  }
}

}  // namespace xamg

// Host-side AMG hierarchy of the library (built once, then frozen and
// uploaded).  Internal to the library.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/xamg_gpu.h"

namespace xamg {

struct HostCsr {
  int n = 0, ncols = 0;
  std::vector<int32_t> rowptr;  // n + 1
  std::vector<int32_t> col;     // nnz, ascending per row
  std::vector<double> val;      // nnz
  int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

struct HostLevel {
  HostCsr A;                 // n x n
  HostCsr P;                 // n x n_next (empty on the coarsest level)
  HostCsr R;                 // n_next x n, R = P^T
  std::vector<int32_t> cf;   // 1 = coarse point
  std::vector<double> dinv;  // 1 / a_ii
  double lo = 0, hi = 0, lam = 0, gersh = 0;  // Chebyshev interval data
};

struct HostHier {
  std::vector<HostLevel> lv;
  int cheb_steps = 2;
  int nc = 0;                  // rows of the coarsest level
  std::vector<double> lu;      // nc x nc row-major LU factors (L unit lower)
  std::vector<int32_t> piv;    // row interchanges, piv[k] swapped with k
};

// Builds the hierarchy.  Returns an XAMG_* code.
int build_hierarchy(const xamg_csr &A, const xamg_amg_params &p, HostHier &h);

// The setup parameters and the frozen hierarchy as a byte blob, and back
// (hier_io.cpp); load_hier returns XAMG_ERR_INVALID_ARG for a blob that is
// not a complete, well-formed hierarchy of this format.
std::vector<char> save_hier(const xamg_amg_params &p, const HostHier &h);
int load_hier(const void *blob, size_t bytes, xamg_amg_params &p, HostHier &h);

}  // namespace xamg

// hier_io.cpp -- the frozen host hierarchy as a byte blob and back
// (xamg_hier_save / xamg_hier_load): the setup parameters, every level's A,
// P, R, coarse/fine flags, inverse diagonal and Chebyshev interval, and the
// coarsest LU factors.  Fields are written one by one in the host's byte
// order behind a magic string, a format version and a byte-order marker;
// loading checks every length and index against the blob and the level
// sizes, so a truncated or corrupted blob is rejected, never read past.
#include <cstring>

#include "hier_host.h"

namespace xamg {
namespace {

constexpr char kMagic[8] = {'X', 'A', 'M', 'G', 'H', 'I', 'E', 'R'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kOrder = 0x01020304u;

struct Writer {
  std::vector<char> out;
  void raw(const void *p, size_t n) {
    const char *c = static_cast<const char *>(p);
    out.insert(out.end(), c, c + n);
  }
  template <class T>
  void put(T v) {
    raw(&v, sizeof(v));
  }
  template <class T>
  void vec(const std::vector<T> &v) {
    put<uint64_t>(v.size());
    if (!v.empty()) raw(v.data(), v.size() * sizeof(T));
  }
  void csr(const HostCsr &m) {
    put<int32_t>(m.n);
    put<int32_t>(m.ncols);
    vec(m.rowptr);
    vec(m.col);
    vec(m.val);
  }
};

struct Reader {
  const char *p;
  size_t left;
  bool ok = true;
  bool raw(void *dst, size_t n) {
    if (!ok || n > left) return ok = false;
    std::memcpy(dst, p, n);
    p += n;
    left -= n;
    return true;
  }
  template <class T>
  T get() {
    T v{};
    raw(&v, sizeof(v));
    return v;
  }
  template <class T>
  bool vec(std::vector<T> &v) {
    const uint64_t n = get<uint64_t>();
    if (!ok || n > left / sizeof(T)) return ok = false;
    v.resize((size_t)n);
    return n == 0 || raw(v.data(), (size_t)n * sizeof(T));
  }
  bool csr(HostCsr &m) {
    m.n = get<int32_t>();
    m.ncols = get<int32_t>();
    return vec(m.rowptr) && vec(m.col) && vec(m.val);
  }
};

// A well-formed CSR of nrows x ncols (possibly 0 x 0): rowptr of nrows + 1
// non-decreasing offsets from 0 to nnz, columns in range.
bool csr_ok(const HostCsr &m, int nrows, int ncols) {
  if (m.n != nrows || m.ncols != ncols) return false;
  if (nrows == 0) return m.rowptr.size() <= 1 && m.col.empty() && m.val.empty();
  if (m.rowptr.size() != (size_t)nrows + 1 || m.rowptr[0] != 0) return false;
  for (int i = 0; i < nrows; ++i)
    if (m.rowptr[i + 1] < m.rowptr[i]) return false;
  const int64_t nnz = m.rowptr[nrows];
  if (m.col.size() != (size_t)nnz || m.val.size() != (size_t)nnz) return false;
  for (int32_t c : m.col)
    if (c < 0 || c >= ncols) return false;
  return true;
}

}  // namespace

std::vector<char> save_hier(const xamg_amg_params &p, const HostHier &h) {
  Writer w;
  w.raw(kMagic, sizeof(kMagic));
  w.put<uint32_t>(kVersion);
  w.put<uint32_t>(kOrder);
  w.put<double>(p.theta);
  w.put<int32_t>(p.max_coarse);
  w.put<int32_t>(p.max_levels);
  w.put<int32_t>(p.cheb_steps);
  w.put<int32_t>(p.power_iters);
  w.put<double>(p.cheb_lo_frac);
  w.put<double>(p.cheb_hi_safety);
  w.put<int32_t>(p.max_dense);
  w.put<int32_t>(p.nthreads);
  w.put<int32_t>(p.device_upload);
  w.put<uint32_t>((uint32_t)h.lv.size());
  w.put<int32_t>(h.cheb_steps);
  w.put<int32_t>(h.nc);
  for (const HostLevel &L : h.lv) {
    w.csr(L.A);
    w.csr(L.P);
    w.csr(L.R);
    w.vec(L.cf);
    w.vec(L.dinv);
    w.put<double>(L.lo);
    w.put<double>(L.hi);
    w.put<double>(L.lam);
    w.put<double>(L.gersh);
  }
  w.vec(h.lu);
  w.vec(h.piv);
  return std::move(w.out);
}

int load_hier(const void *blob, size_t bytes, xamg_amg_params &p, HostHier &h) {
  if (!blob) return XAMG_ERR_INVALID_ARG;
  Reader r{static_cast<const char *>(blob), bytes};
  char magic[8];
  if (!r.raw(magic, sizeof(magic)) || std::memcmp(magic, kMagic, sizeof(magic)) != 0)
    return XAMG_ERR_INVALID_ARG;
  if (r.get<uint32_t>() != kVersion || r.get<uint32_t>() != kOrder) return XAMG_ERR_INVALID_ARG;
  p.theta = r.get<double>();
  p.max_coarse = r.get<int32_t>();
  p.max_levels = r.get<int32_t>();
  p.cheb_steps = r.get<int32_t>();
  p.power_iters = r.get<int32_t>();
  p.cheb_lo_frac = r.get<double>();
  p.cheb_hi_safety = r.get<double>();
  p.max_dense = r.get<int32_t>();
  p.nthreads = r.get<int32_t>();
  p.device_upload = r.get<int32_t>();
  const uint32_t L = r.get<uint32_t>();
  h.cheb_steps = r.get<int32_t>();
  h.nc = r.get<int32_t>();
  if (!r.ok || L == 0 || L > 64 || h.cheb_steps < 1 || h.cheb_steps > 4) return XAMG_ERR_INVALID_ARG;
  h.lv.assign(L, HostLevel());
  for (uint32_t l = 0; l < L; ++l) {
    HostLevel &V = h.lv[l];
    if (!r.csr(V.A) || !r.csr(V.P) || !r.csr(V.R) || !r.vec(V.cf) || !r.vec(V.dinv))
      return XAMG_ERR_INVALID_ARG;
    V.lo = r.get<double>();
    V.hi = r.get<double>();
    V.lam = r.get<double>();
    V.gersh = r.get<double>();
  }
  if (!r.vec(h.lu) || !r.vec(h.piv) || r.left != 0) return XAMG_ERR_INVALID_ARG;
  // structure: level sizes chain through P (n_l x n_{l+1}) and R (the
  // transpose shape); the coarsest level has no P / R and holds the LU
  for (uint32_t l = 0; l < L; ++l) {
    const HostLevel &V = h.lv[l];
    const int n = V.A.n;
    if (n <= 0 || !csr_ok(V.A, n, n)) return XAMG_ERR_INVALID_ARG;
    // coarse / fine flags on every level but the coarsest, which has none
    const bool last = l + 1 == L;
    if (V.dinv.size() != (size_t)n || V.cf.size() != (last ? 0 : (size_t)n)) return XAMG_ERR_INVALID_ARG;
    if (l + 1 < L) {
      const int nn = h.lv[l + 1].A.n;
      if (!csr_ok(V.P, n, nn) || !csr_ok(V.R, nn, n)) return XAMG_ERR_INVALID_ARG;
      if (!(V.hi > V.lo) || !(V.lo > 0.0)) return XAMG_ERR_INVALID_ARG;
    } else if (!csr_ok(V.P, 0, 0) || !csr_ok(V.R, 0, 0)) {
      return XAMG_ERR_INVALID_ARG;
    }
  }
  const int nc = h.lv[L - 1].A.n;
  if (h.nc != nc || h.lu.size() != (size_t)nc * nc || h.piv.size() != (size_t)nc) return XAMG_ERR_INVALID_ARG;
  for (int32_t q : h.piv)
    if (q < 0 || q >= nc) return XAMG_ERR_INVALID_ARG;
  return XAMG_OK;
}

}  // namespace xamg

// Checkpoint file of a hierarchy: the operators, transfers, coordinates and
// coarse points of every level (the result of Alg. 1's graph and EMIN phases),
// so that a hierarchy can be stored and rebuilt without repeating its setup, or
// built from operators another program computed.  The layout is described with
// amg_hierarchy_export in include/emin_amg.h.  Values are written in the host's
// byte order (little-endian on every machine this library builds for).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>

#include "setup.hpp"

namespace emin {
namespace {

constexpr char kMagic[8] = {'E', 'M', 'I', 'N', 'A', 'M', 'G', '1'};
constexpr int32_t kVersion = 1;

struct FileCloser {
  void operator()(FILE* f) const {
    if (f) std::fclose(f);
  }
};
using File = std::unique_ptr<FILE, FileCloser>;

class Writer {
 public:
  explicit Writer(const std::string& path) : f_(std::fopen(path.c_str(), "wb")) {
    if (!f_) throw std::runtime_error("cannot open " + path + " for writing");
  }
  void bytes(const void* p, size_t n) {
    if (n && std::fwrite(p, 1, n, f_.get()) != n) throw std::runtime_error("write failed");
  }
  template <typename T>
  void scalar(T v) {
    bytes(&v, sizeof(T));
  }
  template <typename T>
  void array(const std::vector<T>& v) {
    bytes(v.data(), v.size() * sizeof(T));
  }
  void csr(const Csr& M) {
    scalar<int32_t>(M.nrows);
    scalar<int32_t>(M.ncols);
    scalar<int64_t>(M.nnz());
    std::vector<int64_t> rp(M.rowptr.begin(), M.rowptr.end());
    if (rp.empty()) rp.assign(M.nrows + 1, 0);
    array(rp);
    array(M.col);
    array(M.val);
  }
  void close() {
    if (std::fclose(f_.release()) != 0) throw std::runtime_error("closing the checkpoint file failed");
  }

 private:
  File f_;
};

class Reader {
 public:
  explicit Reader(const std::string& path) : f_(std::fopen(path.c_str(), "rb")), path_(path) {
    if (!f_) throw std::runtime_error("cannot open " + path);
  }
  void bytes(void* p, size_t n) {
    if (n && std::fread(p, 1, n, f_.get()) != n) throw std::runtime_error(path_ + ": truncated file");
  }
  template <typename T>
  T scalar() {
    T v;
    bytes(&v, sizeof(T));
    return v;
  }
  template <typename T>
  std::vector<T> array(int64_t n, const char* what) {
    if (n < 0 || n > (int64_t(1) << 40)) throw std::runtime_error(path_ + ": bad length of " + what);
    std::vector<T> v((size_t)n);
    bytes(v.data(), v.size() * sizeof(T));
    return v;
  }
  // A CSR block of the given shape (ncols < 0: any column count): row pointers from
  // 0, nondecreasing, ending at nnz; columns strictly ascending within a row and
  // inside [0, ncols).
  Csr csr(int nrows, int ncols, const char* what) {
    const int32_t r = scalar<int32_t>(), c = scalar<int32_t>();
    const int64_t nnz = scalar<int64_t>();
    if (ncols < 0 && c >= 0) ncols = c;
    if (r != nrows || c != ncols)
      throw std::runtime_error(path_ + ": " + what + " is " + std::to_string(r) + " x " + std::to_string(c) +
                               ", expected " + std::to_string(nrows) + " x " + std::to_string(ncols));
    Csr M;
    M.nrows = nrows;
    M.ncols = ncols;
    M.rowptr = array<int64_t>((int64_t)nrows + 1, what);
    M.col = array<int>(nnz, what);
    M.val = array<double>(nnz, what);
    if (M.rowptr[0] != 0 || M.rowptr[nrows] != nnz) throw std::runtime_error(path_ + ": " + what + ": bad row pointers");
    for (int i = 0; i < nrows; ++i) {
      if (M.rowptr[i + 1] < M.rowptr[i]) throw std::runtime_error(path_ + ": " + what + ": row pointers decrease");
      for (int64_t t = M.rowptr[i]; t < M.rowptr[i + 1]; ++t) {
        if (M.col[t] < 0 || M.col[t] >= ncols) throw std::runtime_error(path_ + ": " + what + ": column out of range");
        if (t > M.rowptr[i] && M.col[t] <= M.col[t - 1])
          throw std::runtime_error(path_ + ": " + what + ": columns not strictly ascending");
      }
    }
    return M;
  }

 private:
  File f_;
  std::string path_;
};

}  // namespace

void write_hierarchy(const std::vector<HostLevel>& levels, bool symmetric, const std::string& path) {
  Writer w(path);
  w.bytes(kMagic, sizeof(kMagic));
  w.scalar<int32_t>(kVersion);
  w.scalar<int32_t>((int32_t)levels.size());
  w.scalar<int32_t>(symmetric ? 1 : 0);
  for (size_t l = 0; l < levels.size(); ++l) {
    const HostLevel& L = levels[l];
    w.scalar<int32_t>(L.dim);
    w.scalar<int32_t>(L.n_v);
    w.scalar<int32_t>(L.n_p);
    w.scalar<int32_t>(L.pinned);
    w.csr(L.A);
    w.csr(L.B);
    w.csr(L.Bt);
    w.array(L.vX);
    w.array(L.pX);
    w.array(L.p2v);
    w.array(L.dirichlet);
    if (l + 1 < levels.size()) {
      w.csr(L.P);
      w.csr(L.Pp);
      w.csr(L.R);
      w.csr(L.Rp);
      w.scalar<int32_t>((int32_t)L.Cp.size());
      w.array(L.Cp);
      w.scalar<int32_t>((int32_t)L.Cv.size());
      w.array(L.Cv);
    }
  }
  w.close();
}

std::vector<HostLevel> read_hierarchy(const std::string& path, bool* symmetric) {
  Reader r(path);
  char magic[8];
  r.bytes(magic, sizeof(magic));
  if (std::memcmp(magic, kMagic, sizeof(magic)) != 0) throw std::runtime_error(path + ": not a hierarchy checkpoint");
  const int32_t version = r.scalar<int32_t>();
  if (version != kVersion) throw std::runtime_error(path + ": unsupported checkpoint version " + std::to_string(version));
  const int32_t nlev = r.scalar<int32_t>();
  const int32_t sym = r.scalar<int32_t>();
  if (nlev < 1 || nlev > 64) throw std::runtime_error(path + ": bad number of levels");
  if (symmetric) *symmetric = sym != 0;
  std::vector<HostLevel> levels((size_t)nlev);
  for (int l = 0; l < nlev; ++l) {
    HostLevel& L = levels[l];
    L.dim = r.scalar<int32_t>();
    L.n_v = r.scalar<int32_t>();
    L.n_p = r.scalar<int32_t>();
    L.pinned = r.scalar<int32_t>();
    if (L.dim < 2 || L.dim > 3 || L.n_v < 0 || L.n_p < 1 || L.pinned < -1 || L.pinned >= L.n_p)
      throw std::runtime_error(path + ": bad sizes on level " + std::to_string(l));
    if (l > 0) {
      const HostLevel& F = levels[l - 1];
      if (L.dim != F.dim || L.n_v != F.P.ncols || L.n_p != F.Pp.ncols)
        throw std::runtime_error(path + ": level " + std::to_string(l) + " does not match the transfers above it");
    }
    const int nu = L.dim * L.n_v;
    L.A = r.csr(L.n_v, L.n_v, "A");
    L.B = r.csr(L.n_p, nu, "B");
    L.Bt = r.csr(nu, L.n_p, "Bt");
    L.vX = r.array<double>((int64_t)L.n_v * L.dim, "velocity coordinates");
    L.pX = r.array<double>((int64_t)L.n_p * L.dim, "pressure coordinates");
    L.p2v = r.array<int>(L.n_p, "p2v");
    L.dirichlet = r.array<unsigned char>(L.n_v, "Dirichlet mask");
    for (int v : L.p2v)
      if (v < -1 || v >= L.n_v) throw std::runtime_error(path + ": p2v out of range");
    if (l + 1 < nlev) {
      // the transfers' column counts are the next level's sizes, checked when it is read
      L.P = r.csr(L.n_v, -1, "P");
      L.Pp = r.csr(L.n_p, -1, "Pp");
      const int nvc = L.P.ncols;
      L.R = r.csr(nvc, L.n_v, "R");
      L.Rp = r.csr(L.Pp.ncols, L.n_p, "Rp");
      const int32_t ncp = r.scalar<int32_t>();
      L.Cp = r.array<int>(ncp, "Cp");
      const int32_t ncv = r.scalar<int32_t>();
      L.Cv = r.array<int>(ncv, "Cv");
      if (ncp != L.Pp.ncols || ncv != nvc) throw std::runtime_error(path + ": coarse point counts differ from P's");
      for (int c : L.Cp)
        if (c < 0 || c >= L.n_p) throw std::runtime_error(path + ": coarse pressure out of range");
      for (int c : L.Cv)
        if (c < 0 || c >= L.n_v) throw std::runtime_error(path + ": coarse velocity out of range");
    }
  }
  return levels;
}

}  // namespace emin

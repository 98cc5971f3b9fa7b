// Numeric hierarchy setup on the GPU (see gpu_setup.hpp).
#include "gpu_setup.hpp"
#include "trace.hpp"

#include <algorithm>
#include <cstdint>
#include <stdexcept>
#include <string>

namespace emin {
namespace {

#define SETUP_CUDA(call)                                                                \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw std::runtime_error(std::string("cuda (device setup): ") + #call + ": " +   \
                               cudaGetErrorString(e_));                                 \
  } while (0)

constexpr int kThreads = 256;
constexpr int kDotBlocks = 304;  // 2 per SM on 152 SMs

unsigned blocks_for(long long n) { return (unsigned)std::max<long long>(1, (n + kThreads - 1) / kThreads); }

// ---------------------------------------------------------------------------
// Kernels.  Rows use int64 offsets and int32 columns, as the host's Csr.

// C = A B on C's pattern, one warp per row of C, lanes over the row's entries:
// C_ij = sum over k (ascending) of A_ik B_kj, a merge of row i of A with column j
// of B.  B's columns are given in compressed-column form (bcp, bri); the value of
// the entry at column position q is bv[bperm[q]] (bv[q] when bperm is null).
__global__ void k_spgemm_pattern(int nrows, const int64_t* __restrict__ arp, const int* __restrict__ aci,
                                 const double* __restrict__ av, const int64_t* __restrict__ bcp,
                                 const int* __restrict__ bri, const int64_t* __restrict__ bperm,
                                 const double* __restrict__ bv, const int64_t* __restrict__ crp,
                                 const int* __restrict__ cci, double* __restrict__ cv) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nrows) return;
  const int64_t a0 = arp[warp], a1 = arp[warp + 1];
  for (int64_t t = crp[warp] + lane; t < crp[warp + 1]; t += 32) {
    const int j = cci[t];
    int64_t p = a0, q = bcp[j];
    const int64_t qe = bcp[j + 1];
    double acc = 0.0;
    while (p < a1 && q < qe) {
      const int ka = aci[p], kb = bri[q];
      if (ka == kb) {
        acc += av[p] * bv[bperm ? bperm[q] : q];
        ++p;
        ++q;
      } else if (ka < kb) {
        ++p;
      } else {
        ++q;
      }
    }
    cv[t] = acc;
  }
}

// Braess-Sarazin diagonal (Section 5.2): D_i = sum_j |A_ij|, 1/c on Dirichlet rows.
__global__ void k_abs_row_sums(int n, const int64_t* __restrict__ rp, const double* __restrict__ v,
                               const unsigned char* __restrict__ dirichlet, double inv_c, double* __restrict__ D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t t = rp[i]; t < rp[i + 1]; ++t) s += fabs(v[t]);
  D[i] = dirichlet[i] ? inv_c : s;
}

// B D^-1: every entry of B divided by D of its column's velocity node.
__global__ void k_scale_columns(long long nnz, const int* __restrict__ ci, const double* __restrict__ v, int n_v,
                                const double* __restrict__ D, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  out[t] = v[t] * (1.0 / D[ci[t] % n_v]);
}

// The diagonal of a square matrix (0 where not stored).
__global__ void k_diagonal(int n, const int64_t* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ v, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
    if (ci[t] == i) s += v[t];
  d[i] = s;
}

// eq. e:filtering on the matrix's own pattern: an off-diagonal entry with
// |z_ij| <= tau sqrt(|z_ii z_jj|) becomes 0 and its value is added to the
// diagonal (row sums kept).  One thread per row, the row's dropped values summed
// in column order.
__global__ void k_filter_lump(int n, const int64_t* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ z, const double* __restrict__ d, double tau,
                              double* __restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double lump = 0.0;
  int64_t diag = -1;
  for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
    const int j = ci[t];
    if (j == i) {
      diag = t;
      continue;
    }
    const double v = z[t];
    if (fabs(v) <= tau * sqrt(fabs(d[i] * d[j]))) {
      lump += v;
      f[t] = 0.0;
    } else {
      f[t] = v;
    }
  }
  if (diag >= 0) f[diag] = d[i] + lump;
}

// EMIN initial guess (Section 4.3): the pattern divided by its row count.
__global__ void k_pattern_average(int n, const int64_t* __restrict__ rp, double* __restrict__ p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = rp[i], e = rp[i + 1];
  for (int64_t t = b; t < e; ++t) p[t] = 1.0 / (double)(e - b);
}

// Orthogonal projection onto {pattern, zero row sums} (each row minus its mean
// over the pattern), times sign.
__global__ void k_project_rows(int n, const int64_t* __restrict__ rp, const double* __restrict__ g, double sign,
                               double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = rp[i], e = rp[i + 1];
  if (b == e) return;
  double s = 0.0;
  for (int64_t t = b; t < e; ++t) s += g[t];
  const double mean = s / (double)(e - b);
  for (int64_t t = b; t < e; ++t) out[t] = sign * (g[t] - mean);
}

// Deterministic dot product: per-block partial sums in a fixed order, then one
// block adds the partials in a fixed order.
__global__ void k_dot_partial(long long n, const double* __restrict__ x, const double* __restrict__ y,
                              double* __restrict__ part) {
  __shared__ double sm[kThreads / 32];
  double s = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    s += x[t] * y[t];
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) b += sm[w];
    part[blockIdx.x] = b;
  }
}

// (one warp)
__global__ void k_dot_final(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += 32) s += part[b];
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (threadIdx.x == 0) *out = s;
}

// alpha = num / den (0 when den = 0), then p = p0 + alpha r on the pattern.
__global__ void k_emin_update(long long nnz, const double* __restrict__ num, const double* __restrict__ den,
                              const double* __restrict__ p0, const double* __restrict__ r, double* __restrict__ p) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  const double alpha = *den != 0.0 ? *num / *den : 0.0;
  p[t] = p0[t] + alpha * r[t];
}

// dst[t] = src[map[t]]: values of a transposed or replicated pattern.
__global__ void k_gather(long long n, const int64_t* __restrict__ map, const double* __restrict__ src,
                         double* __restrict__ dst) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  dst[t] = src[map[t]];
}

// The pinned pressure's row of S is the identity row (its update is exact).
__global__ void k_pin_row(const int64_t* __restrict__ rp, const int* __restrict__ ci, int pinned, double* __restrict__ v) {
  for (int64_t t = rp[pinned]; t < rp[pinned + 1]; ++t) v[t] = ci[t] == pinned ? 1.0 : 0.0;
}

// One (strip parity, color) group of the dense Gauss-Seidel map M (n x n,
// row-major): for every row i of the group and every column q,
// M_iq = (delta_iq - sum_{j != i} S_ij M_jq) / S_ii.  The rows of a group share no
// entry of S, so they are independent; blockIdx.y picks the row, the threads the
// columns.
__global__ void k_dense_gs_group(int n, const int* __restrict__ rows, const int64_t* __restrict__ rp,
                                 const int* __restrict__ ci, const double* __restrict__ sv, double* __restrict__ M) {
  const int i = rows[blockIdx.y];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double acc = (q == i) ? 1.0 : 0.0, diag = 0.0;
  for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
    const int j = ci[t];
    if (j == i) {
      diag += sv[t];
      continue;
    }
    acc -= sv[t] * M[(size_t)j * n + q];
  }
  M[(size_t)i * n + q] = diag != 0.0 ? acc * (1.0 / diag) : 0.0;
}

// ---------------------------------------------------------------------------
// Host side: device memory, patterns and compressed-column maps.

// Device allocations released together.
struct Arena {
  std::vector<void*> ptrs;
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  ~Arena() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it for the next launch checks
      throw std::runtime_error(std::string("cudaMalloc (device setup): ") + cudaGetErrorString(e));
    }
    ptrs.push_back(p);
    return (T*)p;
  }
  template <typename T>
  T* copy(const std::vector<T>& h) {
    T* d = alloc<T>(h.size());
    if (!h.empty()) SETUP_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
  }
};

// A sparsity pattern on the device.
struct DPat {
  int nrows = 0, ncols = 0;
  int64_t nnz = 0;
  const int64_t* rp = nullptr;
  const int* ci = nullptr;
};
// Compressed-column view of a pattern: column j's entries are rows ri[cp[j]..cp[j+1])
// (ascending) at row-major positions perm[...] (null: the row-major order itself).
struct DCsc {
  const int64_t* cp = nullptr;
  const int* ri = nullptr;
  const int64_t* perm = nullptr;
};

DPat upload_pattern(Arena& a, const Csr& M) {
  DPat d;
  d.nrows = M.nrows;
  d.ncols = M.ncols;
  d.nnz = M.nnz();
  std::vector<int64_t> rp(M.rowptr.begin(), M.rowptr.end());
  if (rp.empty()) rp.assign(M.nrows + 1, 0);
  d.rp = a.copy(rp);
  d.ci = a.copy(M.col);
  return d;
}

// Compressed columns of a pattern: counting sort of the entries by column, rows
// ascending within a column.
DCsc upload_csc(Arena& a, const Csr& M) {
  std::vector<int64_t> cp(M.ncols + 1, 0), perm(M.nnz());
  std::vector<int> ri(M.nnz());
  for (int64_t t = 0; t < M.nnz(); ++t) cp[M.col[t] + 1]++;
  for (int j = 0; j < M.ncols; ++j) cp[j + 1] += cp[j];
  std::vector<int64_t> pos(cp.begin(), cp.end() - 1);
  for (int i = 0; i < M.nrows; ++i)
    for (int64_t t = M.rowptr[i]; t < M.rowptr[i + 1]; ++t) {
      const int64_t q = pos[M.col[t]]++;
      ri[q] = i;
      perm[q] = t;
    }
  DCsc d;
  d.cp = a.copy(cp);
  d.ri = a.copy(ri);
  d.perm = a.copy(perm);
  return d;
}

// The transposed pattern as a row-major pattern (its rows are M's columns) with
// the gather map from M's positions.
DPat transposed_pattern(const DPat& M, const DCsc& c) {
  DPat t;
  t.nrows = M.ncols;
  t.ncols = M.nrows;
  t.nnz = M.nnz;
  t.rp = c.cp;
  t.ci = c.ri;
  return t;
}

// I_d (x) M as a pattern, with the map from its positions to M's.
Csr kron_pattern(int d, const Csr& M, std::vector<int64_t>& map) {
  Csr K = kron_identity(d, M);
  map.resize(K.nnz());
  int64_t q = 0;
  for (int c = 0; c < d; ++c)
    for (int64_t t = 0; t < M.nnz(); ++t) map[q++] = t;
  return K;
}

// Pattern of a product, computed once per structure on the host.
Csr product_pattern(const Csr& A, const Csr& B) { return spgemm(A, B); }

}  // namespace

// Per level: the patterns of every operand and product of the numeric setup, and
// the compressed-column maps of the right factors.
struct DeviceSetupPlan {
  struct Level {
    int dim = 2, n_v = 0, n_p = 0, pinned = -1;
    DPat A, B, Bt, S, Z;
    DCsc A_csc, Bt_csc, Z_csc;
    const unsigned char* dirichlet = nullptr;
    // transfers and Galerkin products (all but the coarsest level)
    DPat P, Pp, R, Rp, Pv, Rv, RA, RpB, RvBt;
    DCsc B_csc, P_csc, Pp_csc, Pv_csc;
    const int64_t* pv_map = nullptr;  // Pv position -> P position
    const int64_t* rv_map = nullptr;  // Rv position -> R position
  };
  Arena mem;
  std::vector<Level> levels;
  bool symmetric = true;
  int device = -1;
};

namespace {

std::shared_ptr<DeviceSetupPlan> make_plan(const std::vector<HostLevel>& H, bool symmetric) {
  auto plan = std::make_shared<DeviceSetupPlan>();
  SETUP_CUDA(cudaGetDevice(&plan->device));
  plan->symmetric = symmetric;
  Arena& a = plan->mem;
  plan->levels.resize(H.size());
  for (size_t l = 0; l < H.size(); ++l) {
    const HostLevel& L = H[l];
    DeviceSetupPlan::Level& P = plan->levels[l];
    P.dim = L.dim;
    P.n_v = L.n_v;
    P.n_p = L.n_p;
    P.pinned = L.pinned;
    P.A = upload_pattern(a, L.A);
    P.B = upload_pattern(a, L.B);
    P.Bt = upload_pattern(a, L.Bt);
    P.S = upload_pattern(a, L.S);
    P.Bt_csc = upload_csc(a, L.Bt);
    P.dirichlet = a.copy(L.dirichlet);
    if (l + 1 == H.size()) continue;
    const Csr Z = product_pattern(L.B, transpose(L.B));
    P.Z = upload_pattern(a, Z);
    P.Z_csc = upload_csc(a, Z);
    P.A_csc = upload_csc(a, L.A);
    P.B_csc = upload_csc(a, L.B);
    P.P = upload_pattern(a, L.P);
    P.Pp = upload_pattern(a, L.Pp);
    P.R = upload_pattern(a, L.R);
    P.Rp = upload_pattern(a, L.Rp);
    P.P_csc = upload_csc(a, L.P);
    P.Pp_csc = upload_csc(a, L.Pp);
    std::vector<int64_t> pmap, rmap;
    const Csr Pv = kron_pattern(L.dim, L.P, pmap), Rv = kron_pattern(L.dim, L.R, rmap);
    P.Pv = upload_pattern(a, Pv);
    P.Rv = upload_pattern(a, Rv);
    P.Pv_csc = upload_csc(a, Pv);
    P.pv_map = a.copy(pmap);
    P.rv_map = a.copy(rmap);
    P.RA = upload_pattern(a, product_pattern(L.R, L.A));
    P.RpB = upload_pattern(a, product_pattern(L.Rp, L.B));
    P.RvBt = upload_pattern(a, product_pattern(Rv, L.Bt));
  }
  return plan;
}

// The numeric kernels' launches on one stream, with scratch from an arena.
struct Launcher {
  Arena& w;
  cudaStream_t s;
  double* part;  // kDotBlocks partial sums
  Launcher(Arena& a, cudaStream_t st) : w(a), s(st), part(a.alloc<double>(kDotBlocks)) {}

  double* vec(int64_t n) { return w.alloc<double>((size_t)n); }
  // C = A B on C's pattern (B given by its compressed columns and row-major values)
  void spgemm(const DPat& A, const double* av, const DCsc& B, const double* bv, const DPat& C, double* cv) {
    if (C.nrows == 0) return;
    k_spgemm_pattern<<<blocks_for((long long)C.nrows * 32), kThreads, 0, s>>>(C.nrows, A.rp, A.ci, av, B.cp, B.ri,
                                                                               B.perm, bv, C.rp, C.ci, cv);
    SETUP_CUDA(cudaGetLastError());
  }
  void gather(int64_t n, const int64_t* map, const double* src, double* dst) {
    if (n == 0) return;
    k_gather<<<blocks_for(n), kThreads, 0, s>>>(n, map, src, dst);
    SETUP_CUDA(cudaGetLastError());
  }
  void dot(int64_t n, const double* x, const double* y, double* out) {
    k_dot_partial<<<kDotBlocks, kThreads, 0, s>>>(n, x, y, part);
    k_dot_final<<<1, 32, 0, s>>>(kDotBlocks, part, out);
    SETUP_CUDA(cudaGetLastError());
  }
  void filter(const DPat& M, const double* mv, double tau, double* out) {
    double* d = vec(M.nrows);
    k_diagonal<<<blocks_for(M.nrows), kThreads, 0, s>>>(M.nrows, M.rp, M.ci, mv, d);
    k_filter_lump<<<blocks_for(M.nrows), kThreads, 0, s>>>(M.nrows, M.rp, M.ci, mv, d, tau, out);
    SETUP_CUDA(cudaGetLastError());
  }
  // One EMIN step (Section 4.3) for the energy matrix At on the pattern N: P0 =
  // pattern / row count, R0 = -Proj(At P0); CG: alpha = <R0,R0> / <R0, At R0>;
  // GMRES: Q = Proj(At R0), alpha = <R0,Q> / <Q,Q>; out = P0 + alpha R0.
  void emin(const DPat& At, const double* atv, const DPat& N, const DCsc& Ncsc, bool cg, double* out) {
    double* p0 = vec(N.nnz);
    double* g = vec(N.nnz);
    double* r0 = vec(N.nnz);
    double* w2 = vec(N.nnz);
    double* nd = vec(2);
    k_pattern_average<<<blocks_for(N.nrows), kThreads, 0, s>>>(N.nrows, N.rp, p0);
    spgemm(At, atv, Ncsc, p0, N, g);
    k_project_rows<<<blocks_for(N.nrows), kThreads, 0, s>>>(N.nrows, N.rp, g, -1.0, r0);
    spgemm(At, atv, Ncsc, r0, N, w2);
    if (cg) {
      dot(N.nnz, r0, r0, nd);
      dot(N.nnz, r0, w2, nd + 1);
    } else {
      double* q = vec(N.nnz);
      k_project_rows<<<blocks_for(N.nrows), kThreads, 0, s>>>(N.nrows, N.rp, w2, 1.0, q);
      dot(N.nnz, r0, q, nd);
      dot(N.nnz, q, q, nd + 1);
    }
    if (N.nnz) k_emin_update<<<blocks_for(N.nnz), kThreads, 0, s>>>(N.nnz, nd, nd + 1, p0, r0, out);
    SETUP_CUDA(cudaGetLastError());
  }
};

void download(const double* d, std::vector<double>& h, cudaStream_t s) {
  if (!h.empty()) SETUP_CUDA(cudaMemcpyAsync(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
}

}  // namespace

std::vector<HostLevel> build_hierarchy_reuse_device(HostLevel fine, const std::vector<HostLevel>& prev,
                                                    const SetupParams& prm, std::shared_ptr<DeviceSetupPlan>& plan,
                                                    cudaStream_t s) {
  const HostLevel& F0 = prev.at(0);
  if (fine.dim != F0.dim || fine.n_v != F0.n_v || fine.n_p != F0.n_p || fine.pinned != F0.pinned ||
      fine.A.rowptr != F0.A.rowptr || fine.A.col != F0.A.col || fine.B.rowptr != F0.B.rowptr ||
      fine.B.col != F0.B.col)
    throw std::runtime_error("reused hierarchy does not match the problem's structure");
  int dev = -1;
  SETUP_CUDA(cudaGetDevice(&dev));
  if (!plan || plan->device != dev || plan->levels.size() != prev.size() || plan->symmetric != prm.symmetric) {
    TraceRange r("device setup: patterns and maps of the structure");
    plan = make_plan(prev, prm.symmetric);
  }
  TraceRange range("device setup: numeric (filtering, EMIN, R, RAP, S)");
  const size_t nl = prev.size();
  const double tau = prm.tau1_for(fine.dim);
  Arena work;
  Launcher K(work, s);
  // per level: values of A, B, Bt (the level's operator), D, S, and the transfers
  struct Vals {
    double *A = nullptr, *B = nullptr, *Bt = nullptr, *D = nullptr, *S = nullptr;
    double *P = nullptr, *Pp = nullptr, *R = nullptr, *Rp = nullptr;
  };
  std::vector<Vals> v(nl);
  v[0].A = work.copy(fine.A.val);
  v[0].B = work.copy(fine.B.val);
  v[0].Bt = work.copy(fine.Bt.val);
  for (size_t l = 0; l < nl; ++l) {
    const DeviceSetupPlan::Level& P = plan->levels[l];
    Vals& V = v[l];
    // Braess-Sarazin data (Section 5.2): D, B D^-1 and S = B D^-1 Bt
    V.D = K.vec(P.n_v);
    k_abs_row_sums<<<blocks_for(P.n_v), kThreads, 0, s>>>(P.n_v, P.A.rp, V.A, P.dirichlet, 1.0 / prm.c, V.D);
    double* bd = K.vec(P.B.nnz);
    if (P.B.nnz) k_scale_columns<<<blocks_for(P.B.nnz), kThreads, 0, s>>>(P.B.nnz, P.B.ci, V.B, P.n_v, V.D, bd);
    V.S = K.vec(P.S.nnz);
    K.spgemm(P.B, bd, P.Bt_csc, V.Bt, P.S, V.S);
    if (P.pinned >= 0) k_pin_row<<<1, 1, 0, s>>>(P.S.rp, P.S.ci, P.pinned, V.S);
    SETUP_CUDA(cudaGetLastError());
    if (l + 1 == nl) break;
    // filtered auxiliary matrices (eq. e:filtering): B B^T for pressures, A for velocities
    double* z = K.vec(P.Z.nnz);
    K.spgemm(P.B, V.B, DCsc{P.B.rp, P.B.ci, nullptr}, V.B, P.Z, z);
    double* ap = K.vec(P.Z.nnz);
    double* av = K.vec(P.A.nnz);
    K.filter(P.Z, z, tau, ap);
    K.filter(P.A, V.A, tau, av);
    // EMIN (Section 4.3) and restriction: R = P^T (Stokes) or EMIN on the transposed
    // operators with the transposed pattern (Oseen, Petrov-Galerkin)
    V.P = K.vec(P.P.nnz);
    V.Pp = K.vec(P.Pp.nnz);
    V.R = K.vec(P.R.nnz);
    V.Rp = K.vec(P.Rp.nnz);
    K.emin(P.Z, ap, P.Pp, P.Pp_csc, prm.symmetric, V.Pp);
    K.emin(P.A, av, P.P, P.P_csc, prm.symmetric, V.P);
    if (prm.symmetric) {
      K.gather(P.R.nnz, P.P_csc.perm, V.P, V.R);
      K.gather(P.Rp.nnz, P.Pp_csc.perm, V.Pp, V.Rp);
    } else {
      double* avt = K.vec(P.A.nnz);
      double* apt = K.vec(P.Z.nnz);
      K.gather(P.A.nnz, P.A_csc.perm, av, avt);
      K.gather(P.Z.nnz, P.Z_csc.perm, ap, apt);
      double* rt = K.vec(P.P.nnz);
      double* rpt = K.vec(P.Pp.nnz);
      K.emin(transposed_pattern(P.A, P.A_csc), avt, P.P, P.P_csc, false, rt);
      K.emin(transposed_pattern(P.Z, P.Z_csc), apt, P.Pp, P.Pp_csc, false, rpt);
      K.gather(P.R.nnz, P.P_csc.perm, rt, V.R);
      K.gather(P.Rp.nnz, P.Pp_csc.perm, rpt, V.Rp);
    }
    // Petrov-Galerkin product, block by block (Alg. 1): A_c = R A P,
    // B_c = Rp B (I (x) P), Bt_c = (I (x) R) Bt Pp
    const DeviceSetupPlan::Level& C = plan->levels[l + 1];
    Vals& W = v[l + 1];
    double* pv = K.vec(P.Pv.nnz);
    double* rv = K.vec(P.Rv.nnz);
    K.gather(P.Pv.nnz, P.pv_map, V.P, pv);
    K.gather(P.Rv.nnz, P.rv_map, V.R, rv);
    double* ra = K.vec(P.RA.nnz);
    double* rpb = K.vec(P.RpB.nnz);
    double* rvbt = K.vec(P.RvBt.nnz);
    W.A = K.vec(C.A.nnz);
    W.B = K.vec(C.B.nnz);
    W.Bt = K.vec(C.Bt.nnz);
    K.spgemm(P.R, V.R, P.A_csc, V.A, P.RA, ra);
    K.spgemm(P.RA, ra, P.P_csc, V.P, C.A, W.A);
    K.spgemm(P.Rp, V.Rp, P.B_csc, V.B, P.RpB, rpb);
    K.spgemm(P.RpB, rpb, P.Pv_csc, pv, C.B, W.B);
    K.spgemm(P.Rv, rv, P.Bt_csc, V.Bt, P.RvBt, rvbt);
    K.spgemm(P.RvBt, rvbt, P.Pp_csc, V.Pp, C.Bt, W.Bt);
  }
  // the levels: prev's patterns, coarse points and Gauss-Seidel order; the new values
  std::vector<HostLevel> out(nl);
  out[0] = std::move(fine);
  for (size_t l = 0; l < nl; ++l) {
    const HostLevel& H = prev[l];
    HostLevel& L = out[l];
    if (l > 0) {
      const HostLevel& U = out[l - 1];
      L.dim = H.dim;
      L.n_v = H.n_v;
      L.n_p = H.n_p;
      L.pinned = -1;
      L.A = H.A;
      L.B = H.B;
      L.Bt = H.Bt;
      download(v[l].A, L.A.val, s);
      download(v[l].B, L.B.val, s);
      download(v[l].Bt, L.Bt.val, s);
      // project_coordinates (injection) and the coarse co-location map
      L.vX.resize((size_t)L.n_v * L.dim);
      L.pX.resize((size_t)L.n_p * L.dim);
      for (int t = 0; t < L.n_v; ++t)
        for (int k = 0; k < L.dim; ++k) L.vX[(size_t)t * L.dim + k] = U.vX[(size_t)U.Cv[t] * L.dim + k];
      for (int t = 0; t < L.n_p; ++t)
        for (int k = 0; k < L.dim; ++k) L.pX[(size_t)t * L.dim + k] = U.pX[(size_t)U.Cp[t] * L.dim + k];
      L.p2v = H.p2v;
      L.dirichlet.assign(L.n_v, 0);
    }
    L.D.assign(L.n_v, 0.0);
    download(v[l].D, L.D, s);
    L.S = H.S;
    download(v[l].S, L.S.val, s);
    L.colors = H.colors;
    L.n_colors = H.n_colors;
    L.gs_strip = H.gs_strip;
    if (l + 1 < nl) {
      L.Cp = H.Cp;
      L.Cv = H.Cv;
      L.P = H.P;
      L.Pp = H.Pp;
      L.R = H.R;
      L.Rp = H.Rp;
      download(v[l].P, L.P.val, s);
      download(v[l].Pp, L.Pp.val, s);
      download(v[l].R, L.R.val, s);
      download(v[l].Rp, L.Rp.val, s);
    }
  }
  SETUP_CUDA(cudaStreamSynchronize(s));
  return out;
}

void form_dense_gs_device(std::vector<HostLevel>& levels, int iters, cudaStream_t s) {
  TraceRange range("device setup: dense Gauss-Seidel maps");
  for (size_t l = 0; l + 1 < levels.size(); ++l) {
    HostLevel& L = levels[l];
    if (L.n_p > kGsDenseMaxRows) continue;
    const int n = L.n_p, T = L.gs_strip, ncol = L.n_colors;
    const int nstrips = std::max(1, (n + T - 1) / T);
    // rows in relaxation order, grouped by (strip parity, color): a group's rows
    // share no entry of S
    std::vector<int> order, goff(1, 0);
    order.reserve(n);
    for (int par = 0; par < 2; ++par)
      for (int c = 0; c < ncol; ++c) {
        for (int st = par; st < nstrips; st += 2)
          for (int i = st * T; i < std::min(n, (st + 1) * T); ++i)
            if (L.colors[i] == c) order.push_back(i);
        goff.push_back((int)order.size());
      }
    Arena a;
    const DPat S = upload_pattern(a, L.S);
    const double* sv = a.copy(L.S.val);
    const int* rows = a.copy(order);
    double* M = a.alloc<double>((size_t)n * n);
    SETUP_CUDA(cudaMemsetAsync(M, 0, sizeof(double) * (size_t)n * n, s));
    for (int it = 0; it < iters; ++it)
      for (size_t g = 0; g + 1 < goff.size(); ++g) {
        const int cnt = goff[g + 1] - goff[g];
        if (cnt == 0) continue;
        k_dense_gs_group<<<dim3(blocks_for(n), cnt), kThreads, 0, s>>>(n, rows + goff[g], S.rp, S.ci, sv, M);
      }
    SETUP_CUDA(cudaGetLastError());
    L.gs_dense.assign((size_t)n * n, 0.0);
    download(M, L.gs_dense, s);
    SETUP_CUDA(cudaStreamSynchronize(s));
  }
}

}  // namespace emin

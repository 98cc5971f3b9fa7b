// C ABI (include/emin_amg.h): hierarchy creation, V-cycle application and the
// flexible GMRES driver with its FP64 Arnoldi / Givens kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "gpu_setup.hpp"
#include "hierarchy.hpp"
#include "trace.hpp"

using namespace emin;

namespace {

thread_local std::string g_last_error;

amg_status fail(amg_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

// ---------------------------------------------------------------------------
// FGMRES kernels (FP64).  Vectors are N x K interleaved; a block of basis
// vectors is nv consecutive vectors of N*K entries.

constexpr int kRedBlocks = 608;  // 4 blocks per SM on 152 SMs for the streaming reductions

// Blocks of a streaming reduction over NK entries: one entry per thread at most,
// and at most kRedBlocks (small problems: few partial sums to combine).
inline int red_blocks(long long NK) {
  const long long b = (NK + kBlock - 1) / kBlock;
  return (int)std::max(1LL, std::min<long long>(kRedBlocks, b));
}

// Second grid dimension of the inner products: when the entries fill fewer blocks
// than the SMs, the basis vectors are split over blockIdx.y too, so the FP64 work
// (slow on this GPU's FP64 pipe) spreads over more SMs.
inline int dot_split(int rb, int nd) { return std::max(1, std::min(nd, kRedBlocks / 4 / rb)); }

// part[(blk*nd + i)*K + k] = sum over this block's entries with rhs k of V_i[e] * w[e],
// for i < nv, plus w[e]^2 at i = nv when self is set (nd = nv + self); blk is
// blockIdx.x, and blockIdx.y takes every gridDim.y-th i.  Nothing is done when cond
// is given and *cond == 0.
template <int K, typename TV>
__global__ void __launch_bounds__(kBlock) k_mdot_partial(long long NK, int nv, int self, const TV* __restrict__ V,
                                                         const double* __restrict__ w, double* __restrict__ part,
                                                         const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  __shared__ double sm[kBlock / 32][K];
  const int k = threadIdx.x % K;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int nd = nv + self;
  for (int i = blockIdx.y; i < nd; i += gridDim.y) {
    double acc = 0.0;
    if (i < nv) {
      const TV* Vi = V + (size_t)i * NK;
      for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < NK; e += stride)
        acc += (double)Vi[e] * w[e];
    } else {
      for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < NK; e += stride) acc += w[e] * w[e];
    }
#pragma unroll
    for (int off = 16; off >= K; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) < K) sm[threadIdx.x >> 5][k] = acc;
    __syncthreads();
    if (threadIdx.x < K) {
      double t = 0.0;
      for (int wp = 0; wp < kBlock / 32; ++wp) t += sm[wp][threadIdx.x];
      part[((size_t)blockIdx.x * nd + i) * K + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// out[t] (+)= sum over blocks of part, t = i*K + k: one warp per output, each lane
// summing a fixed stride of the partials, then a fixed shuffle tree, so the
// result does not depend on scheduling.
__global__ void k_reduce_partials(int nblk, int nvK, const double* __restrict__ part, double* __restrict__ out,
                                  int accumulate, int take_sqrt, const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= nvK) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * nvK + t];
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    if (take_sqrt) s = sqrt(s);
    out[t] = accumulate ? out[t] + s : s;
  }
}

// w -= sum_i V_i h_i (per rhs); with nrm_part, also the partial sums of |w|^2.
template <int K, typename TV>
__global__ void __launch_bounds__(kBlock) k_maxpy(long long NK, int nv, const TV* __restrict__ V,
                                                  const double* __restrict__ h, double* __restrict__ w,
                                                  double* __restrict__ nrm_part, const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  __shared__ double sm[kBlock / 32][K];
  const int k = threadIdx.x % K;
  const long long stride = (long long)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < NK; e += stride) {
    double s = w[e];
    for (int i = 0; i < nv; ++i) s -= (double)V[(size_t)i * NK + e] * h[i * K + k];
    w[e] = s;
    acc += s * s;
  }
  if (!nrm_part) return;
#pragma unroll
  for (int off = 16; off >= K; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) < K) sm[threadIdx.x >> 5][k] = acc;
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int wp = 0; wp < kBlock / 32; ++wp) s += sm[wp][threadIdx.x];
    nrm_part[(size_t)blockIdx.x * K + threadIdx.x] = s;
  }
}

// v = w / nrm for active columns, 0 otherwise (one FP64 division per column and
// block; the elements are multiplied by the reciprocal), written in one pass both
// to the FP64 basis vector and, converted, to the V-cycle's input.
template <int K, typename TZ>
__global__ void k_scale_pack(long long NK, const double* __restrict__ w, const double* __restrict__ nrm,
                             const int* __restrict__ active, double* __restrict__ v, TZ* __restrict__ in) {
  __shared__ double inv[K];
  if (threadIdx.x < K) {
    const double n = nrm[threadIdx.x];
    inv[threadIdx.x] = (active[threadIdx.x] && n > 0.0) ? 1.0 / n : 0.0;
  }
  __syncthreads();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NK) return;
  const double x = w[e] * inv[(int)(e % K)];
  v[e] = x;
  in[e] = (TZ)x;
}

// The sum k_reduce_partials forms for output t (same order, so the same bits), by
// the calling warp; every lane gets it.
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ part, int nblk, int nvK, int t) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * nvK + t];
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// Selective re-orthogonalisation test (Daniel, Gragg, Kaufman and Stewart 1976):
// after one classical Gram-Schmidt pass, w' is re-orthogonalised when
// |w'| < |w| / sqrt(2) for some active column.  |w'| comes from the nblk block
// partial sums of |w'|^2 in part (warp k sums column k; 32 K threads).  slot holds
// |w|^2 on entry and |w'| on exit (the norm used when no second pass runs);
// *flag = 1 asks for the second pass.
__global__ void k_reorth_check(int K, double* __restrict__ slot, const double* __restrict__ part, int nblk,
                               const int* __restrict__ active, int* __restrict__ flag) {
  const int k = threadIdx.x >> 5;
  int need = 0;
  if (k < K) {
    const double n1 = sqrt(warp_sum_partials(part, nblk, K, k));
    if ((threadIdx.x & 31) == 0) {
      const double w2 = slot[k];
      need = active[k] && (n1 * n1 < 0.5 * w2);
      slot[k] = n1;
    }
  }
  const int any = __syncthreads_or(need);
  if (threadIdx.x == 0) *flag = any;
}

// Column j of the Hessenberg matrix for every rhs: apply the previous Givens
// rotations, form the new one, update the residual recurrence, retire
// columns that converged, broke down or ran out of iterations.  When *reorth is
// set the second Gram-Schmidt pass ran: first its coefficients h2 (nv per column)
// are added to the column and the new vector's norm |w''| (hcol row nv) is formed
// from the nblk partial sums in part (warp k, column k; 32 K threads).
__global__ void k_givens(int j, int m, int K, double* __restrict__ hcol, GmresState st,
                         const double* __restrict__ bnorm, double rtol, int* __restrict__ n_active,
                         const int* __restrict__ reorth, const double* __restrict__ part, int nblk,
                         const double* __restrict__ h2, int nv) {
  if (*reorth) {
    const int w = threadIdx.x >> 5;
    if (w < K) {
      const double n2 = sqrt(warp_sum_partials(part, nblk, K, w));
      if ((threadIdx.x & 31) == 0) hcol[(size_t)nv * K + w] = n2;
    }
    for (int t = threadIdx.x; t < nv * K; t += blockDim.x) hcol[t] += h2[t];
    __syncthreads();
  }
  const int k = threadIdx.x;
  int still = 0;
  if (k < K && st.active[k]) {
    double col[2];
    // rotate the column in place into Hm
    for (int i = 0; i <= j + 1; ++i) st.Hm[((size_t)i * m + j) * K + k] = hcol[(size_t)i * K + k];
    for (int i = 0; i < j; ++i) {
      col[0] = st.Hm[((size_t)i * m + j) * K + k];
      col[1] = st.Hm[((size_t)(i + 1) * m + j) * K + k];
      const double c = st.cs[i * K + k], s = st.sn[i * K + k];
      st.Hm[((size_t)i * m + j) * K + k] = c * col[0] + s * col[1];
      st.Hm[((size_t)(i + 1) * m + j) * K + k] = -s * col[0] + c * col[1];
    }
    const double a = st.Hm[((size_t)j * m + j) * K + k];
    const double b = st.Hm[((size_t)(j + 1) * m + j) * K + k];
    const double r = hypot(a, b);
    const double c = r == 0.0 ? 1.0 : a / r, s = r == 0.0 ? 0.0 : b / r;
    st.cs[j * K + k] = c;
    st.sn[j * K + k] = s;
    st.Hm[((size_t)j * m + j) * K + k] = r;
    st.Hm[((size_t)(j + 1) * m + j) * K + k] = 0.0;
    const double gj = st.gv[j * K + k];
    st.gv[(j + 1) * K + k] = -s * gj;
    st.gv[j * K + k] = c * gj;
    st.jcount[k] = j + 1;
    const double est = fabs(st.gv[(j + 1) * K + k]) / bnorm[k];
    st.resest[k] = est;
    still = 1;
    if (est <= rtol) {
      st.flags[k] = 1;
      still = 0;
    } else if (b == 0.0) {
      st.flags[k] = 2;
      still = 0;
    } else if (j + 1 >= st.budget[k]) {
      still = 0;
    }
    st.active[k] = still;
  }
  const int cnt = __syncthreads_count(still);
  if (threadIdx.x == 0) *n_active = cnt;
}

// Back substitution H y = g per column over its jcount rows.
__global__ void k_solve_y(int m, int K, GmresState st, double* __restrict__ y, int nmax) {
  const int k = threadIdx.x;
  if (k >= K) return;
  const int n = st.jcount[k];
  for (int i = nmax - 1; i >= n; --i) y[i * K + k] = 0.0;
  for (int i = n - 1; i >= 0; --i) {
    double s = st.gv[i * K + k];
    for (int l = i + 1; l < n; ++l) s -= st.Hm[((size_t)i * m + l) * K + k] * y[l * K + k];
    y[i * K + k] = s / st.Hm[((size_t)i * m + i) * K + k];
  }
}

// x += sum_i Z_i y_i.
template <int K, typename TZ>
__global__ void __launch_bounds__(kBlock) k_update_x(long long NK, int nz, const TZ* __restrict__ Z,
                                                     const double* __restrict__ y, double* __restrict__ x) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NK) return;
  const int k = (int)(e % K);
  double s = x[e];
  for (int i = 0; i < nz; ++i) s += (double)Z[(size_t)i * NK + e] * y[i * K + k];
  x[e] = s;
}

// ---------------------------------------------------------------------------
// Workspace carving: the same walk counts the bytes (Krylov::bytes_for) and
// allocates them (Krylov::init), so the two always agree.

struct Carver {
  bool count_only = true;
  size_t total = 0;
  std::vector<void*>* list = nullptr;
  template <typename U>
  U* get(size_t n) {
    const size_t b = (std::max<size_t>(n, 1) * sizeof(U) + 255) / 256 * 256;
    total += b;
    if (count_only) return nullptr;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();  // an allocation failure is not sticky: clear it for the next launch checks
      throw std::runtime_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    list->push_back(p);
    return (U*)p;
  }
};

void carve(Krylov& w, Carver& c) {
  const size_t NK = (size_t)w.N * w.K, K = w.K, m = w.m;
  w.V = c.get<double>(NK * (m + 1));
  w.Z = w.f32 ? (void*)c.get<float>(NK * m) : (void*)c.get<double>(NK * m);
  w.w = c.get<double>(NK);
  w.bK = c.get<double>(NK);
  w.xK = c.get<double>(NK);
  w.rK = c.get<double>(NK);
  w.hbuf = c.get<double>((m + 2) * K);
  w.part = c.get<double>((size_t)kRedBlocks * (m + 2) * K);
  w.y = c.get<double>((m + 1) * K);
  w.bnorm = c.get<double>(K);
  w.rnorm = c.get<double>(K);
  w.st.Hm = c.get<double>((m + 1) * m * K);
  w.st.cs = c.get<double>(m * K);
  w.st.sn = c.get<double>(m * K);
  w.st.gv = c.get<double>((m + 1) * K);
  w.st.active = c.get<int>(K);
  w.st.jcount = c.get<int>(K);
  w.st.budget = c.get<int>(K);
  w.st.flags = c.get<int>(K);
  w.st.resest = c.get<double>(K);
  w.n_active = c.get<int>(1);
  w.reorth = c.get<int>(1);
}

}  // namespace

namespace emin {

int round_k(int nrhs) {
  int K = 1;
  while (K < nrhs) K <<= 1;
  return K;
}

size_t Krylov::bytes_for(long long N, int K, int m, bool f32) {
  Krylov w;
  w.N = N;
  w.K = K;
  w.m = m;
  w.f32 = f32;
  Carver c;
  carve(w, c);
  return c.total;
}

void Krylov::init(long long N_, int K_, int m_, bool f32_) {
  release();
  N = N_;
  K = K_;
  m = m_;
  f32 = f32_;
  Carver c;
  c.count_only = false;
  c.list = &mem;
  try {
    carve(*this, c);
    bytes = c.total;
    if (cudaMallocHost(&host_i, sizeof(int) * kHostInts) != cudaSuccess ||
        cudaMallocHost(&host_d, sizeof(double) * kHostDoubles) != cudaSuccess)
      throw std::runtime_error("cudaMallocHost for the solver's pinned words failed");
  } catch (...) {
    release();
    throw;
  }
}

void Krylov::release() {
  for (void* p : mem) cudaFree(p);
  mem.clear();
  if (host_i) cudaFreeHost(host_i);
  if (host_d) cudaFreeHost(host_d);
  host_i = nullptr;
  host_d = nullptr;
  bytes = 0;
  K = m = 0;
}

namespace fgmres_detail {

// Norms of the K columns of an N x K FP64 block into out[k] (deterministic).
template <int K>
void col_norms(const Krylov& w, const double* v, double* out, cudaStream_t s, long long& launches) {
  const long long NK = w.N * K;
  const int rb = red_blocks(NK);
  k_mdot_partial<K, double><<<rb, kBlock, 0, s>>>(NK, 1, 0, v, v, w.part, nullptr);
  k_reduce_partials<<<(K * 32 + 127) / 128, 128, 0, s>>>(rb, K, w.part, out, 0, 1, nullptr);
  launches += 2;
}

// Restarted flexible GMRES for K interleaved columns, one chunk per advance():
//   start       b -> bK (packed), x = 0, |b| per column      -> host
//   cycle begin r0 / |r0| into V_0 for the columns still running
//   step j      z_j = M^-1 v_j (V-cycle graph), w = A z_j, classical Gram-Schmidt
//               with selective second pass, Givens update   -> host: columns active
//   cycle end   x += Z y, r = b - A x in FP64, |r|           -> host
//   finish      x unpacked into the caller's layout (and copied to the host)
template <int K, typename TZ>
class FgmresTask final : public SolveTask {
 public:
  FgmresTask(amg_hierarchy_core* h, VCycleIface* vc, Krylov* ws, const std::vector<SolveSegment>& segs, int nrhs,
             double rtol, int restart, int maxit, cudaStream_t s)
      : h_(h), vc_(vc), w_(ws), segs_(segs), nrhs_(nrhs), restart_(restart), maxit_(maxit), rtol_(rtol), s_(s),
        N_(h->N), NK_(h->N * K), gNK_(grid_for(h->N * K)), bn_(K, 0.0), rel_(K, 0.0), total_(K, 0), done_(K, 0),
        flag_(K, 0) {
    for (cudaEvent_t& e : ev_) EMIN_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  ~FgmresTask() override {
    for (cudaEvent_t e : ev_)
      if (e) cudaEventDestroy(e);
  }
  cudaEvent_t ready() const override { return ready_; }

  bool advance() override {
    static const char* kPhase[] = {"FGMRES: start", "FGMRES: Arnoldi step", "FGMRES: Arnoldi step",
                                   "FGMRES: restart cycle end", "FGMRES: finish", "FGMRES: done"};
    TraceRange range(kPhase[phase_]);
    switch (phase_) {
      case kStart:
        start();
        phase_ = kNorms;
        return chunk_done();
      case kNorms:
        for (int k = 0; k < K; ++k) {
          bn_[k] = w_->host_d[k];
          if (k >= nrhs_ || bn_[k] == 0.0) done_[k] = 1;
        }
        if (!any_left()) return finish();
        begin_cycle();
        phase_ = kStep;
        return true;
      case kStep: {
        // the results of step seen_ (its slot) are on the host
        const int slot = seen_ & 1;
        if (w_->host_i[kSlotInts + 2 * slot + 1] != 0)
          throw std::runtime_error("cuda: a bounded device wait timed out (Gauss-Seidel strips or ILU substitution)");
        const int n_active = w_->host_i[kSlotInts + 2 * slot];
        for (int k = 0; k < K; ++k) est_[2][k] = est_[1][k], est_[1][k] = w_->host_d[kSlotDoubles + 32 * slot + k];
        ++seen_;
        if (n_active == 0 || seen_ >= restart_) {
          // every column stopped at step seen_ - 1; a step issued beyond it found no
          // active column and changed nothing but the unused tail of V and Z
          j_ = issued_;
          end_cycle();
          return chunk_done();
        }
        if (issued_ == seen_) issue_step();  // not issued ahead: the next step now
        if (issued_ < restart_ && !final_step_likely()) issue_step();
        ready_ = ev_[seen_ & 1];
        return true;
      }
      case kCycle: {
        bool left = false;
        for (int k = 0; k < K; ++k) {
          if (done_[k]) continue;
          const int used = w_->host_i[k];
          total_[k] += used;
          rel_[k] = w_->host_d[k] / bn_[k];
          if (w_->host_i[64 + k] == 2 && rel_[k] > rtol_) flag_[k] = 2;
          if (rel_[k] <= rtol_ || total_[k] >= maxit_ || flag_[k] == 2 || used == 0)
            done_[k] = 1;
          else
            left = true;
        }
        if (!left) return finish();
        begin_cycle();
        phase_ = kStep;
        return true;
      }
      case kFinish:
        phase_ = kDone;
        return false;
      case kDone:
        return false;
    }
    return false;
  }

  amg_status column_status(int k) const override {
    if (k < 0 || k >= nrhs_ || bn_[k] == 0.0 || rel_[k] <= rtol_) return AMG_OK;
    return flag_[k] == 2 ? AMG_BREAKDOWN : AMG_NOT_CONVERGED;
  }

  amg_status result(int* iters, double* relres) const override {
    amg_status st = AMG_OK;
    for (int k = 0; k < nrhs_; ++k) {
      if (iters) iters[k] = total_[k];
      if (relres) relres[k] = bn_[k] == 0.0 ? 0.0 : rel_[k];
      if (bn_[k] != 0.0 && rel_[k] > rtol_) st = flag_[k] == 2 ? AMG_BREAKDOWN : AMG_NOT_CONVERGED;
    }
    return st;
  }

 private:
  enum Phase { kStart, kNorms, kStep, kCycle, kFinish, kDone };
  // pinned host words of the two step result slots: (active columns, error word) at
  // host_i[kSlotInts + 2 slot], the columns' residual estimates at
  // host_d[kSlotDoubles + 32 slot]
  static constexpr int kSlotInts = 32, kSlotDoubles = 64;

  // An event after the chunk just enqueued, the one the next advance() waits for.
  bool chunk_done() {
    EMIN_CUDA(cudaEventRecord(ev_[2], s_));
    ready_ = ev_[2];
    return true;
  }

  // Enqueue Arnoldi step issued_ (after the normalisation of its basis vector),
  // its results into slot issued_ & 1, and that slot's event.
  void issue_step() {
    // v_j = (r or w) / its norm, into the basis and the V-cycle's input
    const bool first = issued_ == 0;
    k_scale_pack<K, TZ><<<gNK_, kBlock, 0, s_>>>(NK_, first ? w_->rK : w_->w,
                                                first ? w_->rnorm : w_->hbuf + (size_t)issued_ * K, w_->st.active,
                                                w_->V + (size_t)issued_ * NK_, (TZ*)vc_->input(0));
    ++launches;
    j_ = issued_;
    step();
    const int slot = issued_ & 1;
    EMIN_CUDA(cudaMemcpyAsync(w_->host_i + kSlotInts + 2 * slot, w_->n_active, sizeof(int), cudaMemcpyDeviceToHost,
                              s_));
    EMIN_CUDA(cudaMemcpyAsync(w_->host_i + kSlotInts + 2 * slot + 1, vc_->error_flag(), sizeof(int),
                              cudaMemcpyDeviceToHost, s_));
    EMIN_CUDA(cudaMemcpyAsync(w_->host_d + kSlotDoubles + 32 * slot, w_->st.resest, sizeof(double) * K,
                              cudaMemcpyDeviceToHost, s_));
    EMIN_CUDA(cudaEventRecord(ev_[slot], s_));
    ++issued_;
  }

  // Whether the step just issued (seen_, not yet seen) will probably stop every
  // running column: each column's residual estimate extrapolated by its last
  // reduction factor reaches 4 rtol.  Then no further step is queued ahead, which
  // would find nothing left to do.
  bool final_step_likely() const {
    if (seen_ < 2) return false;
    bool all = true;
    for (int k = 0; k < K && all; ++k) {
      if (done_[k]) continue;
      const double e1 = est_[1][k], e2 = est_[2][k];
      if (!(e1 > 0.0) || !(e2 > 0.0)) continue;  // a column that stopped: no opinion
      all = e1 * (e1 / e2) <= 4.0 * rtol_;
    }
    return all;
  }

  bool any_left() const {
    return std::any_of(done_.begin(), done_.end(), [](int d) { return !d; });
  }

  void start() {
    // a wait that timed out in an earlier call does not fail this one
    EMIN_CUDA(cudaMemsetAsync(vc_->error_flag(), 0, sizeof(int), s_));
    for (const SolveSegment& g : segs_)
      if (g.b_host)
        EMIN_CUDA(cudaMemcpyAsync(const_cast<double*>(g.b), g.b_host, sizeof(double) * N_ * g.ncols,
                                  cudaMemcpyHostToDevice, s_));
    if (segs_.size() == 1) {
      k_pack<double, double, K><<<gNK_, kBlock, 0, s_>>>(N_, segs_[0].b, nrhs_, nrhs_, w_->bK);
      ++launches;
    } else {
      if (nrhs_ < K) EMIN_CUDA(cudaMemsetAsync(w_->bK, 0, sizeof(double) * NK_, s_));
      int col0 = 0;
      for (const SolveSegment& g : segs_) {
        k_pack_cols<K><<<grid_for(N_ * g.ncols), kBlock, 0, s_>>>(N_, g.b, g.ncols, w_->bK, col0);
        ++launches;
        col0 += g.ncols;
      }
    }
    EMIN_CUDA(cudaMemsetAsync(w_->xK, 0, sizeof(double) * NK_, s_));
    col_norms<K>(*w_, w_->bK, w_->bnorm, s_, launches);
    EMIN_CUDA(cudaMemcpyAsync(w_->host_d, w_->bnorm, sizeof(double) * K, cudaMemcpyDeviceToHost, s_));
    // r = b for the first cycle
    EMIN_CUDA(cudaMemcpyAsync(w_->rK, w_->bK, sizeof(double) * NK_, cudaMemcpyDeviceToDevice, s_));
  }

  // Start vector v0 = r / |r| for the columns still running; g = (|r|, 0, ...).
  void begin_cycle() {
    int* act = w_->host_i + 128;
    int* bud = w_->host_i + 192;
    for (int k = 0; k < K; ++k) {
      act[k] = !done_[k];
      bud[k] = std::min(restart_, maxit_ - total_[k]);
      if (bud[k] <= 0) act[k] = 0;
    }
    EMIN_CUDA(cudaMemcpyAsync(w_->st.active, act, sizeof(int) * K, cudaMemcpyHostToDevice, s_));
    EMIN_CUDA(cudaMemcpyAsync(w_->st.budget, bud, sizeof(int) * K, cudaMemcpyHostToDevice, s_));
    EMIN_CUDA(cudaMemsetAsync(w_->st.jcount, 0, sizeof(int) * K, s_));
    EMIN_CUDA(cudaMemsetAsync(w_->st.flags, 0, sizeof(int) * K, s_));
    EMIN_CUDA(cudaMemsetAsync(w_->st.gv, 0, sizeof(double) * (restart_ + 1) * K, s_));
    col_norms<K>(*w_, w_->rK, w_->rnorm, s_, launches);
    EMIN_CUDA(cudaMemcpyAsync(w_->st.gv, w_->rnorm, sizeof(double) * K, cudaMemcpyDeviceToDevice, s_));
    j_ = 0;
    issued_ = seen_ = 0;
    for (auto& e : est_) std::fill(e.begin(), e.end(), 0.0);
    issue_step();
    if (restart_ > 1) issue_step();
    ready_ = ev_[0];
  }

  void step() {
    const int j = j_;
    TZ* Z = (TZ*)w_->Z;
    // z_j = M^-1 v_j through the captured V-cycle (v_j is in its input: issue_step)
    EMIN_CUDA(cudaGetLastError());
    EMIN_CUDA(vc_->run(K, s_));
    EMIN_CUDA(cudaMemcpyAsync(Z + (size_t)j * NK_, vc_->output(0), sizeof(TZ) * NK_, cudaMemcpyDeviceToDevice, s_));
    // w = A z_j in FP64
    if (vc_->is_fp32()) {
      EMIN_CUDA(vc_->apply_ff((const float*)(Z + (size_t)j * NK_), w_->w, K, s_));
    } else {
      EMIN_CUDA(apply_finest_f64(h_->v64, Z + (size_t)j * NK_, false, nullptr, w_->w, K, s_));
      ++launches;
    }
    // classical Gram-Schmidt, re-orthogonalised only when the first pass cancelled
    // more than half of |w| (k_reorth_check)
    const int nv = j + 1;
    double* hn = w_->hbuf + (size_t)nv * K;  // |w|^2, then the norm of the new vector
    double* h2 = w_->y;                      // scratch for the correction coefficients
    const unsigned rnv = (unsigned)((nv * K * 32 + 127) / 128);
    const int rb = red_blocks(NK_);
    k_mdot_partial<K, double><<<dim3(rb, dot_split(rb, nv + 1)), kBlock, 0, s_>>>(NK_, nv, 1, w_->V, w_->w, w_->part,
                                                                                  nullptr);
    k_reduce_partials<<<((nv + 1) * K * 32 + 127) / 128, 128, 0, s_>>>(rb, (nv + 1) * K, w_->part, w_->hbuf,
                                                                        0, 0, nullptr);
    k_maxpy<K, double><<<rb, kBlock, 0, s_>>>(NK_, nv, w_->V, w_->hbuf, w_->w, w_->part, nullptr);
    k_reorth_check<<<1, 32 * K, 0, s_>>>(K, hn, w_->part, rb, w_->st.active, w_->reorth);
    k_mdot_partial<K, double><<<dim3(rb, dot_split(rb, nv)), kBlock, 0, s_>>>(NK_, nv, 0, w_->V, w_->w, w_->part,
                                                                              w_->reorth);
    k_reduce_partials<<<rnv, 128, 0, s_>>>(rb, nv * K, w_->part, h2, 0, 0, w_->reorth);
    k_maxpy<K, double><<<rb, kBlock, 0, s_>>>(NK_, nv, w_->V, h2, w_->w, w_->part, w_->reorth);
    k_givens<<<1, 32 * K, 0, s_>>>(j, restart_, K, w_->hbuf, w_->st, w_->bnorm, rtol_, w_->n_active, w_->reorth,
                                   w_->part, rb, h2, nv);
    launches += 8;
    EMIN_CUDA(cudaGetLastError());
  }

  // x += Z y with y from the triangular systems; true residual r = b - A x in FP64.
  void end_cycle() {
    const int nmax = std::min(j_, restart_);
    k_solve_y<<<1, 32, 0, s_>>>(restart_, K, w_->st, w_->y, nmax);
    k_update_x<K, TZ><<<gNK_, kBlock, 0, s_>>>(NK_, nmax, (const TZ*)w_->Z, w_->y, w_->xK);
    launches += 2;
    EMIN_CUDA(apply_finest_f64(h_->v64, w_->xK, false, w_->bK, w_->rK, K, s_));
    ++launches;
    col_norms<K>(*w_, w_->rK, w_->rnorm, s_, launches);
    EMIN_CUDA(cudaMemcpyAsync(w_->host_d, w_->rnorm, sizeof(double) * K, cudaMemcpyDeviceToHost, s_));
    EMIN_CUDA(cudaMemcpyAsync(w_->host_i, w_->st.jcount, sizeof(int) * K, cudaMemcpyDeviceToHost, s_));
    EMIN_CUDA(cudaMemcpyAsync(w_->host_i + 64, w_->st.flags, sizeof(int) * K, cudaMemcpyDeviceToHost, s_));
    phase_ = kCycle;
  }
  // (end_cycle's caller records the chunk's event: chunk_done)

  bool finish() {
    if (segs_.size() == 1) {
      k_unpack<double, double, K><<<grid_for(N_ * nrhs_), kBlock, 0, s_>>>(N_, w_->xK, nrhs_, segs_[0].x, nrhs_);
      ++launches;
    } else {
      int col0 = 0;
      for (const SolveSegment& g : segs_) {
        k_unpack_cols<K><<<grid_for(N_ * g.ncols), kBlock, 0, s_>>>(N_, w_->xK, col0, g.ncols, g.x);
        ++launches;
        col0 += g.ncols;
      }
    }
    EMIN_CUDA(cudaGetLastError());
    for (const SolveSegment& g : segs_)
      if (g.x_host)
        EMIN_CUDA(cudaMemcpyAsync(g.x_host, g.x, sizeof(double) * N_ * g.ncols, cudaMemcpyDeviceToHost, s_));
    phase_ = kFinish;
    return chunk_done();
  }

  amg_hierarchy_core* h_;
  VCycleIface* vc_;
  Krylov* w_;
  std::vector<SolveSegment> segs_;
  int nrhs_, restart_, maxit_;
  double rtol_;
  cudaStream_t s_;
  long long N_, NK_;
  unsigned gNK_;
  std::vector<double> bn_, rel_;
  std::vector<int> total_, done_, flag_;
  Phase phase_ = kStart;
  int j_ = 0;
  int issued_ = 0, seen_ = 0;  // Arnoldi steps of the current cycle enqueued / whose results were read
  cudaEvent_t ev_[3] = {nullptr, nullptr, nullptr};  // step slots 0 and 1, other chunks
  cudaEvent_t ready_ = nullptr;
  std::vector<double> est_[3] = {std::vector<double>(K, 0.0), std::vector<double>(K, 0.0),
                                 std::vector<double>(K, 0.0)};  // [1] last seen step's estimates, [2] the one before
};

template <typename TZ>
std::unique_ptr<SolveTask> make_task_t(int K, amg_hierarchy_core* h, VCycleIface* vc, Krylov* ws,
                                       const std::vector<SolveSegment>& g, int nrhs, double rtol, int restart,
                                       int maxit, cudaStream_t s) {
  switch (K) {
    case 1: return std::make_unique<FgmresTask<1, TZ>>(h, vc, ws, g, nrhs, rtol, restart, maxit, s);
    case 2: return std::make_unique<FgmresTask<2, TZ>>(h, vc, ws, g, nrhs, rtol, restart, maxit, s);
    case 4: return std::make_unique<FgmresTask<4, TZ>>(h, vc, ws, g, nrhs, rtol, restart, maxit, s);
    case 8: return std::make_unique<FgmresTask<8, TZ>>(h, vc, ws, g, nrhs, rtol, restart, maxit, s);
    case 16: return std::make_unique<FgmresTask<16, TZ>>(h, vc, ws, g, nrhs, rtol, restart, maxit, s);
    case 32: return std::make_unique<FgmresTask<32, TZ>>(h, vc, ws, g, nrhs, rtol, restart, maxit, s);
  }
  throw std::runtime_error("nrhs must be in 1..32");
}

}  // namespace fgmres_detail

std::unique_ptr<SolveTask> make_solve_task(amg_hierarchy_core* h, VCycleIface* vc, Krylov* ws,
                                           const std::vector<SolveSegment>& segs, double rtol, int restart, int maxit,
                                           cudaStream_t s) {
  int nrhs = 0;
  for (const SolveSegment& g : segs) {
    if (g.ncols < 1 || !g.b || !g.x) throw std::runtime_error("empty or null solve segment");
    nrhs += g.ncols;
  }
  const int K = round_k(nrhs);
  if (nrhs < 1 || K > 32 || K > vc->kmax()) throw std::runtime_error("nrhs exceeds the V-cycle's max_nrhs");
  if (ws->N != h->N || ws->K != K || ws->m < restart || ws->f32 != vc->is_fp32())
    throw std::runtime_error("solver workspace does not match the solve");
  using fgmres_detail::make_task_t;
  if (vc->is_fp32()) return make_task_t<float>(K, h, vc, ws, segs, nrhs, rtol, restart, maxit, s);
  return make_task_t<double>(K, h, vc, ws, segs, nrhs, rtol, restart, maxit, s);
}

std::unique_ptr<SolveTask> make_solve_task(amg_hierarchy_core* h, VCycleIface* vc, Krylov* ws, const double* b,
                                           double* x, const double* b_host, double* x_host, int nrhs, double rtol,
                                           int restart, int maxit, cudaStream_t s) {
  SolveSegment g;
  g.b = b;
  g.x = x;
  g.b_host = b_host;
  g.x_host = x_host;
  g.ncols = nrhs;
  return make_solve_task(h, vc, ws, std::vector<SolveSegment>{g}, rtol, restart, maxit, s);
}

}  // namespace emin

namespace {

void ensure_ws(amg_hierarchy* h, int K, int m) {
  const bool f32 = h->prm.vcycle_fp32 != 0;
  if (h->kry && h->kry->K == K && h->kry->m >= m && h->kry->f32 == f32) return;
  h->kry.reset();
  auto w = std::make_unique<Krylov>();
  w->init(h->N, K, m, f32);
  h->kry = std::move(w);
}

// One Gram-Schmidt pass with nv basis vectors on the solver's own workspace (zeroed
// first: the FP64 work does not depend on the values), timed with CUDA events on
// `s`: the inner products with the norm (k_mdot_partial, nv + 1 outputs per column)
// and the update with the norm (k_maxpy), each averaged over reps launches.
template <int K>
void profile_arnoldi_k(amg_hierarchy* h, int nv, int reps, double* ms_dot, double* ms_update, cudaStream_t s) {
  Krylov& w = *h->kry;
  const long long NK = w.N * K;
  EMIN_CUDA(cudaMemsetAsync(w.V, 0, sizeof(double) * (size_t)NK * (nv + 1), s));
  EMIN_CUDA(cudaMemsetAsync(w.w, 0, sizeof(double) * (size_t)NK, s));
  EMIN_CUDA(cudaMemsetAsync(w.hbuf, 0, sizeof(double) * (size_t)(nv + 2) * K, s));
  const int rb = red_blocks(NK);
  cudaEvent_t e[3];
  for (cudaEvent_t& ev : e) EMIN_CUDA(cudaEventCreate(&ev));
  float tot_dot = 0.f, tot_upd = 0.f;
  for (int rep = 0; rep <= reps; ++rep) {  // rep 0 warms up
    EMIN_CUDA(cudaEventRecord(e[0], s));
    k_mdot_partial<K, double><<<dim3(rb, dot_split(rb, nv + 1)), kBlock, 0, s>>>(NK, nv, 1, w.V, w.w, w.part, nullptr);
    EMIN_CUDA(cudaEventRecord(e[1], s));
    k_maxpy<K, double><<<rb, kBlock, 0, s>>>(NK, nv, w.V, w.hbuf, w.w, w.part, nullptr);
    EMIN_CUDA(cudaEventRecord(e[2], s));
    EMIN_CUDA(cudaEventSynchronize(e[2]));
    float a = 0.f, b = 0.f;
    EMIN_CUDA(cudaEventElapsedTime(&a, e[0], e[1]));
    EMIN_CUDA(cudaEventElapsedTime(&b, e[1], e[2]));
    if (rep > 0) tot_dot += a, tot_upd += b;
  }
  for (cudaEvent_t ev : e) cudaEventDestroy(ev);
  h->launches += 2LL * (reps + 1);
  *ms_dot = tot_dot / reps;
  *ms_update = tot_upd / reps;
}

amg_status fgmres_blocking(amg_hierarchy* h, const double* b, double* x, const double* bh, double* xh, int nrhs,
                           double rtol, int restart, int maxit, int* iters, double* relres, cudaStream_t s) {
  ensure_ws(h, round_k(nrhs), restart);
  auto task = make_solve_task(h, h->vc(), h->kry.get(), b, x, bh, xh, nrhs, rtol, restart, maxit, s);
  bool more = true;
  while (more) {
    more = task->advance();
    h->launches += task->launches;
    task->launches = 0;
    if (cudaEvent_t e = task->ready(); more && e)
      EMIN_CUDA(cudaEventSynchronize(e));
    else
      EMIN_CUDA(cudaStreamSynchronize(s));
  }
  EMIN_CUDA(cudaStreamSynchronize(s));
  return task->result(iters, relres);
}

template <int K, typename T>
void vcycle_k(amg_hierarchy* h, const double* r, double* z, int nrhs, cudaStream_t s) {
  VCycleIface* vc = h->vc();
  const long long N = h->N;
  k_pack<double, T, K><<<grid_for(N * K), kBlock, 0, s>>>(N, r, nrhs, nrhs, (T*)vc->input(0)); ++h->launches;
  EMIN_CUDA(cudaGetLastError());
  EMIN_CUDA(vc->run(K, s));
  k_unpack<T, double, K><<<grid_for(N * nrhs), kBlock, 0, s>>>(N, (const T*)vc->output(0), nrhs, z, nrhs); ++h->launches;
  EMIN_CUDA(cudaGetLastError());
}

template <typename T>
void vcycle_dispatch(amg_hierarchy* h, const double* r, double* z, int nrhs, cudaStream_t s) {
  switch (round_k(nrhs)) {
    case 1: vcycle_k<1, T>(h, r, z, nrhs, s); break;
    case 2: vcycle_k<2, T>(h, r, z, nrhs, s); break;
    case 4: vcycle_k<4, T>(h, r, z, nrhs, s); break;
    case 8: vcycle_k<8, T>(h, r, z, nrhs, s); break;
    case 16: vcycle_k<16, T>(h, r, z, nrhs, s); break;
    case 32: vcycle_k<32, T>(h, r, z, nrhs, s); break;
  }
}

template <int K>
void apply_k(amg_hierarchy* h, const double* x, double* y, int nrhs, cudaStream_t s) {
  const long long N = h->N;
  k_pack<double, double, K><<<grid_for(N * K), kBlock, 0, s>>>(N, x, nrhs, nrhs, h->kry->bK); ++h->launches;
  EMIN_CUDA(cudaGetLastError());
  EMIN_CUDA(apply_finest_f64(h->v64, h->kry->bK, false, nullptr, h->kry->w, K, s)); ++h->launches;
  k_unpack<double, double, K><<<grid_for(N * nrhs), kBlock, 0, s>>>(N, h->kry->w, nrhs, y, nrhs); ++h->launches;
  EMIN_CUDA(cudaGetLastError());
}

bool check_csr(const int* rp, const int* ci, int nrows, int ncols, std::string& why) {
  if (!rp || rp[0] != 0) {
    why = "rowptr must start at 0";
    return false;
  }
  for (int i = 0; i < nrows; ++i) {
    if (rp[i + 1] < rp[i]) {
      why = "rowptr not monotone at row " + std::to_string(i);
      return false;
    }
    for (int t = rp[i]; t < rp[i + 1]; ++t) {
      if (ci[t] < 0 || ci[t] >= ncols) {
        why = "column out of range in row " + std::to_string(i);
        return false;
      }
      if (t > rp[i] && ci[t] <= ci[t - 1]) {
        why = "columns not strictly ascending in row " + std::to_string(i);
        return false;
      }
    }
  }
  return true;
}

Csr to_csr(const int* rp, const int* ci, const double* v, int nrows, int ncols) {
  Csr M;
  M.resize_rows(nrows, ncols);
  for (int i = 0; i <= nrows; ++i) M.rowptr[i] = rp[i];
  M.col.assign(ci, ci + rp[nrows]);
  M.val.assign(v, v + rp[nrows]);
  return M;
}

// Scratch of amg_apply_noalloc: a file-scope device array, so that entry point
// never allocates.  Each device that loads the library holds these 16 MiB until
// the process exits.  Host code must not pass the array's name to a kernel (it
// is a host-side stand-in); it passes the address cudaGetSymbolAddress returns
// for the current device, looked up once per device.
constexpr long long kNoAllocScratchDoubles = 2LL << 20;              // 16 MiB of doubles
constexpr long long kNoAllocMaxEntries = kNoAllocScratchDoubles / 2;  // per buffer: padded x and y
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mutex;
std::vector<double*> g_noalloc_ptr;  // per device ordinal, filled on the first call on that device

double* noalloc_scratch(std::string& why) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if ((int)g_noalloc_ptr.size() <= dev) g_noalloc_ptr.resize(dev + 1, nullptr);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      why = std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e);
      return nullptr;
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  return g_noalloc_ptr[dev];
}

template <int K>
void apply_noalloc_k(amg_hierarchy* h, const double* x, double* y, int nrhs, double* xs, double* ys,
                     cudaStream_t s) {
  const long long N = h->N;
  k_pack<double, double, K><<<grid_for(N * K), kBlock, 0, s>>>(N, x, nrhs, nrhs, xs);
  ++h->launches;
  EMIN_CUDA(cudaGetLastError());
  EMIN_CUDA(apply_finest_f64(h->v64, xs, false, nullptr, ys, K, s));
  ++h->launches;
  k_unpack<double, double, K><<<grid_for(N * nrhs), kBlock, 0, s>>>(N, ys, nrhs, y, nrhs);
  ++h->launches;
  EMIN_CUDA(cudaGetLastError());
}

}  // namespace

extern "C" {

amg_status amg_apply_noalloc(amg_handle h, const double* x, double* y, int nrhs, void* stream) {
  if (!h || !x || !y) return fail(AMG_ERR_ARG, "amg_apply_noalloc: null argument");
  if (!h->v64) return fail(AMG_ERR_ARG, "amg_apply_noalloc: hierarchy was built with host_only");
  if (nrhs < 1 || nrhs > 32) return fail(AMG_ERR_ARG, "amg_apply_noalloc: nrhs must be in 1..32");
  const int K = round_k(nrhs);
  if ((long long)h->N * K > kNoAllocMaxEntries)
    return fail(AMG_ERR_ARG, "amg_apply_noalloc: N * K = " + std::to_string((long long)h->N * K) +
                                 " exceeds the static scratch of " + std::to_string(kNoAllocMaxEntries) +
                                 " doubles per operand (K = nrhs rounded up to a power of two)");
  std::string why;
  double* scratch = noalloc_scratch(why);
  if (!scratch) return fail(AMG_ERR_CUDA, "amg_apply_noalloc: " + why);
  double* xs = scratch;
  double* ys = scratch + kNoAllocMaxEntries;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    switch (K) {
      case 1: apply_noalloc_k<1>(h, x, y, nrhs, xs, ys, s); break;
      case 2: apply_noalloc_k<2>(h, x, y, nrhs, xs, ys, s); break;
      case 4: apply_noalloc_k<4>(h, x, y, nrhs, xs, ys, s); break;
      case 8: apply_noalloc_k<8>(h, x, y, nrhs, xs, ys, s); break;
      case 16: apply_noalloc_k<16>(h, x, y, nrhs, xs, ys, s); break;
      case 32: apply_noalloc_k<32>(h, x, y, nrhs, xs, ys, s); break;
    }
  } catch (const std::exception& e) {
    return fail(AMG_ERR_CUDA, std::string("amg_apply_noalloc: ") + e.what());
  }
  return AMG_OK;
}

void amg_params_default(amg_params* p) {
  if (!p) return;
  p->tau1 = -1.0;
  p->tau2sq = 1.5e-3;
  p->omega = 0.666;
  p->omega_on_D = 0;
  p->gs_iters = 5;
  p->pre = 2;
  p->post = 2;
  p->max_coarse = 200;
  p->max_levels = 12;
  p->vcycle_fp32 = 0;
  p->max_nrhs = 8;
  p->host_only = 0;
  p->autotune = 1;
  p->smoother = 0;
  p->vanka_omega = 0.5;
  p->ilu_order = 0;
  p->coarse = 0;
  p->device_setup = 1;
  p->vanka_max_mib = 16384.0;
}

const char* amg_last_error(void) { return g_last_error.c_str(); }

namespace {
amg_status create_impl(const amg_problem* pb, const amg_params* prm_in, void* stream, amg_handle* out,
                       const amg_hierarchy* reuse);
bool same_pattern(const Csr& M, const int* rp, const int* ci, int nrows) {
  if (M.nrows != nrows) return false;
  for (int i = 0; i <= nrows; ++i)
    if (M.rowptr[i] != rp[i]) return false;
  for (int64_t t = 0; t < M.rowptr[nrows]; ++t)
    if (M.col[t] != ci[t]) return false;
  return true;
}
}  // namespace

amg_status amg_hierarchy_create(const amg_problem* pb, const amg_params* prm_in, void* stream, amg_handle* out) {
  TraceRange range("amg_hierarchy_create");
  return create_impl(pb, prm_in, stream, out, nullptr);
}

amg_status amg_hierarchy_create_reuse(amg_handle prev, const amg_problem* pb, const amg_params* prm_in, void* stream,
                                      amg_handle* out) {
  if (!prev || !pb || !out) return fail(AMG_ERR_ARG, "null previous hierarchy, problem or output handle");
  *out = nullptr;
  const HostLevel& F = prev->host[0];
  if (pb->dim != F.dim || pb->n_vnodes != F.n_v || pb->n_pnodes != F.n_p)
    return fail(AMG_ERR_ARG, "the problem's sizes differ from the previous hierarchy's");
  if (!pb->A_rowptr || !pb->A_col || !pb->B_rowptr || !pb->B_col) return fail(AMG_ERR_ARG, "null problem array");
  if (!same_pattern(F.A, pb->A_rowptr, pb->A_col, F.n_v) || !same_pattern(F.B, pb->B_rowptr, pb->B_col, F.n_p))
    return fail(AMG_ERR_ARG, "the sparsity of A or B differs from the previous hierarchy's");
  TraceRange range("amg_hierarchy_create_reuse");
  return create_impl(pb, prm_in, stream, out, prev);
}

namespace {
// The parameters of a create or import call (defaults for NULL); "" if valid, else why not.
std::string check_params(const amg_params* prm_in, amg_params& prm) {
  if (prm_in)
    prm = *prm_in;
  else
    amg_params_default(&prm);
  if (prm.max_nrhs < 1 || prm.max_nrhs > 32) return "max_nrhs must be in 1..32";
  if (prm.gs_iters < 0 || prm.pre < 0 || prm.post < 0 || prm.omega <= 0.0) return "invalid smoother parameters";
  if (prm.smoother < 0 || prm.smoother > 2) return "smoother must be 0 (Braess-Sarazin), 1 (Vanka) or 2 (ILU(1))";
  if (prm.smoother == 1 && !(prm.vanka_omega > 0.0)) return "vanka_omega must be positive";
  if (!(prm.vanka_max_mib > 0.0) || prm.vanka_max_mib > 1e9) return "vanka_max_mib must be in (0, 1e9]";
  if (prm.ilu_order != 0 && prm.ilu_order != 1) return "ilu_order must be 0 or 1";
  if (prm.coarse != 0 && prm.coarse != 1) return "coarse must be 0 (pseudo-inverse) or 1 (Vanka)";
  if (prm.coarse == 1 && !(prm.vanka_omega > 0.0)) return "vanka_omega must be positive";
  if (prm.device_setup != 0 && prm.device_setup != 1) return "device_setup must be 0 or 1";
  return "";
}

SetupParams setup_params(const amg_params& prm, bool symmetric) {
  SetupParams sp;
  sp.tau1 = prm.tau1;
  sp.tau2sq = prm.tau2sq;
  sp.c = prm.omega_on_D ? 1.0 / prm.omega : prm.omega;
  sp.max_coarse = prm.max_coarse;
  sp.max_levels = prm.max_levels;
  sp.symmetric = symmetric;
  sp.vanka = prm.smoother == 1;
  sp.ilu = prm.smoother == 2;
  sp.ilu_order = prm.ilu_order;
  sp.vanka_coarse = prm.coarse == 1;
  sp.gs_iters = prm.gs_iters;
  sp.vanka_max_bytes = (size_t)(prm.vanka_max_mib * 1048576.0);
  return sp;
}

// The device cycles of a hierarchy whose host levels are complete (throws).
void upload_handle(amg_hierarchy* h, const SetupParams& sp, void* stream) {
  const amg_params& prm = h->prm;
  h->N = h->host[0].N();
  if (prm.host_only) return;
  const double vomega = prm.smoother == 1 ? prm.vanka_omega : 0.0;
  const double comega = prm.coarse == 1 ? prm.vanka_omega : 0.0;
  h->v64 = make_vcycle_f64(h->host, sp.c, prm.gs_iters, prm.pre, prm.post, round_k(prm.max_nrhs), vomega, sp.ilu,
                           comega);
  h->v64->set_autotune(prm.autotune != 0);
  if (prm.vcycle_fp32) {
    h->v32 = make_vcycle_f32(h->host, sp.c, prm.gs_iters, prm.pre, prm.post, round_k(prm.max_nrhs), vomega, sp.ilu,
                             comega);
    h->v32->set_autotune(prm.autotune != 0);
  }
  EMIN_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
}

amg_status create_impl(const amg_problem* pb, const amg_params* prm_in, void* stream, amg_handle* out,
                       const amg_hierarchy* reuse) {
  if (!pb || !out) return fail(AMG_ERR_ARG, "null problem or output handle");
  *out = nullptr;
  amg_params prm;
  std::string why = check_params(prm_in, prm);
  if (!why.empty()) return fail(AMG_ERR_ARG, why);
  if (pb->dim < 2 || pb->dim > 3 || pb->n_vnodes <= 0 || pb->n_pnodes <= 0)
    return fail(AMG_ERR_ARG, "dim must be 2 or 3 and node counts positive");
  if (!pb->A_val || !pb->B_val || !pb->vcoords || !pb->pcoords || !pb->p2v || !pb->v_dirichlet)
    return fail(AMG_ERR_ARG, "null problem array");
  if (pb->pinned_p >= pb->n_pnodes) return fail(AMG_ERR_ARG, "pinned pressure out of range");
  if (!check_csr(pb->A_rowptr, pb->A_col, pb->n_vnodes, pb->n_vnodes, why)) return fail(AMG_ERR_ARG, "A: " + why);
  if (!check_csr(pb->B_rowptr, pb->B_col, pb->n_pnodes, pb->dim * pb->n_vnodes, why))
    return fail(AMG_ERR_ARG, "B: " + why);
  for (int k = 0; k < pb->n_pnodes; ++k)
    if (pb->p2v[k] < -1 || pb->p2v[k] >= pb->n_vnodes) return fail(AMG_ERR_ARG, "p2v out of range");
  std::unique_ptr<amg_hierarchy> h(new amg_hierarchy());
  try {
    HostLevel fine;
    fine.dim = pb->dim;
    fine.n_v = pb->n_vnodes;
    fine.n_p = pb->n_pnodes;
    fine.pinned = pb->pinned_p;
    fine.A = to_csr(pb->A_rowptr, pb->A_col, pb->A_val, fine.n_v, fine.n_v);
    fine.B = to_csr(pb->B_rowptr, pb->B_col, pb->B_val, fine.n_p, fine.dim * fine.n_v);
    fine.Bt = transpose(fine.B);
    fine.vX.assign(pb->vcoords, pb->vcoords + (size_t)fine.n_v * fine.dim);
    fine.pX.assign(pb->pcoords, pb->pcoords + (size_t)fine.n_p * fine.dim);
    fine.p2v.assign(pb->p2v, pb->p2v + fine.n_p);
    fine.dirichlet.assign(pb->v_dirichlet, pb->v_dirichlet + fine.n_v);
    SetupParams sp = setup_params(prm, pb->symmetric != 0);
    const bool on_device = prm.device_setup && !prm.host_only;
    sp.dense_gs = !on_device;
    if (reuse && on_device) {
      // numeric setup on the GPU with the previous hierarchy's patterns; the plan
      // (patterns and maps on the device) is shared along the sequence
      h->host = build_hierarchy_reuse_device(std::move(fine), reuse->host, sp, reuse->plan, (cudaStream_t)stream);
      h->plan = reuse->plan;
      complete_hierarchy(h->host, sp, false);
    } else {
      sp.reuse = reuse ? &reuse->host : nullptr;
      h->host = build_hierarchy(std::move(fine), sp);
    }
    if (on_device) form_dense_gs_device(h->host, prm.gs_iters, (cudaStream_t)stream);
    h->prm = prm;
    h->symmetric = sp.symmetric;
    TraceRange r("upload of the device hierarchy");
    upload_handle(h.get(), sp, stream);
  } catch (const std::bad_alloc&) {
    return fail(AMG_ERR_OOM, "host allocation failed during setup");
  } catch (const std::exception& e) {
    const std::string m = e.what();
    if (m.find("cudaMalloc") != std::string::npos) return fail(AMG_ERR_OOM, m);
    return fail(m.find("cuda") != std::string::npos ? AMG_ERR_CUDA : AMG_ERR_SETUP, m);
  }
  *out = h.release();
  return AMG_OK;
}

}  // namespace

amg_status amg_hierarchy_export(amg_handle h, const char* path) {
  if (!h || !path) return fail(AMG_ERR_ARG, "amg_hierarchy_export: null handle or path");
  try {
    write_hierarchy(h->host, h->symmetric, path);
  } catch (const std::exception& e) {
    return fail(AMG_ERR_ARG, std::string("amg_hierarchy_export: ") + e.what());
  }
  return AMG_OK;
}

amg_status amg_hierarchy_import(const char* path, const amg_params* prm_in, void* stream, amg_handle* out) {
  if (!path || !out) return fail(AMG_ERR_ARG, "amg_hierarchy_import: null path or output handle");
  *out = nullptr;
  amg_params prm;
  std::string why = check_params(prm_in, prm);
  if (!why.empty()) return fail(AMG_ERR_ARG, "amg_hierarchy_import: " + why);
  std::unique_ptr<amg_hierarchy> h(new amg_hierarchy());
  bool symmetric = true;
  try {
    h->host = read_hierarchy(path, &symmetric);
  } catch (const std::bad_alloc&) {
    return fail(AMG_ERR_OOM, "amg_hierarchy_import: host allocation failed");
  } catch (const std::exception& e) {
    return fail(AMG_ERR_ARG, std::string("amg_hierarchy_import: ") + e.what());
  }
  try {
    SetupParams sp = setup_params(prm, symmetric);
    const bool on_device = prm.device_setup && !prm.host_only;
    sp.dense_gs = !on_device;
    complete_hierarchy(h->host, sp, true);
    if (on_device) form_dense_gs_device(h->host, prm.gs_iters, (cudaStream_t)stream);
    h->prm = prm;
    h->symmetric = symmetric;
    upload_handle(h.get(), sp, stream);
  } catch (const std::bad_alloc&) {
    return fail(AMG_ERR_OOM, "amg_hierarchy_import: host allocation failed");
  } catch (const std::exception& e) {
    const std::string m = e.what();
    return fail(m.find("cuda") != std::string::npos ? AMG_ERR_CUDA : AMG_ERR_SETUP, "amg_hierarchy_import: " + m);
  }
  *out = h.release();
  return AMG_OK;
}

amg_status amg_vcycle_apply(amg_handle h, const double* r, double* z, int nrhs, void* stream) {
  if (!h || !r || !z) return fail(AMG_ERR_ARG, "null argument");
  if (!h->vc()) return fail(AMG_ERR_ARG, "hierarchy was built with host_only");
  if (nrhs < 1 || round_k(nrhs) > h->vc()->kmax()) return fail(AMG_ERR_ARG, "nrhs exceeds max_nrhs");
  try {
    if (h->prm.vcycle_fp32)
      vcycle_dispatch<float>(h, r, z, nrhs, (cudaStream_t)stream);
    else
      vcycle_dispatch<double>(h, r, z, nrhs, (cudaStream_t)stream);
  } catch (const std::exception& e) {
    return fail(AMG_ERR_CUDA, e.what());
  }
  return AMG_OK;
}

amg_status amg_apply(amg_handle h, const double* x, double* y, int nrhs, void* stream) {
  if (!h || !x || !y) return fail(AMG_ERR_ARG, "null argument");
  if (!h->vc()) return fail(AMG_ERR_ARG, "hierarchy was built with host_only");
  if (nrhs < 1 || round_k(nrhs) > h->vc()->kmax()) return fail(AMG_ERR_ARG, "nrhs exceeds max_nrhs");
  try {
    ensure_ws(h, round_k(nrhs), h->kry ? h->kry->m : 1);
    cudaStream_t s = (cudaStream_t)stream;
    switch (round_k(nrhs)) {
      case 1: apply_k<1>(h, x, y, nrhs, s); break;
      case 2: apply_k<2>(h, x, y, nrhs, s); break;
      case 4: apply_k<4>(h, x, y, nrhs, s); break;
      case 8: apply_k<8>(h, x, y, nrhs, s); break;
      case 16: apply_k<16>(h, x, y, nrhs, s); break;
      case 32: apply_k<32>(h, x, y, nrhs, s); break;
    }
  } catch (const std::exception& e) {
    return fail(AMG_ERR_CUDA, e.what());
  }
  return AMG_OK;
}

amg_status amg_fgmres_solve(amg_handle h, const double* b, double* x, int nrhs, double rtol, int restart, int maxit,
                            int* iters, double* relres, void* stream) {
  if (!h || !b || !x) return fail(AMG_ERR_ARG, "null argument");
  if (!h->vc()) return fail(AMG_ERR_ARG, "hierarchy was built with host_only");
  if (nrhs < 1 || round_k(nrhs) > h->vc()->kmax()) return fail(AMG_ERR_ARG, "nrhs exceeds max_nrhs");
  if (restart < 1 || maxit < 1 || !(rtol > 0.0)) return fail(AMG_ERR_ARG, "restart, maxit and rtol must be positive");
  try {
    return fgmres_blocking(h, b, x, nullptr, nullptr, nrhs, rtol, restart, maxit, iters, relres, (cudaStream_t)stream);
  } catch (const std::bad_alloc&) {
    return fail(AMG_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    const std::string m = e.what();
    return fail(m.find("cudaMalloc") != std::string::npos ? AMG_ERR_OOM : AMG_ERR_CUDA, m);
  }
}

amg_status amg_fgmres_solve_host(amg_handle h, const double* b_host, double* x_host, int nrhs, double rtol,
                                 int restart, int maxit, int* iters, double* relres, void* stream) {
  if (!h || !b_host || !x_host) return fail(AMG_ERR_ARG, "null argument");
  if (!h->vc()) return fail(AMG_ERR_ARG, "hierarchy was built with host_only");
  if (nrhs < 1 || round_k(nrhs) > h->vc()->kmax()) return fail(AMG_ERR_ARG, "nrhs exceeds max_nrhs");
  if (restart < 1 || maxit < 1 || !(rtol > 0.0)) return fail(AMG_ERR_ARG, "restart, maxit and rtol must be positive");
  if (!h->stage_b) {
    const size_t cap = sizeof(double) * (size_t)h->N * h->vc()->kmax();
    if (cudaMalloc(&h->stage_b, cap) != cudaSuccess || cudaMalloc(&h->stage_x, cap) != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it for the next launch checks
      if (h->stage_b) cudaFree(h->stage_b);
      if (h->stage_x) cudaFree(h->stage_x);
      h->stage_b = h->stage_x = nullptr;  // both or neither
      return fail(AMG_ERR_OOM, "cudaMalloc for the host-solve staging buffers");
    }
  }
  try {
    return fgmres_blocking(h, (const double*)h->stage_b, (double*)h->stage_x, b_host, x_host, nrhs, rtol, restart,
                           maxit, iters, relres, (cudaStream_t)stream);
  } catch (const std::bad_alloc&) {
    return fail(AMG_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    const std::string m = e.what();
    return fail(m.find("cudaMalloc") != std::string::npos ? AMG_ERR_OOM : AMG_ERR_CUDA, m);
  }
}

amg_status amg_profile_vcycle(amg_handle h, int nrhs, int reps, double* ms, long long* count, void* stream) {
  if (!h || !ms || !count || reps < 1) return fail(AMG_ERR_ARG, "null argument or reps < 1");
  if (!h->vc()) return fail(AMG_ERR_ARG, "hierarchy was built with host_only");
  if (nrhs < 1 || round_k(nrhs) > h->vc()->kmax()) return fail(AMG_ERR_ARG, "nrhs exceeds max_nrhs");
  const int n = h->vc()->levels() * kNumClasses;
  std::fill(ms, ms + n, 0.0);
  std::fill(count, count + n, 0LL);
  cudaError_t e = h->vc()->profile(round_k(nrhs), reps, (cudaStream_t)stream, ms, count);
  if (e != cudaSuccess) return fail(AMG_ERR_CUDA, cudaGetErrorString(e));
  return AMG_OK;
}

amg_status amg_profile_arnoldi(amg_handle h, int nrhs, int nv, int reps, double* ms_dot, double* ms_update,
                               void* stream) {
  if (!h || !ms_dot || !ms_update || reps < 1 || nv < 1) return fail(AMG_ERR_ARG, "null argument, reps or nv < 1");
  if (!h->vc()) return fail(AMG_ERR_ARG, "hierarchy was built with host_only");
  if (nrhs < 1 || round_k(nrhs) > h->vc()->kmax()) return fail(AMG_ERR_ARG, "nrhs exceeds max_nrhs");
  try {
    const int K = round_k(nrhs);
    ensure_ws(h, K, nv);
    switch (K) {
      case 1: profile_arnoldi_k<1>(h, nv, reps, ms_dot, ms_update, (cudaStream_t)stream); break;
      case 2: profile_arnoldi_k<2>(h, nv, reps, ms_dot, ms_update, (cudaStream_t)stream); break;
      case 4: profile_arnoldi_k<4>(h, nv, reps, ms_dot, ms_update, (cudaStream_t)stream); break;
      case 8: profile_arnoldi_k<8>(h, nv, reps, ms_dot, ms_update, (cudaStream_t)stream); break;
      case 16: profile_arnoldi_k<16>(h, nv, reps, ms_dot, ms_update, (cudaStream_t)stream); break;
      case 32: profile_arnoldi_k<32>(h, nv, reps, ms_dot, ms_update, (cudaStream_t)stream); break;
    }
  } catch (const std::bad_alloc&) {
    return fail(AMG_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    const std::string m = e.what();
    return fail(m.find("cudaMalloc") != std::string::npos ? AMG_ERR_OOM : AMG_ERR_CUDA, m);
  }
  return AMG_OK;
}

long long amg_kernel_launches(amg_handle h) {
  if (!h) return 0;
  return h->launches + (h->v64 ? h->v64->launches() : 0) + (h->v32 ? h->v32->launches() : 0);
}

int amg_num_levels(amg_handle h) { return h ? (int)h->host.size() : 0; }

amg_status amg_level_get_info(amg_handle h, int level, amg_level_info* info) {
  if (!h || !info || level < 0 || level >= (int)h->host.size()) return fail(AMG_ERR_ARG, "bad handle or level");
  const HostLevel& L = h->host[level];
  info->dim = L.dim;
  info->n_v = L.n_v;
  info->n_p = L.n_p;
  info->pinned = L.pinned;
  info->nnz_A = L.A.nnz();
  info->nnz_B = L.B.nnz();
  info->nnz_Bt = L.Bt.nnz();
  info->nnz_S = L.S.nnz();
  info->n_colors = L.n_colors;
  info->nnz_P = L.P.nnz();
  info->nnz_Pp = L.Pp.nnz();
  info->nnz_R = L.R.nnz();
  info->nnz_Rp = L.Rp.nnz();
  info->n_cp = (int)L.Cp.size();
  info->n_cv = (int)L.Cv.size();
  info->gs_strip = L.gs_strip;
  return AMG_OK;
}

amg_status amg_level_get_matrix(amg_handle h, int level, int which, long long* rowptr, int* col, double* val) {
  if (!h || level < 0 || level >= (int)h->host.size()) return fail(AMG_ERR_ARG, "bad handle or level");
  const HostLevel& L = h->host[level];
  const Csr* M = nullptr;
  switch (which) {
    case 0: M = &L.A; break;
    case 1: M = &L.B; break;
    case 2: M = &L.Bt; break;
    case 3: M = &L.S; break;
    case 4: M = &L.P; break;
    case 5: M = &L.Pp; break;
    case 6: M = &L.R; break;
    case 7: M = &L.Rp; break;
    default: return fail(AMG_ERR_ARG, "which must be 0..7");
  }
  if (rowptr)
    for (size_t i = 0; i < M->rowptr.size(); ++i) rowptr[i] = M->rowptr[i];
  if (col) std::copy(M->col.begin(), M->col.end(), col);
  if (val) std::copy(M->val.begin(), M->val.end(), val);
  return AMG_OK;
}

amg_status amg_level_get_points(amg_handle h, int level, int* cp, int* cv, int* colors, double* D) {
  if (!h || level < 0 || level >= (int)h->host.size()) return fail(AMG_ERR_ARG, "bad handle or level");
  const HostLevel& L = h->host[level];
  if (cp) std::copy(L.Cp.begin(), L.Cp.end(), cp);
  if (cv) std::copy(L.Cv.begin(), L.Cv.end(), cv);
  if (colors) std::copy(L.colors.begin(), L.colors.end(), colors);
  if (D) std::copy(L.D.begin(), L.D.end(), D);
  return AMG_OK;
}

amg_status amg_level_get_vanka(amg_handle h, int level, int* nblocks, int* ndofs, int* ncolors, int* ptr,
                               int* dofs, int* colors) {
  if (!h || level < 0 || level >= (int)h->host.size()) return fail(AMG_ERR_ARG, "bad handle or level");
  const HostLevel& L = h->host[level];
  if (L.vk_ptr.empty()) return fail(AMG_ERR_ARG, "the level has no Vanka blocks");
  if (nblocks) *nblocks = (int)L.vk_ptr.size() - 1;
  if (ndofs) *ndofs = (int)L.vk_dofs.size();
  if (ncolors) *ncolors = L.vk_ncolors;
  if (ptr) std::copy(L.vk_ptr.begin(), L.vk_ptr.end(), ptr);
  if (dofs) std::copy(L.vk_dofs.begin(), L.vk_dofs.end(), dofs);
  if (colors) std::copy(L.vk_colors.begin(), L.vk_colors.end(), colors);
  return AMG_OK;
}

amg_status amg_level_get_ilu(amg_handle h, int level, int* n, long long* nnz_lower, long long* nnz_upper,
                             int* depth_lower, int* depth_upper, int* perm, int* lower_ptr, int* lower_col,
                             double* lower_val, int* upper_ptr, int* upper_col, double* upper_val, double* pivots) {
  if (!h || level < 0 || level >= (int)h->host.size()) return fail(AMG_ERR_ARG, "bad handle or level");
  const HostLevel& L = h->host[level];
  if (L.il_perm.empty()) return fail(AMG_ERR_ARG, "the level has no ILU(1) factors");
  if (n) *n = L.N();
  if (nnz_lower) *nnz_lower = L.il_L.nnz();
  if (nnz_upper) *nnz_upper = L.il_U.nnz();
  if (depth_lower) *depth_lower = L.il_depthL;
  if (depth_upper) *depth_upper = L.il_depthU;
  if (perm) std::copy(L.il_perm.begin(), L.il_perm.end(), perm);
  if (lower_ptr) std::copy(L.il_L.rowptr.begin(), L.il_L.rowptr.end(), lower_ptr);
  if (lower_col) std::copy(L.il_L.col.begin(), L.il_L.col.end(), lower_col);
  if (lower_val) std::copy(L.il_L.val.begin(), L.il_L.val.end(), lower_val);
  if (upper_ptr) std::copy(L.il_U.rowptr.begin(), L.il_U.rowptr.end(), upper_ptr);
  if (upper_col) std::copy(L.il_U.col.begin(), L.il_U.col.end(), upper_col);
  if (upper_val) std::copy(L.il_U.val.begin(), L.il_U.val.end(), upper_val);
  if (pivots) std::copy(L.il_diag.begin(), L.il_diag.end(), pivots);
  return AMG_OK;
}

amg_status amg_level_get_gs_map(amg_handle h, int level, int* n, double* M) {
  if (!h || level < 0 || level >= (int)h->host.size()) return fail(AMG_ERR_ARG, "bad handle or level");
  const HostLevel& L = h->host[level];
  if (L.gs_dense.empty()) return fail(AMG_ERR_ARG, "the level has no dense Gauss-Seidel map");
  if (n) *n = L.n_p;
  if (M) std::copy(L.gs_dense.begin(), L.gs_dense.end(), M);
  return AMG_OK;
}

amg_status amg_coarse_inverse(amg_handle h, int* n, double* X) {
  if (!h || h->host.empty()) return fail(AMG_ERR_ARG, "bad handle");
  const HostLevel& C = h->host.back();
  if (n) *n = C.N();
  if (X) std::copy(C.pinv.begin(), C.pinv.end(), X);
  return AMG_OK;
}

amg_status amg_set_wait_limit(amg_handle h, long long polls) {
  if (!h) return fail(AMG_ERR_ARG, "bad handle");
  const unsigned long long lim = polls > 0 ? (unsigned long long)polls : kSpinLimit;
  for (VCycleIface* v : {h->v64, h->v32}) {
    if (!v) continue;
    const cudaError_t e = v->set_wait_limit(lim);
    if (e != cudaSuccess) return fail(AMG_ERR_CUDA, std::string("amg_set_wait_limit: ") + cudaGetErrorString(e));
  }
  return AMG_OK;
}

int amg_gs_variant(amg_handle h, int level, int nrhs, int* cluster, float* ms) {
  if (!h || !h->vc() || nrhs < 1 || nrhs > 32) return -1;
  return h->vc()->gs_choice(level, round_k(nrhs), cluster, ms);
}

amg_status amg_set_gs_variant(amg_handle h, int level, int nrhs, int variant, int cluster) {
  if (!h || !h->vc()) return fail(AMG_ERR_ARG, "amg_set_gs_variant: null handle or host-only hierarchy");
  if (nrhs < 1 || nrhs > 32) return fail(AMG_ERR_ARG, "amg_set_gs_variant: nrhs must be in 1..32");
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(AMG_ERR_CUDA, "amg_set_gs_variant: device synchronise");
  const int K = round_k(nrhs);
  for (VCycleIface* vc : {h->v32, h->v64})
    if (vc && K <= vc->kmax() && !vc->set_gs_choice(level, K, variant, cluster))
      return fail(AMG_ERR_ARG, "amg_set_gs_variant: the variant does not apply to this level and nrhs");
  return AMG_OK;
}

int amg_row_shape(amg_handle h, int level, int nrhs, int kernel) {
  if (!h || !h->vc() || nrhs < 1 || nrhs > 32) return -1;
  return h->vc()->row_shape(level, round_k(nrhs), kernel);
}

void amg_hierarchy_destroy(amg_handle h) { delete h; }

}  // extern "C"

// Device-resident hierarchy and the V-cycle driver (Alg. 1's cycle) for one
// arithmetic type T.  The cycle for K right-hand sides is captured once into a
// CUDA graph and replayed.
#pragma once

#include <cuda_runtime.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "device.cuh"
#include "setup.hpp"

namespace emin {

// Type-erased V-cycle so the FGMRES driver can hold an FP64 or an FP32 one.
struct VCycleIface {
  virtual ~VCycleIface() = default;
  virtual bool is_fp32() const = 0;
  virtual int kmax() const = 0;
  virtual void* input(int level) = 0;   // level's right-hand side buffer, N_l x K
  virtual void* output(int level) = 0;  // level's solution buffer, N_l x K
  // Enqueue one cycle on level 0 (reads input(0), writes output(0)).
  virtual cudaError_t run(int K, cudaStream_t s) = 0;
  virtual size_t device_bytes() const = 0;
  virtual int levels() const = 0;
  // Run `reps` cycles without the graph, with CUDA events around every launch;
  // add each launch's time to ms[level * kNumClasses + class] and count it.
  virtual cudaError_t profile(int K, int reps, cudaStream_t s, double* ms, long long* count) = 0;
  // Kernels launched so far by run() and profile() (graph replays count every kernel node).
  virtual long long launches() const = 0;
};

// Kernel classes reported by profile().
enum KernelClass { kVelocity = 0, kSchurRhs, kGsColor, kUpdate, kResidual, kRestrict, kProlong, kCoarse, kNumClasses };

#define EMIN_CUDA(call)                                                                 \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw std::runtime_error(std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

template <typename T>
class DeviceVCycle : public VCycleIface {
 public:
  struct Buf {
    T *b = nullptr, *x = nullptr, *y = nullptr, *g = nullptr, *dp = nullptr, *r = nullptr;
  };

  DeviceVCycle(const std::vector<HostLevel>& levels, double cfac, int gs_iters, int pre, int post, int kmax)
      : c_(cfac), cfac_((T)cfac), gs_iters_(gs_iters), pre_(pre), post_(post), kmax_(kmax) {
    try {
      for (size_t l = 0; l < levels.size(); ++l) upload_level(levels[l], l + 1 == levels.size());
      for (size_t l = 0; l + 1 < levels.size(); ++l) {
        views_[l].n_vc = levels[l + 1].n_v;
        views_[l].n_pc = levels[l + 1].n_p;
      }
      const HostLevel& C = levels.back();
      Nc_ = C.N();
      pinv_ = alloc_copy<double>(C.pinv);
    } catch (...) {
      release();
      throw;
    }
  }
  ~DeviceVCycle() override { release(); }

  bool is_fp32() const override { return sizeof(T) == 4; }
  int kmax() const override { return kmax_; }
  void* input(int level) override { return buf_[level].b; }
  void* output(int level) override { return buf_[level].x; }
  size_t device_bytes() const override { return bytes_; }
  const LevelView<T>& view(int l) const { return views_[l]; }
  int num_levels() const { return (int)views_.size(); }
  int levels() const override { return (int)views_.size(); }

  cudaError_t profile(int K, int reps, cudaStream_t s, double* ms, long long* count) override {
    if (kslot(K) < 0 || K > kmax_) return cudaErrorInvalidValue;
    for (int rep = 0; rep < reps; ++rep) {
      recs_.clear();
      enq_kernels_ = 0;
      prof_on_ = true;
      switch (K) {
        case 1: enqueue<1>(s); break;
        case 2: enqueue<2>(s); break;
        case 4: enqueue<4>(s); break;
        case 8: enqueue<8>(s); break;
        case 16: enqueue<16>(s); break;
        case 32: enqueue<32>(s); break;
      }
      prof_on_ = false;
      launches_ += enq_kernels_;
      cudaError_t e = cudaStreamSynchronize(s);
      for (auto& r : recs_) {
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        ms[r.level * kNumClasses + r.cls] += t;
        count[r.level * kNumClasses + r.cls] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
      }
      recs_.clear();
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }

  cudaError_t run(int K, cudaStream_t s) override {
    const int slot = kslot(K);
    if (slot < 0 || K > kmax_) return cudaErrorInvalidValue;
    if (!graphs_[slot]) {
      cudaError_t e = capture(K, slot);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGraphLaunch(graphs_[slot], s);
    if (e == cudaSuccess) launches_ += graph_kernels_[slot];
    return e;
  }
  long long launches() const override { return launches_; }

  // Enqueue the cycle without a graph (used for capture).
  template <int K>
  void enqueue(cudaStream_t s) {
    const int nl = (int)views_.size();
    for (int l = 0; l + 1 < nl; ++l) {
      smooth<K>(l, pre_, true, s);
      const LevelView<T>& L = views_[l];
      mark_begin(l, kResidual, s);
      k_block_spmv<T, T, T, K, true><<<grid_for((long long)(L.n_v + L.n_p) * K), kBlock, 0, s>>>(
          L, buf_[l].b, buf_[l].x, buf_[l].r);
      mark_end(s);
      mark_begin(l, kRestrict, s);
      k_restrict<T, K><<<grid_for((long long)(L.n_vc + L.n_pc) * K), kBlock, 0, s>>>(L, buf_[l].r, buf_[l + 1].b);
      mark_end(s);
    }
    mark_begin(nl - 1, kCoarse, s);  // every kernel launch of the cycle is preceded by mark_begin
    k_coarse_solve<T, K><<<grid_for((long long)Nc_ * K), kBlock, 0, s>>>(Nc_, pinv_, buf_[nl - 1].b, buf_[nl - 1].x);
    mark_end(s);
    for (int l = nl - 2; l >= 0; --l) {
      const LevelView<T>& L = views_[l];
      mark_begin(l, kProlong, s);
      k_prolong<T, K><<<grid_for((long long)(L.n_v + L.n_p) * K), kBlock, 0, s>>>(L, buf_[l + 1].x, buf_[l].x);
      mark_end(s);
      smooth<K>(l, post_, false, s);
    }
  }

 private:
  static int kslot(int K) {
    switch (K) {
      case 1: return 0;
      case 2: return 1;
      case 4: return 2;
      case 8: return 3;
      case 16: return 4;
      case 32: return 5;
      default: return -1;
    }
  }

  template <int K>
  void smooth(int l, int sweeps, bool from_zero, cudaStream_t s) {
    const LevelView<T>& L = views_[l];
    const Buf& B = buf_[l];
    const std::vector<int>& off = color_off_[l];
    for (int sw = 0; sw < sweeps; ++sw) {
      const int zero = (from_zero && sw == 0) ? 1 : 0;
      mark_begin(l, kVelocity, s);
      k_bs_velocity<T, K><<<grid_for((long long)L.n_v * K), kBlock, 0, s>>>(L, B.b, B.x, B.y, zero);
      mark_end(s);
      mark_begin(l, kSchurRhs, s);
      k_schur_rhs<T, K><<<grid_for((long long)L.n_p * K), kBlock, 0, s>>>(L, B.b, B.x, B.y, B.g, cfac_, zero);
      mark_end(s);
      cudaMemsetAsync(B.dp, 0, sizeof(T) * (size_t)L.n_p * K, s);
      for (int it = 0; it < gs_iters_; ++it)
        for (size_t c = 0; c + 1 < off.size(); ++c) {
          mark_begin(l, kGsColor, s);
          k_gs_color<T, K><<<grid_for((long long)(off[c + 1] - off[c]) * K), kBlock, 0, s>>>(L, B.g, B.dp, off[c],
                                                                                              off[c + 1]);
          mark_end(s);
        }
      mark_begin(l, kUpdate, s);
      k_bs_update<T, K><<<grid_for((long long)(L.n_v + L.n_p) * K), kBlock, 0, s>>>(L, B.y, B.dp, B.x, zero);
      mark_end(s);
    }
  }

  struct Rec {
    int level, cls;
    cudaEvent_t a, b;
  };
  void mark_begin(int level, int cls, cudaStream_t s) {
    ++enq_kernels_;
    if (!prof_on_) return;
    Rec r{level, cls, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, s);
    recs_.push_back(r);
  }
  void mark_end(cudaStream_t s) {
    if (prof_on_) cudaEventRecord(recs_.back().b, s);
  }

  cudaError_t capture(int K, int slot) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    enq_kernels_ = 0;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      switch (K) {
        case 1: enqueue<1>(cs); break;
        case 2: enqueue<2>(cs); break;
        case 4: enqueue<4>(cs); break;
        case 8: enqueue<8>(cs); break;
        case 16: enqueue<16>(cs); break;
        case 32: enqueue<32>(cs); break;
      }
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaGraphInstantiate(&graphs_[slot], g, 0);
    graph_kernels_[slot] = enq_kernels_;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e;
  }

  template <typename U>
  U* alloc(size_t n) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(U);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) throw std::runtime_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs_.push_back(p);
    bytes_ += bytes;
    return (U*)p;
  }
  template <typename U, typename V>
  U* alloc_copy(const std::vector<V>& h) {
    std::vector<U> tmp(h.begin(), h.end());
    U* d = alloc<U>(tmp.size());
    if (!tmp.empty()) EMIN_CUDA(cudaMemcpy(d, tmp.data(), tmp.size() * sizeof(U), cudaMemcpyHostToDevice));
    return d;
  }
  DCsr<T> upload(const Csr& M) {
    DCsr<T> d;
    d.nrows = M.nrows;
    std::vector<int> rp(M.rowptr.begin(), M.rowptr.end());
    if (M.rowptr.empty()) rp.assign(1, 0);
    d.rp = alloc_copy<int>(rp);
    d.ci = alloc_copy<int>(M.col);
    d.v = alloc_copy<T>(M.val);
    return d;
  }

  void upload_level(const HostLevel& H, bool coarsest) {
    LevelView<T> L{};
    L.dim = H.dim;
    L.n_v = H.n_v;
    L.n_p = H.n_p;
    L.pinned = H.pinned;
    L.A = upload(H.A);
    L.B = upload(H.B);
    L.Bt = upload(H.Bt);
    // Schur complement rows grouped by color, diagonal split off
    std::vector<int> perm(H.n_p), off(H.n_colors + 1, 0);
    for (int i = 0; i < H.n_p; ++i) off[H.colors[i] + 1]++;
    for (int c = 0; c < H.n_colors; ++c) off[c + 1] += off[c];
    {
      std::vector<int> pos(off.begin(), off.end() - 1);
      for (int i = 0; i < H.n_p; ++i) perm[pos[H.colors[i]]++] = i;
    }
    Csr So;
    So.resize_rows(H.n_p, H.n_p);
    std::vector<double> dinv(H.n_p, 0.0);
    for (int r = 0; r < H.n_p; ++r) {
      const int i = perm[r];
      double diag = 0.0;
      for (int64_t t = H.S.row_begin(i); t < H.S.row_end(i); ++t) {
        if (H.S.col[t] == i) {
          diag += H.S.val[t];
        } else {
          So.col.push_back(H.S.col[t]);
          So.val.push_back(H.S.val[t]);
        }
      }
      dinv[r] = diag != 0.0 ? 1.0 / diag : 0.0;
      So.rowptr[r + 1] = (int64_t)So.col.size();
    }
    L.S = upload(So);
    L.S_perm = alloc_copy<int>(perm);
    L.S_dinv = alloc_copy<T>(dinv);
    std::vector<double> w(H.n_v);
    for (int i = 0; i < H.n_v; ++i) w[i] = H.dirichlet[i] ? 1.0 : 1.0 / (c_ * H.D[i]);
    L.w = alloc_copy<T>(w);
    if (!coarsest) {
      L.P = upload(H.P);
      L.Pp = upload(H.Pp);
      L.R = upload(H.R);
      L.Rp = upload(H.Rp);
    }
    const size_t N = (size_t)H.N() * kmax_;
    Buf B;
    B.b = alloc<T>(N);
    B.x = alloc<T>(N);
    B.r = alloc<T>(N);
    B.y = alloc<T>((size_t)H.dim * H.n_v * kmax_);
    B.g = alloc<T>((size_t)H.n_p * kmax_);
    B.dp = alloc<T>((size_t)H.n_p * kmax_);
    views_.push_back(L);
    buf_.push_back(B);
    color_off_.push_back(off);
  }

  void release() {
    for (auto& g : graphs_)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
    for (void* p : allocs_) cudaFree(p);
    allocs_.clear();
  }

  double c_;
  T cfac_;
  int gs_iters_, pre_, post_, kmax_;
  std::vector<LevelView<T>> views_;
  std::vector<Buf> buf_;
  std::vector<std::vector<int>> color_off_;
  double* pinv_ = nullptr;
  int Nc_ = 0;
  std::vector<void*> allocs_;
  size_t bytes_ = 0;
  cudaGraphExec_t graphs_[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool prof_on_ = false;
  std::vector<Rec> recs_;
  long long enq_kernels_ = 0, launches_ = 0;
  long long graph_kernels_[6] = {0, 0, 0, 0, 0, 0};
};

// Factories, one translation unit per type.
VCycleIface* make_vcycle_f64(const std::vector<HostLevel>& levels, double cfac, int gs, int pre, int post, int kmax);
VCycleIface* make_vcycle_f32(const std::vector<HostLevel>& levels, double cfac, int gs, int pre, int post, int kmax);
// Finest-level FP64 block product out = A x (TX = double or float), or out = b - A x.
cudaError_t apply_finest_f64(VCycleIface* v64, const void* x, bool x_fp32, const double* b, double* out, int K,
                             cudaStream_t s);

}  // namespace emin

// Device-resident hierarchy and the V-cycle driver (Alg. 1's cycle) for one
// arithmetic type T.  The cycle for K right-hand sides is captured once into a
// CUDA graph and replayed.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "device.cuh"
#include "setup.hpp"
#include "trace.hpp"

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
  // Capture the cycle's graph for K without running it (run() captures on first use).
  virtual cudaError_t prepare(int K) = 0;
  virtual size_t device_bytes() const = 0;
  virtual int levels() const = 0;
  // Run `reps` cycles without the graph, with CUDA events around every launch;
  // add each launch's time to ms[level * kNumClasses + class] and count it.
  virtual cudaError_t profile(int K, int reps, cudaStream_t s, double* ms, long long* count) = 0;
  // Kernels launched so far by run() and profile() (graph replays count every kernel node).
  virtual long long launches() const = 0;
  // Device word set when a bounded wait timed out (0 otherwise).
  virtual int* error_flag() const = 0;
  // Poll limit of this cycle's bounded waits (kSpinLimit by default); synchronous.
  virtual cudaError_t set_wait_limit(unsigned long long polls) = 0;
  // FP32 cycles only: out = A z on the finest level for an FP32 z, FP64 result by
  // float-float arithmetic on the FP64 matrix split into two floats.
  virtual cudaError_t apply_ff(const float* z, double* out, int K, cudaStream_t s) = 0;
  // A second cycle on the same device-resident hierarchy: it shares every matrix
  // (read-only) and owns its vectors, counters, error word and graphs, so cycles of
  // the original and its clones can run at the same time on different streams.
  // The original must outlive its clones.  Throws std::runtime_error on failure.
  virtual VCycleIface* clone(int kmax) const = 0;
  // Device bytes a clone with kmax right-hand sides allocates.
  virtual size_t clone_bytes(int kmax) const = 0;
  // Gauss-Seidel variant selection: timed per (level, K) before the first capture
  // when on (the default), fixed heuristics when off.  gs_choice reports the
  // variant of a level for K (-1 not tuned yet, 0 one block, 1 cluster, 2
  // pipelined, 3 one launch per phase), the cluster size and the time measured.
  virtual void set_autotune(bool on) = 0;
  virtual int gs_choice(int level, int K, int* cluster, float* ms) const = 0;
  // Fix the variant of a level for K (the autotuner then leaves it): returns false
  // when the level, K or the variant does not apply (a dense map on a level without
  // one, a cluster size without a plan, a pipelined shape outside 0-3).  A cycle already captured for K is
  // dropped and captured again on its next run.  Not for a cycle whose clones run.
  virtual bool set_gs_choice(int level, int K, int kind, int C) = 0;
  // Row mapping (0-3, see DeviceVCycle::Shape) of a sparse kernel class on a level
  // for K right-hand sides, as tuned or by default; -1 for a bad argument.
  virtual int row_shape(int level, int K, int cls) const = 0;
};

// Kernel classes reported by profile().
enum KernelClass {
  kVelocity = 0, kSchurRhs, kGsColor, kUpdate, kResidual, kRestrict, kProlong, kCoarse, kVanka, kIlu, kNumClasses
};

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
    T* iy = nullptr;  // ILU substitutions' outputs, 2 x N_l x K (ILU cycles only)
  };
  // Strips of a level split over a cluster of C blocks (k_gs_cluster): block c owns
  // spc consecutive strips; plist / poff as GsCluster; extents are maxima over blocks.
  enum GsKind { kGsSingle = 0, kGsCluster = 1, kGsPipe = 2, kGsPhases = 3, kGsDense = 4 };
  struct GsChoice {
    int kind = -1;  // GsKind, -1 = not tuned yet
    int C = 0;      // cluster size; shape of the pipelined kernel (0 heuristic, 1-3 launch_gs_pipe)
    float ms = 0.f; // measured time per launch
  };
  struct ClusterPlan {
    int C = 0, spc = 0, win_max = 0, rows_max = 0, nnz_max = 0;
    int* plist = nullptr;
    int* poff = nullptr;
  };

  DeviceVCycle(const std::vector<HostLevel>& levels, double cfac, int gs_iters, int pre, int post, int kmax,
               double vanka_omega = 0.0, bool ilu = false, double coarse_omega = 0.0)
      : c_(cfac), cfac_((T)cfac), gs_iters_(gs_iters), pre_(pre), post_(post), kmax_(kmax),
        vanka_omega_((T)vanka_omega), ilu_(ilu), coarse_vanka_(coarse_omega > 0.0),
        vk_omega_((T)(vanka_omega > 0.0 ? vanka_omega : coarse_omega)) {
    try {
      if ((long long)levels[0].N() * kmax_ >= (1LL << 31))
        throw std::runtime_error("N * max_nrhs must stay below 2^31 (32-bit vector indices)");
      for (size_t l = 0; l < levels.size(); ++l) upload_level(levels[l], l + 1 == levels.size());
      vk_.resize(levels.size());
      if (vanka_omega > 0.0)
        for (size_t l = 0; l + 1 < levels.size(); ++l) upload_vanka(levels[l], l);
      if (coarse_vanka_) upload_vanka(levels.back(), levels.size() - 1);
      if (ilu_) {
        for (size_t l = 0; l + 1 < levels.size(); ++l) upload_ilu(levels[l]);
        il_ticket_ = alloc<int>(1);
        EMIN_CUDA(cudaMemset(il_ticket_, 0, sizeof(int)));
      }
      tune_ = std::make_shared<std::vector<GsChoice>>(levels.size() * 6);
      rowmap_ = std::make_shared<std::vector<int>>(levels.size() * 6 * kRowClasses, -1);
      vkform_ = std::make_shared<std::vector<int>>(levels.size() * 6, -1);
      ilgrid_ = std::make_shared<std::vector<int>>(levels.size() * 6, -1);
      for (size_t l = 0; l + 1 < levels.size(); ++l) {
        views_[l].n_vc = levels[l + 1].n_v;
        views_[l].n_pc = levels[l + 1].n_p;
      }
      const HostLevel& C = levels.back();
      Nc_ = C.N();
      pinv_ = alloc_copy<double>(C.pinv);
      if (sizeof(T) == 4) build_ff(levels[0]);
      err_ = alloc<int>(4);
      EMIN_CUDA(cudaMemset(err_, 0, 4 * sizeof(int)));
      EMIN_CUDA(set_wait_limit(kSpinLimit));
    } catch (...) {
      release();
      throw;
    }
  }
  ~DeviceVCycle() override { release(); }
  DeviceVCycle(const DeviceVCycle&) = delete;
  DeviceVCycle& operator=(const DeviceVCycle&) = delete;

  VCycleIface* clone(int kmax) const override { return new DeviceVCycle(*this, kmax, CloneTag{}); }
  void set_autotune(bool on) override { autotune_ = on; }
  int row_shape(int level, int K, int cls) const override {
    if (level < 0 || level + 1 >= (int)views_.size() || kslot(K) < 0 || cls < 0 || cls >= kRowClasses) return -1;
    return shape(level, K, cls);
  }
  int gs_choice(int level, int K, int* cluster, float* ms) const override {
    if (level < 0 || level >= (int)views_.size() || kslot(K) < 0) return -1;
    const GsChoice& c = (*tune_)[(size_t)level * 6 + kslot(K)];
    if (cluster) *cluster = c.C;
    if (ms) *ms = c.ms;
    return c.kind;
  }
  bool set_gs_choice(int level, int K, int kind, int C) override {
    const int ks = kslot(K);
    if (level < 0 || level >= (int)views_.size() || ks < 0 || K > kmax_) return false;
    switch (kind) {
      case kGsSingle: case kGsPhases: break;
      case kGsCluster: {
        bool found = false;
        for (const ClusterPlan& P : cplans_[level]) found = found || P.C == C;
        if (!found) return false;
        break;
      }
      case kGsPipe:
        if (C < 0 || C > 3 || gs_stage(level, K) <= 0 || gs_[level].ncol > kMaxColors) return false;
        break;
      case kGsDense:
        if (!gsM_[level] || C != 0) return false;
        break;
      default: return false;
    }
    (*tune_)[(size_t)level * 6 + ks] = {kind, C, 0.f};
    if (graphs_[ks]) {
      cudaGraphExecDestroy(graphs_[ks]);
      graphs_[ks] = nullptr;
    }
    return true;
  }
  size_t clone_bytes(int kmax) const override {
    size_t b = 256;
    for (size_t l = 0; l < views_.size(); ++l) {
      const LevelView<T>& L = views_[l];
      const size_t N = (size_t)L.dim * L.n_v + L.n_p;
      b += ((3 * N + (size_t)L.dim * L.n_v + 2 * (size_t)L.n_p) * kmax * sizeof(T) + 255) / 256 * 256;
      if (ilu_ && l + 1 < views_.size()) b += (2 * N * kmax * sizeof(T) + 255) / 256 * 256;
    }
    for (const GsStrips& P : gs_) b += ((size_t)(P.nstrips + 1) * sizeof(int) + 255) / 256 * 256;
    return b;
  }

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
    try {
      if (autotune_) tune_for(K, s);
    } catch (const std::exception&) {
      return cudaErrorLaunchFailure;
    }
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

  cudaError_t prepare(int K) override {
    const int slot = kslot(K);
    if (slot < 0 || K > kmax_) return cudaErrorInvalidValue;
    return graphs_[slot] ? cudaSuccess : capture(K, slot);
  }

  // Enqueue the cycle without a graph (used for capture).
  template <int K>
  void enqueue(cudaStream_t s) {
    const int nl = (int)views_.size();
    for (int l = 0; l + 1 < nl; ++l) {
      smooth<K>(l, pre_, true, s);
      mark_begin(l, kResidual, s);
      launch_rows<K>(kResidual, l, shape(l, K, kResidual), 0, s);
      mark_end(s);
      mark_begin(l, kRestrict, s);
      launch_rows<K>(kRestrict, l, shape(l, K, kRestrict), 0, s);
      mark_end(s);
    }
    if (coarse_vanka_) {
      // the paper's coarsest relaxation: pre + post Vanka steps from zero
      for (int sw = 0; sw < std::max(1, pre_ + post_); ++sw) vanka_sweep<K>(nl - 1, sw == 0, s);
    } else {
      mark_begin(nl - 1, kCoarse, s);  // every kernel launch of the cycle is preceded by mark_begin
      k_coarse_solve<T, K><<<grid_for((long long)Nc_ * 32), kBlock, 0, s>>>(Nc_, pinv_, buf_[nl - 1].b, buf_[nl - 1].x);
      mark_end(s);
    }
    for (int l = nl - 2; l >= 0; --l) {
      mark_begin(l, kProlong, s);
      launch_rows<K>(kProlong, l, shape(l, K, kProlong), 0, s);
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

  // Row mappings of the sparse kernels (velocity, Schur RHS, update, residual,
  // restriction, prolongation): shape 0 one thread group of K/V threads per row
  // with V = 16 bytes of right-hand sides each; shapes 1 and 2 split a row's
  // entries over 2 or 4 such groups (warp-shuffle sums); shape 3 one column per
  // thread and RowLanes<K>::G lanes per row (the mapping for latency-bound small
  // levels).  The autotuner picks one per (level, K, kernel); without it, shape 3
  // on small levels and shape 0 elsewhere.
  template <int K, int SHAPE>
  struct Shape {
    static constexpr int V = SHAPE == 3 ? 1 : VecWidth<T, K>::V;
    static constexpr int KV = K / V;
    static constexpr int G0 = SHAPE == 0 ? 1 : SHAPE == 1 ? 2 : SHAPE == 2 ? 4 : RowLanes<K>::G;
    static constexpr int G = G0 * KV <= 32 ? G0 : (KV >= 32 ? 1 : 32 / KV);
    static constexpr int W = KV * G;
  };
  static constexpr int kRowShapes = 4;
  static constexpr int kRowClasses = kNumClasses;  // indexed by KernelClass

  int shape(int l, int K, int cls) const {
    const int v = (*rowmap_)[((size_t)l * 6 + kslot(K)) * kRowClasses + cls];
    if (v >= 0) return v;
    return small_level(cls == kRestrict ? l + 1 : l, K) ? 3 : 0;
  }

  template <int K>
  void launch_rows(int cls, int l, int shp, int zero, cudaStream_t s) {
    switch (shp) {
      case 1: return launch_rows_as<K, 1>(cls, l, zero, s);
      case 2: return launch_rows_as<K, 2>(cls, l, zero, s);
      case 3: return launch_rows_as<K, 3>(cls, l, zero, s);
      default: return launch_rows_as<K, 0>(cls, l, zero, s);
    }
  }
  template <int K, int SHAPE>
  void launch_rows_as(int cls, int l, int zero, cudaStream_t s) {
    using S = Shape<K, SHAPE>;
    constexpr int G = S::G, V = S::V, W = S::W;
    const LevelView<T>& L = views_[l];
    const Buf& B = buf_[l];
    switch (cls) {
      case kVelocity:
        k_bs_velocity<T, K, G, V><<<grid_for((long long)L.n_v * W), kBlock, 0, s>>>(L, B.b, B.x, B.y, zero);
        break;
      case kSchurRhs:
        k_schur_rhs<T, K, G, V><<<grid_for((long long)L.n_p * W), kBlock, 0, s>>>(L, B.b, B.x, B.y, B.g, cfac_, zero);
        break;
      case kUpdate:
        k_bs_update<T, K, G, V><<<grid_for((long long)(L.n_v + L.n_p) * W), kBlock, 0, s>>>(L, B.y, B.dp, B.x, zero);
        break;
      case kResidual:
        k_block_spmv<T, K, G, V, true><<<grid_for((long long)(L.n_v + L.n_p) * W), kBlock, 0, s>>>(L, B.b, B.x, B.r);
        break;
      case kRestrict:
        k_restrict<T, K, G, V><<<grid_for((long long)(L.n_vc + L.n_pc) * W), kBlock, 0, s>>>(L, B.r, buf_[l + 1].b);
        break;
      case kProlong:
        k_prolong<T, K, G, V><<<grid_for((long long)(L.n_v + L.n_p) * W), kBlock, 0, s>>>(L, buf_[l + 1].x, B.x);
        break;
    }
  }

  // Vanka step (Section 5.1): the Dirichlet dofs exactly, then one launch per color.
  template <int K>
  void vanka_sweep(int l, bool from_zero, cudaStream_t s) {
    const Buf& B = buf_[l];
    const VankaLevel& V = vk_[l];
    const LevelView<T>& L = views_[l];
    if (from_zero) cudaMemsetAsync(B.x, 0, sizeof(T) * ((size_t)L.dim * L.n_v + L.n_p) * K, s);
    if (V.n_dirichlet > 0) {
      mark_begin(l, kVanka, s);
      k_vanka_exact<T, K><<<grid_for((long long)V.n_dirichlet * K), kBlock, 0, s>>>(V.n_dirichlet, V.dirichlet, B.b, B.x);
      mark_end(s);
    }
    const int form = (*vkform_)[(size_t)l * 6 + kslot(K)];
    for (size_t c = 0; c + 1 < V.coff.size(); ++c) {
      if (V.coff[c + 1] == V.coff[c]) continue;
      mark_begin(l, kVanka, s);
      vanka_color<K>(l, (int)c, form < 0 ? 0 : form, s);
      mark_end(s);
    }
  }
  // ILU(1) step (Section 5): r = b - A x (r = b from x = 0), then the forward and the
  // backward substitution, the second adding (L U)^-1 r to x.
  template <int K>
  void ilu_sweep(int l, bool from_zero, cudaStream_t s) {
    const Buf& B = buf_[l];
    const IluLevel& I = il_[l];
    const T* r = B.b;
    if (!from_zero) {
      mark_begin(l, kResidual, s);
      launch_rows<K>(kResidual, l, shape(l, K, kResidual), 0, s);
      mark_end(s);
      r = B.r;
    }
    const int tuned = (*ilgrid_)[(size_t)l * 6 + kslot(K)];
    ilu_substitutions<K>(l, r, from_zero, tuned > 0 ? tuned : I.blocks, true, s);
  }
  template <int K>
  void ilu_substitutions(int l, const T* r, bool zero, int blocks, bool marks, cudaStream_t s) {
    const Buf& B = buf_[l];
    const IluLevel& I = il_[l];
    const size_t n = (size_t)I.view.n * K;
    cudaMemsetAsync(B.iy, 0xff, sizeof(T) * 2 * n, s);
    if (marks) mark_begin(l, kIlu, s);
    k_ilu_lower<T, K><<<blocks, kIluBlock, 0, s>>>(I.view, r, B.iy, il_ticket_, err_);
    if (marks) mark_end(s);
    if (marks) mark_begin(l, kIlu, s);
    k_ilu_upper<T, K><<<blocks, kIluBlock, 0, s>>>(I.view, B.iy, B.iy + n, B.x, zero ? 1 : 0, il_ticket_, err_);
    if (marks) mark_end(s);
  }
  // ILU grid autotuner: both substitutions of each level timed (CUDA events) with 1, 2,
  // 4, 8 and 16 warps per row of an average dependency level (within 32 warps and 32
  // per SM); the fastest kept in a table shared with the clones.
  template <int K>
  void tune_ilu(cudaStream_t s) {
    if (!ilu_) return;
    const int ks = kslot(K);
    cudaEvent_t e0, e1;
    EMIN_CUDA(cudaEventCreate(&e0));
    EMIN_CUDA(cudaEventCreate(&e1));
    constexpr int wpb = kIluBlock / 32;
    for (int l = 0; l < (int)il_.size(); ++l) {
      int& slot = (*ilgrid_)[(size_t)l * 6 + ks];
      if (slot > 0) continue;
      const IluLevel& I = il_[l];
      // input: the level's residual scratch, zeroed (a cycle writes r before reading it; b
      // may already hold the caller's vector, since tuning runs inside the first cycle)
      cudaMemsetAsync(buf_[l].r, 0, sizeof(T) * (size_t)I.view.n * K, s);
      int best = I.blocks, last = -1;
      float best_ms = 1e30f;
      for (int f = 1; f <= 16; f *= 2) {
        const long long warps = std::min<long long>(std::max<long long>(f * I.per_level, 32), 32LL * sms_);
        const int blocks = (int)((warps + wpb - 1) / wpb);
        if (blocks == last) continue;
        last = blocks;
        float total = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
          cudaEventRecord(e0, s);
          ilu_substitutions<K>(l, buf_[l].r, true, blocks, false, s);
          launches_ += 2;
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) total += ms;
        }
        if (cudaGetLastError() == cudaSuccess && total < best_ms) {
          best_ms = total;
          best = blocks;
        }
      }
      slot = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }

  // One color of a level's Vanka blocks in one of three forms (0 pairs, 1 warp rows
  // with 256 threads, 2 warp rows with 1024 threads).
  template <int K>
  void vanka_color(int l, int c, int form, cudaStream_t s) {
    const VankaLevel& V = vk_[l];
    const Buf& B = buf_[l];
    const int nb = V.coff[c + 1] - V.coff[c];
    const size_t smem = ((size_t)V.max_block * sizeof(int) + 15) / 16 * 16 + (size_t)V.max_block * K * sizeof(T);
    if (form == 1 || form == 2) {
      auto kern = form == 1 ? k_vanka_color<T, K, 256> : k_vanka_color<T, K, 1024>;
      if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<nb, form == 1 ? 256 : 1024, smem, s>>>(views_[l], V.view, V.coff[c], B.b, B.x, vk_omega_);
    } else {
      auto kern = k_vanka_color_pairs<T, K>;
      if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<nb, 128, smem, s>>>(views_[l], V.view, V.coff[c], B.b, B.x, vk_omega_);
    }
  }
  // Vanka autotuner: each form timed on a whole step of each level (CUDA events),
  // the fastest kept in a table shared with the clones.
  template <int K>
  void tune_vanka(cudaStream_t s) {
    if (!(vanka_omega_ > T(0)) && !coarse_vanka_) return;
    const int ks = kslot(K);
    cudaEvent_t e0, e1;
    EMIN_CUDA(cudaEventCreate(&e0));
    EMIN_CUDA(cudaEventCreate(&e1));
    for (int l = 0; l < (int)vk_.size(); ++l) {
      int& slot = (*vkform_)[(size_t)l * 6 + ks];
      if (slot >= 0 || vk_[l].coff.empty()) continue;  // tuned, or a level without Vanka blocks
      int best = 0;
      float best_ms = 1e30f;
      for (int form = 0; form < 3; ++form) {
        float total = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
          cudaEventRecord(e0, s);
          for (size_t c = 0; c + 1 < vk_[l].coff.size(); ++c)
            if (vk_[l].coff[c + 1] > vk_[l].coff[c]) {
              vanka_color<K>(l, (int)c, form, s);
              ++launches_;
            }
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) total += ms;
        }
        if (cudaGetLastError() == cudaSuccess && total < best_ms) {
          best_ms = total;
          best = form;
        }
      }
      slot = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }

  template <int K>
  void smooth(int l, int sweeps, bool from_zero, cudaStream_t s) {
    const LevelView<T>& L = views_[l];
    const Buf& B = buf_[l];
    if (vanka_omega_ > T(0)) {
      for (int sw = 0; sw < sweeps; ++sw) vanka_sweep<K>(l, from_zero && sw == 0, s);
      return;
    }
    if (ilu_) {
      for (int sw = 0; sw < sweeps; ++sw) ilu_sweep<K>(l, from_zero && sw == 0, s);
      return;
    }
    for (int sw = 0; sw < sweeps; ++sw) {
      const int zero = (from_zero && sw == 0) ? 1 : 0;
      mark_begin(l, kVelocity, s);
      launch_rows<K>(kVelocity, l, shape(l, K, kVelocity), zero, s);
      mark_end(s);
      mark_begin(l, kSchurRhs, s);
      launch_rows<K>(kSchurRhs, l, shape(l, K, kSchurRhs), zero, s);
      mark_end(s);
      // the sweeps start from dp = 0; the dense map writes every entry of dp itself
      if (!(gsM_[l] && (*tune_)[(size_t)l * 6 + kslot(K)].kind == kGsDense))
        cudaMemsetAsync(B.dp, 0, sizeof(T) * (size_t)L.n_p * K, s);
      mark_begin(l, kGsColor, s);
      launch_gs<K>(l, s);
      mark_end(s);
      mark_begin(l, kUpdate, s);
      launch_rows<K>(kUpdate, l, shape(l, K, kUpdate), zero, s);
      mark_end(s);
    }
  }

  // Row-mapping autotuner: each sparse kernel of each level timed in every shape
  // (CUDA events, stream s, on the level's own buffers) and the fastest kept;
  // shared with the clones like the Gauss-Seidel table.
  template <int K>
  void tune_rows(cudaStream_t s) {
    const int ks = kslot(K);
    cudaEvent_t e0, e1;
    EMIN_CUDA(cudaEventCreate(&e0));
    EMIN_CUDA(cudaEventCreate(&e1));
    const int classes[] = {kVelocity, kSchurRhs, kUpdate, kResidual, kRestrict, kProlong};
    const bool vanka = vanka_omega_ > T(0);
    for (int l = 0; l + 1 < (int)views_.size(); ++l)
      for (int cls : classes) {
        if ((vanka || ilu_) && (cls == kVelocity || cls == kSchurRhs || cls == kUpdate)) continue;  // not in this cycle
        int& slot = (*rowmap_)[((size_t)l * 6 + ks) * kRowClasses + cls];
        if (slot >= 0) continue;
        int best = -1;
        float best_ms = 1e30f;
        for (int shp = 0; shp < kRowShapes; ++shp) {
          float total = 0.f;
          for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            launch_rows<K>(cls, l, shp, 0, s);
            cudaEventRecord(e1, s);
            ++launches_;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) total += ms;
          }
          if (cudaGetLastError() == cudaSuccess && total < best_ms) {
            best_ms = total;
            best = shp;
          }
        }
        slot = best;
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }

  struct Rec {
    int level, cls;
    cudaEvent_t a, b;
  };
  static constexpr const char* kClassRange[kNumClasses] = {
      "velocity predictor", "Schur right-hand side", "Gauss-Seidel", "update", "residual",
      "restriction", "prolongation", "coarsest solve", "Vanka step", "ILU(1) substitution"};
  // every launch of the cycle is bracketed by mark_begin / mark_end: an NVTX range
  // "L<level> <class>" (host side, so visible when the cycle is captured or profiled)
  // and, when profiling, a CUDA event pair
  void mark_begin(int level, int cls, cudaStream_t s) {
    ++enq_kernels_;
    {
      char name[64];
      std::snprintf(name, sizeof(name), "L%d %s", level, kClassRange[cls]);
      trace_push(name);
    }
    if (!prof_on_) return;
    Rec r{level, cls, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecord(r.a, s);
    recs_.push_back(r);
  }
  void mark_extra(cudaStream_t) { ++enq_kernels_; }
  void mark_end(cudaStream_t s) {
    if (prof_on_) cudaEventRecord(recs_.back().b, s);
    trace_pop();
  }

  // Small levels are latency-bound: their sparse kernels put G > 1 lanes on a row.
  bool small_level(int l, int K) const {
    const LevelView<T>& L = views_[l];
    return (long long)(L.n_v + L.n_p) * K < kSmallLevelItems;
  }

  // Shared memory of the strip kernel for K right-hand sides at a staging level.
  size_t gs_smem(int l, int K, int stage) const {
    const GsStrips& P = gs_[l];
    if (stage == 0) return 0;
    size_t b = (size_t)4 * P.T * K * sizeof(T) + (size_t)P.T * sizeof(T) + (size_t)(2 * P.T + 1) * sizeof(int);
    if (stage == 2) b += (size_t)P.max_strip_nnz * (sizeof(T) + sizeof(int)) + 32;  // + alignment of packed entries
    return (b + 15) / 16 * 16;
  }
  int gs_stage(int l, int K) const {
    const size_t limit = 200 * 1024;
    if (gs_smem(l, K, 2) <= limit) return 2;
    if (gs_smem(l, K, 1) <= limit) return 1;
    return 0;
  }

  // Strip-ordered Gauss-Seidel: the single-block kernel for levels of at most two
  // strips, else the pipelined kernel, else (strip data too large for shared
  // memory) one launch per phase.  No kernel needs its blocks co-resident.
  template <int K>
  void launch_gs(int l, cudaStream_t s) {
    const GsChoice c = (*tune_)[(size_t)l * 6 + kslot(K)];
    if (c.kind >= 0 && launch_gs_as<K>(l, c, s)) return;
    if (launch_gs_level<K>(l, s)) return;
    if (launch_gs_pipe<K>(l, s)) return;
    launch_gs_fallback<K>(l, s);
  }
  template <int K>
  void launch_gs_fallback(int l, cudaStream_t s) {
    if (K <= 8 && gs_lanes_[l] == 4) return launch_gs_g<K, (K <= 8 ? 4 : 1)>(l, s);
    launch_gs_g<K, 1>(l, s);
  }
  template <int K>
  bool launch_gs_as(int l, const GsChoice& c, cudaStream_t s) {
    switch (c.kind) {
      case kGsSingle: return launch_gs_level<K>(l, s, true);
      case kGsCluster: return launch_gs_cluster<K>(l, s, c.C);
      case kGsPipe: return launch_gs_pipe<K>(l, s, c.C);
      case kGsPhases: launch_gs_fallback<K>(l, s); return true;
      case kGsDense:
        if (!gsM_[l]) return false;
        if constexpr (K <= 16)
          k_gs_dense_tile<T, K><<<(views_[l].n_p + kDenseRows - 1) / kDenseRows, kDenseWarps * 32, 0, s>>>(
              views_[l].n_p, gs_ld(views_[l].n_p), gsM_[l], buf_[l].g, buf_[l].dp);
        else
          k_gs_dense<T, K><<<grid_for((long long)views_[l].n_p * 32), kBlock, 0, s>>>(
              views_[l].n_p, gs_ld(views_[l].n_p), gsM_[l], buf_[l].g, buf_[l].dp);
        return true;
    }
    return false;
  }

  // Gauss-Seidel autotuner: for each level, time every variant that applies to K
  // right-hand sides (one block, a cluster of C blocks, the pipelined kernel, one
  // launch per phase) with CUDA events on stream s and keep the fastest.  The
  // variants relax the same rows in the same order but sum a row in different
  // orders, so the table is shared with every clone of the cycle: all of them
  // round alike.  Runs outside graph capture, before the first capture for K.
  template <int K>
  void tune_gs(cudaStream_t s) {
    if (vanka_omega_ > T(0) || ilu_) return;  // no Gauss-Seidel in a Vanka or ILU cycle
    const int ks = kslot(K);
    cudaEvent_t e0, e1;
    EMIN_CUDA(cudaEventCreate(&e0));
    EMIN_CUDA(cudaEventCreate(&e1));
    for (int l = 0; l < (int)views_.size(); ++l) {
      GsChoice& slot = (*tune_)[(size_t)l * 6 + ks];
      if (slot.kind >= 0) continue;
      std::vector<GsChoice> cands;
      if (level_smem(l, K) <= 220 * 1024) cands.push_back({kGsSingle, 1, 0.f});
      for (const ClusterPlan& P : cplans_[l])
        if (cluster_smem(P, K, gs_[l].ncol) <= 220 * 1024) cands.push_back({kGsCluster, P.C, 0.f});
      if (gs_stage(l, K) > 0 && gs_[l].ncol <= kMaxColors)
        for (int v = 0; v < 4; ++v) cands.push_back({kGsPipe, v, 0.f});
      cands.push_back({kGsPhases, 0, 0.f});
      if (gsM_[l]) cands.push_back({kGsDense, 0, 0.f});
      GsChoice best{kGsPhases, 0, 1e30f};
      for (GsChoice c : cands) {
        float total = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 4 && ok; ++rep) {
          cudaMemsetAsync(buf_[l].dp, 0, sizeof(T) * (size_t)views_[l].n_p * K, s);
          cudaEventRecord(e0, s);
          ok = launch_gs_as<K>(l, c, s);
          cudaEventRecord(e1, s);
          if (ok) ++launches_;
          if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) total += ms;  // the first run warms caches and loads the kernel
        }
        cudaGetLastError();
        if (ok && total / 3.f < best.ms) best = {c.kind, c.C, total / 3.f};
      }
      slot = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int err = 0;
    cudaMemcpy(&err, err_, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) throw std::runtime_error("cuda: a Gauss-Seidel wait timed out while tuning");
  }
  void tune_for(int K, cudaStream_t s) {
    switch (K) {
      case 1: tune_rows<1>(s); tune_gs<1>(s); tune_vanka<1>(s); tune_ilu<1>(s); break;
      case 2: tune_rows<2>(s); tune_gs<2>(s); tune_vanka<2>(s); tune_ilu<2>(s); break;
      case 4: tune_rows<4>(s); tune_gs<4>(s); tune_vanka<4>(s); tune_ilu<4>(s); break;
      case 8: tune_rows<8>(s); tune_gs<8>(s); tune_vanka<8>(s); tune_ilu<8>(s); break;
      case 16: tune_rows<16>(s); tune_gs<16>(s); tune_vanka<16>(s); tune_ilu<16>(s); break;
      case 32: tune_rows<32>(s); tune_gs<32>(s); tune_vanka<32>(s); tune_ilu<32>(s); break;
    }
  }

  // Levels of at most two strips whose Schur data fits in one block's shared
  // memory run in a single block: no waits between blocks.
  size_t level_smem(int l, int K) const {
    const LevelView<T>& L = views_[l];
    const size_t nnz = (size_t)s_nnz_[l];
    return ((size_t)2 * L.n_p * K + L.n_p + nnz) * sizeof(T) +
           ((size_t)3 * L.n_p + 1 + nnz + 2 * gs_[l].ncol + 1) * sizeof(int) + 16;
  }
  template <int K>
  bool launch_gs_level(int l, cudaStream_t s, bool any_strips = false) {
    const GsStrips& P = gs_[l];
    if ((P.nstrips > 2 && !any_strips) || level_smem(l, K) > 220 * 1024) return false;
    const double rows_per_group = (double)views_[l].n_p / std::max(1, 2 * P.ncol);
    int G = 1;
    while (G < 4 && K * G * 2 <= 32 && rows_per_group * K * G * 2 <= kGsBlock) G *= 2;
    if (G == 4) return launch_gs_level_g<K, (K <= 8 ? 4 : 1)>(l, s);
    if (G == 2) return launch_gs_level_g<K, (K <= 16 ? 2 : 1)>(l, s);
    return launch_gs_level_g<K, 1>(l, s);
  }
  template <int K, int G>
  bool launch_gs_level_g(int l, cudaStream_t s) {
    const size_t smem = level_smem(l, K);
    auto kern = k_gs_level<T, K, G>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 48 * 1024));
    kern<<<1, kGsBlock, smem, s>>>(views_[l], (const T*)buf_[l].g, buf_[l].dp, (const int*)plist_[l],
                                   (const int*)poff_[l], gs_[l].ncol, gs_iters_);
    return true;
  }

  // A thread-block cluster holding the whole level: the smallest cluster whose
  // blocks fit their share in shared memory and relax a (parity, color) group in
  // one pass, else the largest that fits; false if none fits or launches.
  static size_t cluster_smem(const ClusterPlan& P, int K, int ncol) {
    // dp window, g, 1/S_ii, S values | row offsets, permutation, S columns, plist, poff
    const size_t b = ((size_t)P.win_max * K + (size_t)P.rows_max * K + P.rows_max + P.nnz_max) * sizeof(T) +
                     ((size_t)3 * P.rows_max + 1 + P.nnz_max + 2 * ncol + 1) * sizeof(int);
    return (b + 15) / 16 * 16;
  }
  template <int K>
  bool launch_gs_cluster(int l, cudaStream_t s, int C) {
    const GsStrips& S0 = gs_[l];
    const ClusterPlan* pick = nullptr;
    for (const ClusterPlan& P : cplans_[l])
      if (P.C == C && cluster_smem(P, K, S0.ncol) <= 220 * 1024) pick = &P;
    if (!pick) return false;
    const double rows_per_group = (double)pick->rows_max / (2.0 * std::max(1, S0.ncol));
    int G = 1;
    while (G < 4 && K * G * 2 <= 32 && rows_per_group * K * G * 2 <= kGsBlock) G *= 2;
    if (G == 4) return launch_gs_cluster_g<K, (K <= 8 ? 4 : 1)>(l, *pick, s);
    if (G == 2) return launch_gs_cluster_g<K, (K <= 16 ? 2 : 1)>(l, *pick, s);
    return launch_gs_cluster_g<K, 1>(l, *pick, s);
  }
  template <int K, int G>
  bool launch_gs_cluster_g(int l, const ClusterPlan& P, cudaStream_t s) {
    const size_t smem = cluster_smem(P, K, gs_[l].ncol);
    auto kern = k_gs_cluster<T, K, G>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 48 * 1024));
    if (P.C > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    GsCluster Q{};
    Q.soff = gs_[l].soff;
    Q.plist = P.plist;
    Q.poff = P.poff;
    Q.nstrips = gs_[l].nstrips;
    Q.ncol = gs_[l].ncol;
    Q.T = gs_[l].T;
    Q.iters = gs_iters_;
    Q.spc = P.spc;
    Q.win_max = P.win_max;
    Q.rows_max = P.rows_max;
    Q.nnz_max = P.nnz_max;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.C);
    cfg.blockDim = dim3(kGsBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      return false;
    }
    return cudaLaunchKernelEx(&cfg, kern, views_[l], (const T*)buf_[l].g, buf_[l].dp, Q) == cudaSuccess;
  }

  // Lanes per row for the pipelined kernel: as many as the block has to spare
  // for the average color of a strip (K * G <= 32).
  template <int K>
  bool launch_gs_pipe(int l, cudaStream_t s, int variant = 0) {
    // shapes the autotuner also tries: 1024 threads with (lanes per row, columns per thread)
    switch (variant) {
      case 1: return launch_gs_pipe_v<K, 2, 2, 1024>(l, s);
      case 2: return launch_gs_pipe_v<K, 1, 2, 1024>(l, s);
      case 3: return launch_gs_pipe_v<K, 4, 1, 1024>(l, s);
      default: break;
    }
    const GsStrips& P0 = gs_[l];
    const double rows_per_color = (double)P0.T / std::max(1, P0.ncol);
    int G = 1;
    while (G < 4 && K * G * 2 <= 32 && rows_per_color * K * G * 2 <= kGsPipeBlock) G *= 2;
    if (G == 4) return launch_gs_pipe_g<K, (K <= 8 ? 4 : 1), 1, kGsPipeBlock>(l, s);
    if (G == 2) return launch_gs_pipe_g<K, (K <= 16 ? 2 : 1), 1, kGsPipeBlock>(l, s);
    // a color too large for one pass at one column per thread: two columns per thread
    if (K >= 2 && rows_per_color * K > kGsPipeBlock)
      return launch_gs_pipe_g<K, 1, (K >= 2 ? 2 : 1), kGsPipeBlock>(l, s);
    return launch_gs_pipe_g<K, 1, 1, kGsPipeBlock>(l, s);
  }
  // (GW lanes, VW columns) clamped to what K allows: V <= K, (K / V) * G <= 32.
  template <int K, int GW, int VW, int NT>
  bool launch_gs_pipe_v(int l, cudaStream_t s) {
    constexpr int V = VW <= K ? VW : K;
    constexpr int KV = K / V;
    constexpr int G = GW * KV <= 32 ? GW : (KV >= 32 ? 1 : 32 / KV);
    return launch_gs_pipe_g<K, G, V, NT>(l, s);
  }

  template <int K, int G, int V, int NT>
  bool launch_gs_pipe_g(int l, cudaStream_t s) {
    const LevelView<T>& L = views_[l];
    const Buf& B = buf_[l];
    GsStrips P = gs_[l];
    P.stage = gs_stage(l, K);
    if (P.stage == 0 || P.ncol > kMaxColors) return false;
    const size_t smem = gs_smem(l, K, P.stage);
    auto kern = k_gs_pipe<T, K, G, V, NT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 48 * 1024));
    cudaMemsetAsync(done_[l], 0, sizeof(int) * (P.nstrips + 1), s);
    // one block per strip: as many units in flight as the pipeline can overlap
    kern<<<P.nstrips, NT, smem, s>>>(L, (const T*)B.g, B.dp, P, (const int*)ci_rel_[l], (const int2*)pk_[l],
                                     done_[l], err_);
    return true;
  }

  template <int K, int G>
  void launch_gs_g(int l, cudaStream_t s) {
    const LevelView<T>& L = views_[l];
    const Buf& B = buf_[l];
    GsStrips P = gs_[l];
    P.stage = gs_stage(l, K);
    const size_t smem = gs_smem(l, K, P.stage);
    auto kern = k_gs_strips<T, K, G>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 48 * 1024));
    const int nb = std::max(1, (P.nstrips + 1) / 2);
    if (nb == 1) {
      kern<<<1, kGsBlock, smem, s>>>(L, B.g, B.dp, P, 0, 2 * P.iters);
      return;
    }
    for (int ph = 0; ph < 2 * P.iters; ++ph) {
      if (ph) mark_extra(s);
      kern<<<nb, kGsBlock, smem, s>>>(L, B.g, B.dp, P, ph, ph + 1);
    }
  }

 public:
  // Nonzero when a bounded wait gave up (checked by the solver after a cycle).
  int* error_flag() const override { return err_; }
  cudaError_t set_wait_limit(unsigned long long polls) override {
    return cudaMemcpy(err_ + 2, &polls, sizeof(polls), cudaMemcpyHostToDevice);
  }

  cudaError_t apply_ff(const float* z, double* out, int K, cudaStream_t s) override {
    if (!ff_.A.hi) return cudaErrorInvalidValue;
    switch (K) {
      case 1: return launch_ff<1>(z, out, s);
      case 2: return launch_ff<2>(z, out, s);
      case 4: return launch_ff<4>(z, out, s);
      case 8: return launch_ff<8>(z, out, s);
      case 16: return launch_ff<16>(z, out, s);
      case 32: return launch_ff<32>(z, out, s);
    }
    return cudaErrorInvalidValue;
  }

 private:
  template <int K>
  cudaError_t launch_ff(const float* z, double* out, cudaStream_t s) {
    constexpr int V = VecWidth<float, K>::V;
    constexpr int G4 = (K / V) * 4 <= 32 ? 4 : 1;
    const long long rows = (long long)ff_.n_v + ff_.n_p;
    if (rows * K < (1LL << 16))  // small problem: 4 lanes per row
      k_block_spmv_ff<K, G4, V><<<grid_for(rows * (K / V) * G4), kBlock, 0, s>>>(ff_, z, out);
    else
      k_block_spmv_ff<K, 1, V><<<grid_for(rows * (K / V)), kBlock, 0, s>>>(ff_, z, out);
    ++launches_;
    return cudaGetLastError();
  }

  FFMat upload_ff(const Csr& M) {
    std::vector<int> rp(M.rowptr.begin(), M.rowptr.end());
    std::vector<float> hi(M.val.size()), lo(M.val.size());
    for (size_t t = 0; t < M.val.size(); ++t) {
      hi[t] = (float)M.val[t];
      lo[t] = (float)(M.val[t] - (double)hi[t]);
    }
    FFMat f;
    f.rp = alloc_copy<int>(rp);
    f.ci = alloc_copy<int>(M.col);
    f.hi = alloc_copy<float>(hi);
    f.lo = alloc_copy<float>(lo);
    return f;
  }
  void build_ff(const HostLevel& H) {
    ff_.dim = H.dim;
    ff_.n_v = H.n_v;
    ff_.n_p = H.n_p;
    ff_.pinned = H.pinned;
    ff_.A = upload_ff(H.A);
    ff_.B = upload_ff(H.B);
    ff_.Bt = upload_ff(H.Bt);
  }

  cudaError_t capture(int K, int slot) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    TraceRange range("V-cycle: autotune and graph capture, K = %d", K);
    try {
      if (autotune_) tune_for(K, cs);
    } catch (const std::exception&) {
      cudaStreamDestroy(cs);
      return cudaErrorLaunchFailure;
    }
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
    if (e != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it for the next launch checks
      throw std::runtime_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
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

  struct CloneTag {};
  DeviceVCycle(const DeviceVCycle& o, int kmax, CloneTag)
      : c_(o.c_), cfac_(o.cfac_), gs_iters_(o.gs_iters_), pre_(o.pre_), post_(o.post_), kmax_(kmax),
        vanka_omega_(o.vanka_omega_), ilu_(o.ilu_), coarse_vanka_(o.coarse_vanka_), vk_omega_(o.vk_omega_) {
    try {
      if ((long long)((size_t)o.views_[0].dim * o.views_[0].n_v + o.views_[0].n_p) * kmax_ >= (1LL << 31))
        throw std::runtime_error("N * max_nrhs must stay below 2^31 (32-bit vector indices)");
      views_ = o.views_;
      gs_ = o.gs_;
      gs_lanes_ = o.gs_lanes_;
      ci_rel_ = o.ci_rel_;
      pk_ = o.pk_;
      cplans_ = o.cplans_;
      vk_ = o.vk_;
      il_ = o.il_;
      gsM_ = o.gsM_;
      tune_ = o.tune_;
      rowmap_ = o.rowmap_;
      vkform_ = o.vkform_;
      ilgrid_ = o.ilgrid_;
      sms_ = o.sms_;
      autotune_ = o.autotune_;
      plist_ = o.plist_;
      poff_ = o.poff_;
      s_nnz_ = o.s_nnz_;
      ff_ = o.ff_;
      pinv_ = o.pinv_;
      Nc_ = o.Nc_;
      for (size_t l = 0; l < views_.size(); ++l) {
        buf_.push_back(alloc_bufs(views_[l], l + 1 < views_.size()));
        done_.push_back(alloc<int>(gs_[l].nstrips + 1));
      }
      err_ = alloc<int>(4);
      EMIN_CUDA(cudaMemset(err_, 0, 4 * sizeof(int)));
      EMIN_CUDA(set_wait_limit(kSpinLimit));
      if (ilu_) {
        il_ticket_ = alloc<int>(1);
        EMIN_CUDA(cudaMemset(il_ticket_, 0, sizeof(int)));
      }
    } catch (...) {
      release();
      throw;
    }
  }

  Buf alloc_bufs(const LevelView<T>& L, bool smoothed) {
    const size_t N = ((size_t)L.dim * L.n_v + L.n_p) * kmax_;
    Buf B;
    B.b = alloc<T>(N);
    B.x = alloc<T>(N);
    B.r = alloc<T>(N);
    B.y = alloc<T>((size_t)L.dim * L.n_v * kmax_);
    B.g = alloc<T>((size_t)L.n_p * kmax_);
    B.dp = alloc<T>((size_t)L.n_p * kmax_);
    if (ilu_ && smoothed) B.iy = alloc<T>(2 * N);
    return B;
  }

  // Cluster plans for C = 2, 4, 8, 16 blocks (levels of more than two strips).
  std::vector<ClusterPlan> cluster_plans(int n_p, int Tst, int ncol, int nstrips, const std::vector<int>& soff,
                                         const Csr& So) {
    std::vector<ClusterPlan> plans;
    if (nstrips <= 2) return plans;
    const int stride = ncol + 1;
    for (int C = 2; C <= 16; C *= 2) {
      if (C > nstrips) break;
      ClusterPlan P;
      P.C = C;
      P.spc = (nstrips + C - 1) / C;
      std::vector<int> plist(n_p), poff((size_t)C * (2 * ncol + 1), 0);
      for (int c = 0; c < C; ++c) {
        const int s0 = std::min(c * P.spc, nstrips), s1 = std::min(s0 + P.spc, nstrips);
        if (s1 <= s0) continue;
        const int q0 = soff[(size_t)s0 * stride], q1 = soff[(size_t)(s1 - 1) * stride + ncol];
        const int r_lo = std::min(s0 * Tst, n_p), r_hi = std::min(s1 * Tst, n_p);
        int pos = q0;
        int* po = poff.data() + (size_t)c * (2 * ncol + 1);
        for (int par = 0; par < 2; ++par)
          for (int pc = 0; pc < ncol; ++pc) {
            po[par * ncol + pc] = pos - q0;
            for (int st = s0; st < s1; ++st)
              if ((st & 1) == par)
                for (int r = soff[(size_t)st * stride + pc]; r < soff[(size_t)st * stride + pc + 1]; ++r) plist[pos++] = r;
          }
        po[2 * ncol] = pos - q0;
        P.rows_max = std::max(P.rows_max, q1 - q0);
        P.win_max = std::max(P.win_max, std::min(n_p, r_hi + Tst) - std::max(0, r_lo - Tst));
        P.nnz_max = std::max(P.nnz_max, (int)(So.rowptr[q1] - So.rowptr[q0]));
      }
      P.plist = alloc_copy<int>(plist);
      P.poff = alloc_copy<int>(poff);
      plans.push_back(P);
    }
    return plans;
  }

  void upload_vanka(const HostLevel& H, size_t level) {
    if (H.vk_ptr.empty()) throw std::runtime_error("the hierarchy was built without the Vanka blocks");
    const int nb = (int)H.vk_ptr.size() - 1;
    VankaLevel V;
    std::vector<int> order(nb);
    V.coff.assign(H.vk_ncolors + 1, 0);
    for (int b = 0; b < nb; ++b) ++V.coff[H.vk_colors[b] + 1];
    for (int c = 0; c < H.vk_ncolors; ++c) V.coff[c + 1] += V.coff[c];
    {
      std::vector<int> pos(V.coff.begin(), V.coff.end() - 1);
      for (int b = 0; b < nb; ++b) order[pos[H.vk_colors[b]]++] = b;  // index order within a color
    }
    for (int b = 0; b < nb; ++b) V.max_block = std::max(V.max_block, H.vk_ptr[b + 1] - H.vk_ptr[b]);
    std::vector<long long> off(H.vk_inv_off.begin(), H.vk_inv_off.end());
    V.view.ptr = alloc_copy<int>(H.vk_ptr);
    V.view.dofs = alloc_copy<int>(H.vk_dofs);
    V.view.inv = alloc_copy<T>(H.vk_inv);
    V.view.inv_off = alloc_copy<long long>(off);
    V.view.order = alloc_copy<int>(order);
    V.dirichlet = alloc_copy<int>(H.vk_dirichlet);
    V.n_dirichlet = (int)H.vk_dirichlet.size();
    vk_[level] = V;
  }

  // ILU(1) factors of a level.  Grid: about four warps per row of an average
  // dependency level (rows of a level run concurrently, the next levels' warps wait
  // behind them), at least 32 warps and at most 16 per SM.
  void upload_ilu(const HostLevel& H) {
    if (H.il_perm.empty()) throw std::runtime_error("the hierarchy was built without the ILU(1) factors");
    const int n = H.N();
    IluLevel I;
    I.view.n = n;
    I.view.perm = alloc_copy<int>(H.il_perm);
    I.view.L = upload(H.il_L);
    I.view.U = upload(H.il_U);
    std::vector<double> dinv(n);
    for (int i = 0; i < n; ++i) dinv[i] = 1.0 / H.il_diag[i];
    I.view.dinv = alloc_copy<T>(dinv);
    I.view.schedL = alloc_copy<int>(H.il_schedL);
    I.view.schedU = alloc_copy<int>(H.il_schedU);
    I.depthL = H.il_depthL;
    I.depthU = H.il_depthU;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long per_level = (n + std::max(1, std::min(I.depthL, I.depthU)) - 1) / std::max(1, std::min(I.depthL, I.depthU));
    sms_ = std::max(1, sms);
    I.per_level = per_level;
    const long long warps = std::min<long long>(std::max<long long>(4 * per_level, 32), 16LL * sms_);
    constexpr int wpb = kIluBlock / 32;
    I.blocks = (int)((warps + wpb - 1) / wpb);
    il_.push_back(I);
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
    // Schur complement rows sorted by (strip, color, index), diagonal split off;
    // soff[s * (ncol + 1) + c] is the first sorted row of color c in strip s.
    const int Tst = H.gs_strip, ncol = H.n_colors;
    const int nstrips = std::max(1, (H.n_p + Tst - 1) / Tst);
    std::vector<int> perm(H.n_p), soff((size_t)nstrips * (ncol + 1), 0);
    {
      std::vector<int> cnt((size_t)nstrips * ncol, 0);
      for (int i = 0; i < H.n_p; ++i) cnt[(size_t)(i / Tst) * ncol + H.colors[i]]++;
      std::vector<int> start((size_t)nstrips * ncol, 0);
      int run = 0;
      for (int st = 0; st < nstrips; ++st) {
        for (int c = 0; c < ncol; ++c) {
          soff[(size_t)st * (ncol + 1) + c] = run;
          start[(size_t)st * ncol + c] = run;
          run += cnt[(size_t)st * ncol + c];
        }
        soff[(size_t)st * (ncol + 1) + ncol] = run;
      }
      for (int i = 0; i < H.n_p; ++i) perm[start[(size_t)(i / Tst) * ncol + H.colors[i]]++] = i;
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
    GsStrips gp{};
    gp.nstrips = nstrips;
    gp.ncol = ncol;
    gp.T = Tst;
    gp.iters = gs_iters_;
    gp.max_strip_nnz = 0;
    for (int st = 0; st < nstrips; ++st)
      gp.max_strip_nnz = std::max<int>(gp.max_strip_nnz, (int)(So.rowptr[soff[(size_t)st * (ncol + 1) + ncol]] -
                                                                So.rowptr[soff[(size_t)st * (ncol + 1)]]));
    L.S = upload(So);
    L.S_perm = alloc_copy<int>(perm);
    L.S_dinv = alloc_copy<T>(dinv);
    gp.soff = alloc_copy<int>(soff);
    // S columns relative to the halo start of the row's strip (for the pipelined kernel)
    {
      std::vector<int> rel(So.col.size());
      for (int st = 0; st < nstrips; ++st) {
        const int h0 = std::max(0, st * Tst - Tst);
        for (int r = soff[(size_t)st * (ncol + 1)]; r < soff[(size_t)st * (ncol + 1) + ncol]; ++r)
          for (int64_t t = So.rowptr[r]; t < So.rowptr[r + 1]; ++t) rel[t] = So.col[t] - h0;
      }
      ci_rel_.push_back(alloc_copy<int>(rel));
      if (sizeof(T) == 4) {  // (relative column, FP32 value bits) per entry for the pipelined kernel
        std::vector<int2> pk(So.col.size());
        for (size_t t = 0; t < pk.size(); ++t) {
          const float v = (float)So.val[t];
          int bits;
          std::memcpy(&bits, &v, sizeof(bits));
          pk[t] = make_int2(rel[t], bits);
        }
        pk_.push_back(alloc_copy<int2>(pk));
      } else {
        pk_.push_back(nullptr);
      }
      done_.push_back(alloc<int>(nstrips + 1));
      // rows of each (strip parity, color) group, for the single-block kernel
      std::vector<int> plist, poff(1, 0);
      for (int par = 0; par < 2; ++par)
        for (int c = 0; c < ncol; ++c) {
          for (int st = par; st < nstrips; st += 2)
            for (int r = soff[(size_t)st * (ncol + 1) + c]; r < soff[(size_t)st * (ncol + 1) + c + 1]; ++r)
              plist.push_back(r);
          poff.push_back((int)plist.size());
        }
      plist_.push_back(alloc_copy<int>(plist));
      poff_.push_back(alloc_copy<int>(poff));
      cplans_.push_back(cluster_plans(H.n_p, Tst, ncol, nstrips, soff, So));
      if (H.gs_dense.empty()) {
        gsM_.push_back(nullptr);
      } else {  // rows padded with zeros to gs_ld (aligned 16-byte reads)
        const size_t ld = gs_ld(H.n_p);
        std::vector<double> padded((size_t)H.n_p * ld, 0.0);
        for (int i = 0; i < H.n_p; ++i)
          std::copy(H.gs_dense.begin() + (size_t)i * H.n_p, H.gs_dense.begin() + (size_t)(i + 1) * H.n_p,
                    padded.begin() + (size_t)i * ld);
        gsM_.push_back(alloc_copy<T>(padded));
      }
    }
    // lanes per Schur row: 4 when rows are long enough to share
    const double avg = H.n_p ? (double)So.nnz() / H.n_p : 0.0;
    gs_lanes_.push_back(avg > 16.0 ? 4 : 1);
    gs_.push_back(gp);
    s_nnz_.push_back((long long)So.nnz());
    std::vector<double> w(H.n_v);
    for (int i = 0; i < H.n_v; ++i) w[i] = H.dirichlet[i] ? 1.0 : 1.0 / (c_ * H.D[i]);
    L.w = alloc_copy<T>(w);
    if (!coarsest) {
      L.P = upload(H.P);
      L.Pp = upload(H.Pp);
      L.R = upload(H.R);
      L.Rp = upload(H.Rp);
    }
    views_.push_back(L);
    buf_.push_back(alloc_bufs(L, !coarsest));
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
  T vanka_omega_ = T(0);  // > 0: the Vanka smoother replaces Braess-Sarazin
  bool ilu_ = false;      // ILU(1) replaces Braess-Sarazin
  bool coarse_vanka_ = false;  // Vanka relaxation instead of the pseudo-inverse on the coarsest level
  T vk_omega_ = T(0);          // the Vanka under-relaxation, wherever Vanka runs
  struct IluLevel {
    IluView<T> view{};
    int depthL = 0, depthU = 0, blocks = 1;  // blocks: the untuned grid
    long long per_level = 1;                  // rows per dependency level, on average
  };
  std::vector<IluLevel> il_;  // shared (read-only) with the clones
  int sms_ = 1;
  std::shared_ptr<std::vector<int>> ilgrid_;  // [level * 6 + K slot]: tuned ILU grid (blocks), -1 untuned
  int* il_ticket_ = nullptr;  // ticket counter of the substitutions, zero between launches
  bool autotune_ = true;
  std::vector<LevelView<T>> views_;
  std::vector<Buf> buf_;
  std::vector<GsStrips> gs_;
  std::vector<int> gs_lanes_;
  std::vector<int*> ci_rel_;
  std::vector<int2*> pk_;  // FP32: S entries as (ci_rel, value bits); nullptr in FP64
  std::vector<int*> done_;
  std::vector<int*> plist_, poff_;
  std::vector<std::vector<ClusterPlan>> cplans_;
  // Vanka data per smoothed level (device copies of HostLevel's vk_*)
  struct VankaLevel {
    VankaView<T> view{};
    std::vector<int> coff;  // host: first position in view.order of each color, ncolors + 1
    const int* dirichlet = nullptr;
    int n_dirichlet = 0, max_block = 0;
  };
  std::vector<VankaLevel> vk_;  // one per level; empty (no blocks) where Vanka does not run
  std::shared_ptr<std::vector<int>> vkform_;  // [level * 6 + K slot]: Vanka kernel form, -1 untuned
  std::vector<T*> gsM_;  // dense Gauss-Seidel map of small levels (nullptr elsewhere), rows of gs_ld
  static int gs_ld(int n_p) {
    constexpr int vm = 16 / (int)sizeof(T);
    return (n_p + vm - 1) / vm * vm;
  }
  std::shared_ptr<std::vector<GsChoice>> tune_;  // [level * 6 + K slot], shared with clones
  std::shared_ptr<std::vector<int>> rowmap_;     // [(level * 6 + K slot) * classes + class], -1 untuned
  std::vector<long long> s_nnz_;
  int* err_ = nullptr;
  FFLevel ff_{};
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
// vanka_omega > 0 smooths with Vanka (the levels must carry the Vanka blocks), ilu with
// ILU(1) (the levels must carry the factors), else Braess-Sarazin; coarse_omega > 0
// relaxes the coarsest level with Vanka (it must carry the blocks) instead of the
// pseudo-inverse.
VCycleIface* make_vcycle_f64(const std::vector<HostLevel>& levels, double cfac, int gs, int pre, int post, int kmax,
                             double vanka_omega, bool ilu, double coarse_omega);
VCycleIface* make_vcycle_f32(const std::vector<HostLevel>& levels, double cfac, int gs, int pre, int post, int kmax,
                             double vanka_omega, bool ilu, double coarse_omega);
// Finest-level FP64 block product out = A x (TX = double or float), or out = b - A x.
cudaError_t apply_finest_f64(VCycleIface* v64, const void* x, bool x_fp32, const double* b, double* out, int K,
                             cudaStream_t s);

}  // namespace emin

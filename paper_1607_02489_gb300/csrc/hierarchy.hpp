// Internal to the library: the hierarchy handle behind the C ABI, the flexible
// GMRES workspace and the step-wise solve task that both the blocking solve
// (amg_fgmres_solve) and the request server (amg_server_*) drive.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/emin_amg.h"
#include "gpu_setup.hpp"
#include "setup.hpp"
#include "vcycle.cuh"

namespace emin {

// Rotated Hessenberg matrix and per-column state of K simultaneous FGMRES runs.
struct GmresState {
  double* Hm;      // (m+1) x m x K upper Hessenberg, rotated
  double* cs;      // m x K
  double* sn;      // m x K
  double* gv;      // (m+1) x K
  int* active;     // K
  int* jcount;     // K: basis vectors used in this cycle
  int* budget;     // K: iterations left for the column
  int* flags;      // K: 1 converged (recurrence), 2 breakdown
  double* resest;  // K
};

// FGMRES workspace for K interleaved right-hand sides of length N and restart m.
struct Krylov {
  long long N = 0;
  int K = 0, m = 0;
  bool f32 = false;
  size_t bytes = 0;  // device bytes held
  std::vector<void*> mem;
  double *V = nullptr, *w = nullptr, *bK = nullptr, *xK = nullptr, *rK = nullptr;
  void* Z = nullptr;  // m blocks of N x K, FP32 for an FP32 V-cycle
  double *hbuf = nullptr, *part = nullptr, *y = nullptr, *bnorm = nullptr, *rnorm = nullptr;
  GmresState st{};
  int* n_active = nullptr;
  int* reorth = nullptr;     // device flag: the current Arnoldi step needs a second pass
  int* host_i = nullptr;     // pinned, kHostInts
  double* host_d = nullptr;  // pinned, kHostDoubles
  static constexpr int kHostInts = 256, kHostDoubles = 128;

  Krylov() = default;
  Krylov(const Krylov&) = delete;
  Krylov& operator=(const Krylov&) = delete;
  ~Krylov() { release(); }
  // Allocates everything (throws std::runtime_error naming cudaMalloc on failure).
  void init(long long N, int K, int m, bool f32);
  void release();
  static size_t bytes_for(long long N, int K, int m, bool f32);
};

// One flexible GMRES solve (Section 5, right preconditioning by the V-cycle) as a
// sequence of chunks of device work.  advance() enqueues the next chunk on the
// task's stream and returns true; the caller must let that work complete (stream
// synchronisation or an event recorded after it) before calling advance() again,
// since each step reads the small results the previous chunk copied to pinned host
// memory.  advance() returns false once the solve has finished; result() then
// reports it.  Errors are thrown as std::runtime_error.
class SolveTask {
 public:
  virtual ~SolveTask() = default;
  virtual bool advance() = 0;
  virtual amg_status result(int* iters, double* relres) const = 0;
  // Status of one column: AMG_OK, AMG_NOT_CONVERGED or AMG_BREAKDOWN.
  virtual amg_status column_status(int k) const = 0;
  // The event after which the next advance() may run (its results are then on the
  // host); nullptr: all work enqueued on the task's stream.  While Arnoldi steps
  // run, the task keeps one step queued beyond the one whose results it reads next,
  // so the device does not idle while the host reads them and enqueues more.
  virtual cudaEvent_t ready() const { return nullptr; }
  long long launches = 0;  // kernels this task launched outside the V-cycle graphs
};

// A group of right-hand sides of a solve: ncols columns in the caller's layout
// (device b and x, N x ncols row-major); when b_host / x_host are given, the first
// chunk copies b_host into b and the last copies x out to x_host.
struct SolveSegment {
  const double* b = nullptr;
  double* x = nullptr;
  const double* b_host = nullptr;
  double* x_host = nullptr;
  int ncols = 0;
};

// One solve of the segments' columns side by side (column order = segment order).
// Every column runs its own FGMRES; they share the kernels of K = round_k(total
// columns) <= vc->kmax().
std::unique_ptr<SolveTask> make_solve_task(struct amg_hierarchy_core* h, VCycleIface* vc, Krylov* ws,
                                           const std::vector<SolveSegment>& segs, double rtol, int restart, int maxit,
                                           cudaStream_t s);
// The single-segment form.
std::unique_ptr<SolveTask> make_solve_task(struct amg_hierarchy_core* h, VCycleIface* vc, Krylov* ws, const double* b,
                                           double* x, const double* b_host, double* x_host, int nrhs, double rtol,
                                           int restart, int maxit, cudaStream_t s);

int round_k(int nrhs);

// The parts of a hierarchy a solve needs.
struct amg_hierarchy_core {
  std::vector<HostLevel> host;
  amg_params prm{};
  VCycleIface* v64 = nullptr;  // FP64 cycle; also holds the finest FP64 matrices for residuals
  VCycleIface* v32 = nullptr;
  long long N = 0;
  bool symmetric = true;  // Stokes (R = P^T) or Oseen (Petrov-Galerkin) problem
  // device patterns and maps of this hierarchy's structure, built by the first
  // device reuse of it and shared with the hierarchies reused from it
  mutable std::shared_ptr<DeviceSetupPlan> plan;
  VCycleIface* vc() const { return prm.vcycle_fp32 ? v32 : v64; }
};

}  // namespace emin

struct amg_hierarchy : emin::amg_hierarchy_core {
  std::unique_ptr<emin::Krylov> kry;  // workspace of the blocking solve and of amg_apply
  void* stage_b = nullptr;            // device copies for amg_fgmres_solve_host
  void* stage_x = nullptr;
  long long launches = 0;             // kernels launched outside the V-cycle graphs

  ~amg_hierarchy() {
    kry.reset();
    if (stage_b) cudaFree(stage_b);
    if (stage_x) cudaFree(stage_x);
    delete v64;
    delete v32;
  }
};

// One translation unit per V-cycle arithmetic type: compiled with
// -DEMIN_VCYCLE_DOUBLE (FP64 cycle and the FP64 finest-level product) or
// without it (FP32 cycle with FP32 accumulation).
#include "vcycle.cuh"

namespace emin {

#ifdef EMIN_VCYCLE_DOUBLE

VCycleIface* make_vcycle_f64(const std::vector<HostLevel>& levels, double cfac, int gs, int pre, int post, int kmax,
                             double vanka_omega, bool ilu, double coarse_omega) {
  return new DeviceVCycle<double>(levels, cfac, gs, pre, post, kmax, vanka_omega, ilu, coarse_omega);
}

template <int K>
static void apply_k(const LevelView<double>& L, const double* x, const double* b, double* out, cudaStream_t s) {
  constexpr int V = VecWidth<double, K>::V;
  const unsigned g = grid_for((long long)(L.n_v + L.n_p) * (K / V));
  if (b)
    k_block_spmv<double, K, 1, V, true><<<g, kBlock, 0, s>>>(L, b, x, out);
  else
    k_block_spmv<double, K, 1, V, false><<<g, kBlock, 0, s>>>(L, nullptr, x, out);
}

cudaError_t apply_finest_f64(VCycleIface* v64, const void* x, bool x_fp32, const double* b, double* out, int K,
                             cudaStream_t s) {
  if (x_fp32) return cudaErrorInvalidValue;  // FP32 vectors go through apply_ff (float-float)
  const LevelView<double>& L = static_cast<DeviceVCycle<double>*>(v64)->view(0);
  const double* xd = (const double*)x;
  switch (K) {
    case 1: apply_k<1>(L, xd, b, out, s); break;
    case 2: apply_k<2>(L, xd, b, out, s); break;
    case 4: apply_k<4>(L, xd, b, out, s); break;
    case 8: apply_k<8>(L, xd, b, out, s); break;
    case 16: apply_k<16>(L, xd, b, out, s); break;
    case 32: apply_k<32>(L, xd, b, out, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#else

VCycleIface* make_vcycle_f32(const std::vector<HostLevel>& levels, double cfac, int gs, int pre, int post, int kmax,
                             double vanka_omega, bool ilu, double coarse_omega) {
  return new DeviceVCycle<float>(levels, cfac, gs, pre, post, kmax, vanka_omega, ilu, coarse_omega);
}

#endif

}  // namespace emin

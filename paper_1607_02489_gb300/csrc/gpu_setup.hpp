// Numeric hierarchy setup on the GPU.
//
// For a matrix with the structure of an existing hierarchy's finest level (the
// next system of a Picard sequence, Section 6.1), the coarse points and every
// sparsity pattern are known, so what remains is numeric and data-parallel:
// the filtered auxiliary matrices (eq. e:filtering on B B^T and on the velocity
// block), one EMIN step per transfer (Section 4.3), the restrictions, the
// Petrov-Galerkin products R A P block by block (Alg. 1), and the Braess-Sarazin
// data D and S = B D^-1 B^T (Section 5.2).  Every product is a sparse product
// with a known output pattern, computed entry by entry as a merge of a row of
// the left factor with a column of the right one.  The dense Gauss-Seidel maps
// of small levels (the iterations' linear map, formed by running the ordered
// sweep on every unit vector) are formed on the GPU as well.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "setup.hpp"

namespace emin {

// Sparsity patterns and transpose maps a device reuse needs, built on the host
// from a hierarchy's levels once and shared by every hierarchy with the same
// structure (a Picard sequence's hierarchies).
struct DeviceSetupPlan;

// The hierarchy build_hierarchy(fine, prm with reuse = &prev) returns, with the
// numeric work done on the current device (values agree with the host build to
// rounding).  *plan is built from prev on first use and reused afterwards.  The
// smoother data that depend only on patterns (strips, colors) are prev's; the
// coarsest pseudo-inverse, Vanka blocks and ILU(1) factors are left to
// complete_hierarchy.  Throws std::runtime_error on failure.
std::vector<HostLevel> build_hierarchy_reuse_device(HostLevel fine, const std::vector<HostLevel>& prev,
                                                    const SetupParams& prm, std::shared_ptr<DeviceSetupPlan>& plan,
                                                    cudaStream_t s);

// The dense Gauss-Seidel maps (HostLevel::gs_dense) of the levels of at most
// kGsDenseMaxRows pressures, formed on the current device: the same ordered
// sweeps as the host's form_dense_gs, every column of the map at once.
void form_dense_gs_device(std::vector<HostLevel>& levels, int iters, cudaStream_t s);

}  // namespace emin

// Host-side multigrid hierarchy (Alg. 1) for Q2-Q1 saddle-point systems.
#pragma once

#include <string>
#include <vector>

#include "csr.hpp"

namespace emin {

struct SetupParams {
  double tau1 = -1.0;      // eq. e:filtering; < 0: 0.06 in 2D, 0.015 in 3D
  double tau1_for(int dim) const { return tau1 >= 0.0 ? tau1 : (dim == 2 ? 0.06 : 0.015); }
  double tau2sq = 1.5e-3;  // Alg. 4, tau2 = sqrt(1.5e-3)
  double c = 0.666;        // scale of D in the (1,1) block of the Braess-Sarazin matrix
  int max_coarse = 200;
  int max_levels = 12;
  bool symmetric = true;   // one EMIN CG step, R = P^T; otherwise EMIN GMRES for P and R
  bool vanka = false;      // form the Vanka smoother's blocks (Section 5.1) on every level but the coarsest
  bool vanka_coarse = false;  // form them on the coarsest level too (its Vanka relaxation, Section 6.1)
  bool ilu = false;        // form the ILU(1) factors (Section 5) on every level but the coarsest
  int ilu_order = 0;       // symmetric problems: 0 block order [u_x | u_y | p], 1 by node location
  int gs_iters = 5;        // Gauss-Seidel iterations per Braess-Sarazin step (for the dense map)
  bool dense_gs = true;    // form the dense Gauss-Seidel maps on the host (else the caller forms them)
  size_t vanka_max_bytes = (size_t)16 << 30;  // limit on the FP64 block inverses of one level
  // When set: take the number of levels, the coarse points and the sparsity
  // patterns of P from this hierarchy (built for a matrix of the same structure)
  // and redo only filtering, EMIN, RAP and the smoother data.
  const std::vector<struct HostLevel>* reuse = nullptr;
};

constexpr int kGsDenseMaxRows = 4608;  // dense Gauss-Seidel map: <= 81 MiB in FP32

struct HostLevel {
  int dim = 2, n_v = 0, n_p = 0, pinned = -1;
  Csr A;   // n_v x n_v scalar velocity block
  Csr B;   // n_p x dim*n_v, the (2,1) block
  Csr Bt;  // dim*n_v x n_p, the (1,2) block
  std::vector<double> vX, pX;          // coordinates, row-major
  std::vector<int> p2v;                // co-located velocity node or -1
  std::vector<unsigned char> dirichlet;
  // Braess-Sarazin data (Section 5.2)
  std::vector<double> D;               // |A| row sums; Dirichlet rows 1/c
  Csr S;                               // B D^-1 Bt, pinned row = identity
  std::vector<int> colors;             // greedy coloring of each strip's subgraph of S
  int n_colors = 0;
  int gs_strip = 1;                    // Gauss-Seidel strip length (see form_relaxation)
  // levels of at most kGsDenseMaxRows pressures: M (n_p x n_p, row-major) with dp = M g
  // for gs_iters Gauss-Seidel iterations from dp = 0 in the (strip parity, color, index) order
  std::vector<double> gs_dense;
  // Vanka data (Section 5.1): blocks (global dofs of block b in vk_dofs[vk_ptr[b]..vk_ptr[b+1]),
  // a greedy coloring of the block interaction graph, each block's local matrix
  // inverted (row-major, at vk_inv_off[b]), and the Dirichlet dofs relaxed exactly.
  std::vector<int> vk_ptr, vk_dofs, vk_colors, vk_dirichlet;
  std::vector<int64_t> vk_inv_off;
  std::vector<double> vk_inv;
  int vk_ncolors = 0;
  // ILU(1) data (Section 5): the level's block matrix in the smoother's order
  // (il_perm[position] = dof; natural for symmetric problems, reverse Cuthill-McKee
  // otherwise) factored with one level of fill: il_L its strict lower part (unit
  // diagonal implied), il_U the strict upper part, il_diag the pivots, all in
  // positions of that order.  il_schedL / il_schedU list the rows by (dependency
  // level, position) of the forward / backward substitution; il_depthL / il_depthU
  // count those levels.
  Csr il_L, il_U;
  std::vector<double> il_diag;
  std::vector<int> il_perm, il_schedL, il_schedU;
  int il_depthL = 0, il_depthU = 0;
  // transfers to the next level
  Csr P, Pp, R, Rp;
  std::vector<int> Cp, Cv;             // coarse points (fine indices, ascending)
  // coarsest level
  std::vector<double> pinv;            // N x N row-major pseudo-inverse
  int N() const { return dim * n_v + n_p; }
  long long nnz_total() const {
    return (long long)dim * A.nnz() + B.nnz() + Bt.nnz() + (pinned >= 0 ? 1 : 0);
  }
};

// Builds every level; throws std::runtime_error with a message on failure.
std::vector<HostLevel> build_hierarchy(HostLevel fine, const SetupParams& prm);

// The smoother data of levels whose operators and transfers are given: with
// `relaxation`, the Braess-Sarazin data of every level (D, S, strips, colors);
// then the coarsest pseudo-inverse and, as prm asks, the Vanka blocks, the ILU(1)
// factors and the dense Gauss-Seidel maps.  build_hierarchy ends with it; an
// imported hierarchy goes through it whole.
void complete_hierarchy(std::vector<HostLevel>& levels, const SetupParams& prm, bool relaxation);

// Checkpoint file of a hierarchy's operators and transfers (format in emin_amg.h,
// amg_hierarchy_export).  read_hierarchy checks sizes and CSR structure and throws
// std::runtime_error naming the first problem.
void write_hierarchy(const std::vector<HostLevel>& levels, bool symmetric, const std::string& path);
std::vector<HostLevel> read_hierarchy(const std::string& path, bool* symmetric);

}  // namespace emin

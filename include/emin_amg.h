/*
 * emin_amg.h — C ABI of the GB300 EMIN-AMG solver for Q2-Q1 Stokes / Oseen systems.
 *
 * Method: Prokopenko & Tuminaro, "An algebraic multigrid method for Q2-Q1
 * mixed discretizations of the Navier-Stokes equations" (arXiv 1607.02489).
 * The library builds the multigrid hierarchy of Alg. 1 on the host and applies
 * its V-cycle (Braess-Sarazin relaxation of Section 5.2, EMIN transfers of
 * Section 4) and a flexible GMRES around it with CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *   - The system is the block matrix of eq. stokes_block_system /
 *     ns_block_system, [I_d (x) A, B^T; B, C], where A is the n_v x n_v scalar
 *     velocity block shared by the d components, B is n_p x (d*n_v) with
 *     component-major columns (column c*n_v + i is component c of velocity node
 *     i) and C is zero except for an optional pinned pressure (C_kk = 1).
 *   - Dofs are ordered [u_x | u_y (| u_z) | p], N = d*n_v + n_p.
 *   - A block of nrhs vectors is stored row-major, N x nrhs: entry (dof i,
 *     right-hand side k) is at index i*nrhs + k.  With nrhs = 1 this is a plain
 *     vector.  These buffers are DEVICE pointers owned by the caller, except
 *     in amg_fgmres_solve_host.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); all GPU
 *     work of a call is enqueued on it.  Calls that return results to the host
 *     (iteration counts, residuals) synchronise that stream before returning.
 *   - Every call returns an amg_status; nothing is thrown across the ABI.
 *     amg_last_error() gives a message for the last failing call of the
 *     calling thread.
 *   - A handle is not thread safe: one call at a time per handle.
 */
#ifndef EMIN_AMG_H
#define EMIN_AMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amg_hierarchy* amg_handle;

typedef enum {
  AMG_OK = 0,
  AMG_NOT_CONVERGED = 1, /* FGMRES hit maxit; x, iters and relres are valid */
  AMG_BREAKDOWN = 2,     /* an Arnoldi vector vanished before convergence */
  AMG_ERR_ARG = -1,      /* invalid argument (null pointer, size, malformed CSR) */
  AMG_ERR_OOM = -2,      /* host or device allocation failed */
  AMG_ERR_CUDA = -3,     /* a CUDA call failed */
  AMG_ERR_SETUP = -4     /* the hierarchy could not be built */
} amg_status;

/* The problem, all HOST arrays, 0-based int32 indices, columns ascending in a
 * row, no duplicate entries.  The library copies what it needs during
 * amg_hierarchy_create; the caller may free these afterwards.
 * Section 2 (eq. stokes_block_system, ns_block_system) defines A and B; the
 * node coordinates and the pressure-to-velocity co-location are inputs of the
 * coarsening (Section 4 uses coordinates in its distance heuristics, Alg. 3;
 * Section 4.2 maps coarse pressures to co-located velocities, Alg. 4). */
typedef struct {
  int dim;                         /* 2 or 3 */
  int n_vnodes;                    /* n_v: velocity nodes per component */
  int n_pnodes;                    /* n_p: pressure nodes */
  const int* A_rowptr;             /* n_v + 1 */
  const int* A_col;                /* nnz(A) */
  const double* A_val;             /* nnz(A): the velocity block (nu*A_hat [+ K_hat]) */
  const int* B_rowptr;             /* n_p + 1 */
  const int* B_col;                /* nnz(B), in [0, dim*n_v) */
  const double* B_val;             /* nnz(B) */
  const double* vcoords;           /* n_v x dim, row-major */
  const double* pcoords;           /* n_p x dim, row-major */
  const int* p2v;                  /* n_p: velocity node co-located with each pressure node */
  const unsigned char* v_dirichlet;/* n_v: 1 = Dirichlet node (identity row/column in A, zero B column) */
  int pinned_p;                    /* pinned pressure node (identity in C, zero B row), -1 = none */
  int symmetric;                   /* 1: Stokes (R = P^T, one EMIN CG step); 0: Oseen
                                      (Petrov-Galerkin, one EMIN GMRES step for P and for R) */
} amg_problem;

/* Method parameters; amg_params_default fills the values of Section 6. */
typedef struct {
  double tau1;        /* eq. e:filtering drop tolerance; < 0 (the default) takes 0.06 in 2D
                        (Section 6) and 0.015 in 3D, the threshold that keeps every
                        nearest-neighbour coupling of the Q2 velocity block there */
  double tau2sq;      /* Alg. 4 tolerance squared, 1.5e-3 */
  double omega;       /* Braess-Sarazin relaxation, 0.666 */
  int omega_on_D;     /* 0: M = [omega D, B^T; B, 0] (eq. bs2's factorisation, default);
                         1: M = [D/omega, B^T; B, 0] (eq. bs) */
  int gs_iters;       /* Gauss-Seidel iterations on the Schur complement, 5 */
  int pre, post;      /* BS sweeps before / after the coarse correction, 2 and 2 */
  int max_coarse;     /* stop coarsening at <= this many dofs, 200 */
  int max_levels;     /* 12 */
  int vcycle_fp32;    /* 0: FP64 V-cycle; 1: FP32 V-cycle (FP32 accumulation), FP64 coarsest solve */
  int max_nrhs;       /* largest nrhs later passed to vcycle/fgmres (workspace size), 8 */
  int host_only;      /* 1: build the hierarchy on the host and upload nothing (inspection
                         calls work, solve calls return AMG_ERR_ARG); 0 (default): upload */
  int autotune;       /* 1 (default): before a cycle for K right-hand sides is first captured,
                         time each Gauss-Seidel variant that applies to each level (one block,
                         a thread-block cluster of 2-16 blocks, the pipelined kernel, one launch
                         per phase, the dense map on levels of <= 4608 pressures) and keep the
                         fastest; 0: fixed choice by level size, sweeps only */
  int smoother;       /* 0 (default): Braess-Sarazin (Section 5.2); 1: Vanka (Section 5.1):
                         overlapping blocks, one per pressure dof (the columns of its row of
                         B plus the pressure), relaxed in the order (color, index) of a
                         greedy coloring of the blocks' interaction graph, Dirichlet dofs
                         exactly; pre and post count Vanka steps (the paper's Vanka(1,1));
                         2: ILU(1) (Section 5): incomplete LU of each level's whole block
                         matrix with one level of fill, its diagonal (the zero block's too)
                         kept in the pattern; natural order for symmetric problems, reverse
                         Cuthill-McKee otherwise (Section 6.1); a zero-block pivot that no
                         elimination step reaches becomes -sum_j M_ij M_ji / M_jj over its
                         row; pre and post count ILU steps (the paper's ILU(1)(1,1)) */
  double vanka_omega; /* Vanka under-relaxation, 0.5 (Section 6) */
  int ilu_order;      /* ILU(1) order of a symmetric problem's levels: 0 (default) the dof order
                         [u_x | u_y (| u_z) | p], 1 by node location (lexicographic from the
                         lower-left corner, u_x, u_y (, u_z), p at one node); non-symmetric
                         problems always take reverse Cuthill-McKee */
  int coarse;         /* coarsest level: 0 (default) FP64 pseudo-inverse (exact minimum-norm
                         solve); 1 Vanka relaxation as in the paper (Section 6.1): pre + post
                         Vanka steps (vanka_omega) from zero, whatever the smoother; coarsening
                         then stops before a level that would keep only one pressure (the
                         constant, whose B vanishes: no Vanka step exists there), and setup
                         fails (AMG_ERR_SETUP) if a coarsest Vanka block is still numerically
                         singular (e.g. coarsening reused from a hierarchy built without it) */
  int device_setup;   /* 1 (default): the numeric setup work runs on the GPU where it can:
                         amg_hierarchy_create_reuse forms the filtered auxiliary matrices, the
                         EMIN steps, the restrictions, the Galerkin products and the
                         Braess-Sarazin data there (every pattern is the previous hierarchy's),
                         and every build forms the dense Gauss-Seidel maps there; values agree
                         with the host setup to rounding.  0: all setup on the host.  Ignored
                         with host_only. */
  double vanka_max_mib; /* limit on one level's FP64 Vanka block inverses, 16384 (16 GiB);
                           setup fails (AMG_ERR_SETUP) on a level that needs more (large
                           blocks, e.g. in 3D) */
} amg_params;

void amg_params_default(amg_params* prm);

/* Alg. 1: build the hierarchy on the host (filtering, Alg. 3, Alg. 4, one EMIN
 * step, Petrov-Galerkin products, Braess-Sarazin data, coarsest pseudo-inverse)
 * and upload it to the current CUDA device.  Synchronises `stream` once at the
 * end.  *out is set only on AMG_OK. */
amg_status amg_hierarchy_create(const amg_problem* prob, const amg_params* prm, void* stream,
                                amg_handle* out);

/* A hierarchy for a new matrix of the same structure as prev's finest level (same
 * sizes, same sparsity of A and B; AMG_ERR_ARG otherwise), e.g. the next linear
 * system of a Picard sequence: the number of levels, the coarse pressures and
 * velocities (Alg. 3-4) and the sparsity patterns of the transfers are taken from
 * prev, and filtering, the EMIN steps, restriction, the Galerkin products, the
 * smoother data and the coarsest solve are redone on the new values (Section 6.1:
 * the graph phase dominates setup, and the paper notes that one graph coarsening can
 * serve every linear system of a nonlinear solve).  prev stays valid and independent. */
amg_status amg_hierarchy_create_reuse(amg_handle prev, const amg_problem* problem, const amg_params* params,
                                      void* stream, amg_handle* out);

/* Checkpoint of a hierarchy: write the operators and transfers of every level (the
 * result of Alg. 1's coarsening, EMIN steps and Galerkin products) to a file, and
 * build a hierarchy from such a file without repeating that setup.  Import forms
 * only the smoother data (Section 5: the Braess-Sarazin diagonal, Schur complement
 * and its Gauss-Seidel order, or the Vanka blocks or ILU(1) factors, as prm asks)
 * and the coarsest pseudo-inverse, then uploads like amg_hierarchy_create.  Another
 * program can write the file (a reference implementation's hierarchy, for V-cycle
 * parity independent of the setup); an imported hierarchy also serves as the
 * `prev` of amg_hierarchy_create_reuse.
 *
 * File layout, little-endian, no padding:
 *   char[8] "EMINAMG1"; int32 version = 1; int32 levels; int32 symmetric (1 Stokes,
 *   0 Oseen); then per level l = 0 (finest) .. levels-1:
 *     int32 dim, n_v, n_p, pinned (-1 none)
 *     csr A (n_v x n_v), csr B (n_p x dim*n_v), csr Bt (dim*n_v x n_p)
 *     float64 vcoords[n_v*dim], float64 pcoords[n_p*dim], int32 p2v[n_p],
 *     uint8 dirichlet[n_v]
 *     every level but the last: csr P (n_v x n_v'), csr Pp (n_p x n_p'),
 *     csr R (n_v' x n_v), csr Rp (n_p' x n_p), int32 n_p', int32 Cp[n_p'],
 *     int32 n_v', int32 Cv[n_v'] (coarse points as fine indices; n_v', n_p' the
 *     next level's sizes)
 *   csr: int32 nrows, int32 ncols, int64 nnz, int64 rowptr[nrows+1],
 *        int32 col[nnz] (strictly ascending per row), float64 val[nnz].
 * Import checks every size and CSR structure and returns AMG_ERR_ARG naming the
 * first problem (or a file that cannot be read); export returns AMG_ERR_ARG when
 * the file cannot be written.  prm as for amg_hierarchy_create (NULL: defaults;
 * the coarsening parameters are unused).  Import synchronises `stream` once. */
amg_status amg_hierarchy_export(amg_handle h, const char* path);
amg_status amg_hierarchy_import(const char* path, const amg_params* prm, void* stream, amg_handle* out);

/* z = M^-1 r: one V(pre, post) cycle from a zero initial guess (Alg. 1's relaxation
 * form on every level, coarse correction by R and P).  r and z: device, N x nrhs,
 * FP64; 1 <= nrhs <= max_nrhs.  r and z must not overlap.  Asynchronous. */
amg_status amg_vcycle_apply(amg_handle h, const double* r, double* z, int nrhs, void* stream);

/* Block product y = A x on the finest level (device, N x nrhs, FP64). Asynchronous. */
amg_status amg_apply(amg_handle h, const double* x, double* y, int nrhs, void* stream);

/* y = A x like amg_apply, for callers that cannot allocate device memory during a
 * call: for instance a solver service whose memory budget is fully owned by
 * another allocator (such as PyTorch's caching allocator), where a surprise
 * cudaMalloc could fail, or a latency-bound loop that cannot afford the device
 * synchronisation cudaMalloc/cudaFree bring.  The paper has no counterpart:
 * this is an allocation policy of this library, not a step of the method.
 * It allocates nothing: its scratch (x and y padded to K = nrhs rounded up to a
 * power of two columns) is a 16 MiB array in the library's device memory, held
 * by every device that loads the library until the process exits.  Limit:
 * N * K <= 1,048,576 (for example 2,467 dofs with 32 right-hand sides, or
 * 592,387 dofs with one); larger sizes return AMG_ERR_ARG with a message.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (once per device, that device current); make that first
 * call before any stream capture.  Every call on a device shares the array and
 * its last contents (each call rewrites all it reads), so calls whose GPU work
 * overlaps (different streams or threads on the same device) race; order them.
 * x, y: device, N x nrhs, FP64; 1 <= nrhs <= 32.  Asynchronous. */
amg_status amg_apply_noalloc(amg_handle h, const double* x, double* y, int nrhs, void* stream);

/* Right-preconditioned flexible GMRES with the V-cycle as preconditioner
 * (Section 6 solves every system with GMRES preconditioned by the multigrid
 * cycle), FP64 Arnoldi (classical
 * Gram-Schmidt with one re-orthogonalisation) and Givens rotations on the
 * device, x0 = 0, restarted every `restart` iterations, stopped per column when
 * ||b - A x|| / ||b|| <= rtol (the recurrence residual, then checked with the
 * true residual recomputed in FP64).  b, x: device, N x nrhs.  iters and
 * relres: host arrays of nrhs (may be NULL); relres is the true relative
 * residual.  Synchronises `stream`.  Returns AMG_NOT_CONVERGED if some column
 * did not reach rtol within maxit iterations. */
amg_status amg_fgmres_solve(amg_handle h, const double* b, double* x, int nrhs, double rtol,
                            int restart, int maxit, int* iters, double* relres, void* stream);

/* The same solve with HOST b and x (N x nrhs): the host-to-device copy of b and the
 * device-to-host copy of x are part of the call. */
amg_status amg_fgmres_solve_host(amg_handle h, const double* b_host, double* x_host, int nrhs,
                                 double rtol, int restart, int maxit, int* iters, double* relres,
                                 void* stream);

/* Kernel timing: run `reps` V-cycles on the current contents of the level-0
 * input buffer without the CUDA graph, with a CUDA event pair on `stream`
 * around every kernel launch.  ms and count are caller arrays of
 * amg_num_levels(h) * AMG_NUM_KERNEL_CLASSES; entry [level * AMG_NUM_KERNEL_CLASSES + class] gets the
 * summed milliseconds and the number of launches of that class on that level.
 * Classes: 0 velocity predictor, 1 Schur right-hand side, 2 Gauss-Seidel color
 * sweep, 3 velocity/pressure update, 4 block residual, 5 restriction,
 * 6 prolongation, 7 coarsest solve, 8 Vanka step (its color launches and the exact
 * Dirichlet relaxation), 9 ILU(1) substitution (forward and backward, one launch
 * each; the step's residual counts as class 4).  Synchronises `stream`. */
#define AMG_NUM_KERNEL_CLASSES 10
amg_status amg_profile_vcycle(amg_handle h, int nrhs, int reps, double* ms, long long* count, void* stream);

/* Arnoldi timing: one classical Gram-Schmidt pass with nv basis vectors of N x nrhs on
 * the solver's own FP64 workspace (allocated as for restart = nv, then zeroed: the FP64
 * work does not depend on the values), with CUDA events on `stream`: *ms_dot gets the
 * average time of the inner-product kernel (nv products and the norm, per column) and
 * *ms_update that of the update kernel (w -= V h, with the norm), over `reps` launches
 * after one untimed.  Each does (nv + 1) N nrhs FP64 multiply-adds.  Synchronises
 * `stream`; overwrites the workspace (call it between solves). */
amg_status amg_profile_arnoldi(amg_handle h, int nrhs, int nv, int reps, double* ms_dot, double* ms_update,
                               void* stream);

/* Number of CUDA kernels this handle has launched so far (a replayed V-cycle graph
 * counts each of its kernel nodes).  Host-side counter, no synchronisation. */
long long amg_kernel_launches(amg_handle h);

/* Hierarchy inspection (host copies kept from the setup), for parity checks and
 * checkpoints.  Level 0 is the finest. */
typedef struct {
  int dim, n_v, n_p, pinned;
  long long nnz_A, nnz_B, nnz_Bt, nnz_S;
  int n_colors;
  long long nnz_P, nnz_Pp, nnz_R, nnz_Rp; /* 0 on the coarsest level */
  int n_cp, n_cv;                          /* coarse points chosen on this level (0 on the coarsest) */
  int gs_strip;                            /* Gauss-Seidel strip length T: rows are relaxed in the order
                                              (floor(row / T) mod 2, color, row) */
} amg_level_info;

int amg_num_levels(amg_handle h);
amg_status amg_level_get_info(amg_handle h, int level, amg_level_info* info);

/* Copy one matrix of a level to caller-owned host arrays sized from amg_level_info:
 * which = 0 A, 1 B, 2 Bt (the (1,2) block), 3 S (Schur complement B D^-1 Bt,
 * original row order), 4 P (velocity, one component), 5 Pp, 6 R, 7 Rp.
 * rowptr: nrows + 1 (int64), col: nnz, val: nnz. */
amg_status amg_level_get_matrix(amg_handle h, int level, int which, long long* rowptr, int* col,
                                double* val);

/* Coarse points of a level as fine indices (cp: n_cp pressure nodes, cv: n_cv
 * velocity nodes, ascending), the Gauss-Seidel colors of the pressure nodes
 * (n_p) and the Braess-Sarazin diagonal D (n_v).  Any pointer may be NULL. */
amg_status amg_level_get_points(amg_handle h, int level, int* cp, int* cv, int* colors, double* D);

/* The Vanka blocks of a level (hierarchies built with smoother = 1: every level but
 * the coarsest; with coarse = 1: the coarsest): *nblocks, *ndofs (total dofs over blocks) and *ncolors when the
 * arrays are NULL; otherwise ptr (nblocks + 1), dofs (ndofs, global dof indices)
 * and colors (nblocks) are filled.  AMG_ERR_ARG for a level without blocks. */
amg_status amg_level_get_vanka(amg_handle h, int level, int* nblocks, int* ndofs, int* ncolors, int* ptr,
                               int* dofs, int* colors);

/* The ILU(1) factors of a level (hierarchies built with smoother = 2, every level
 * but the coarsest), in positions of the smoother's order: perm[position] = dof
 * (dofs ordered [u_x | u_y (| u_z) | p]); the strict lower factor (unit diagonal
 * implied) and the strict upper factor as CSR with ascending columns (ptr has
 * n + 1 entries); pivots the diagonal of U.  depth_lower / depth_upper: the number
 * of dependency levels of the forward / backward substitution (its critical path
 * in rows).  Sizes only when the arrays are NULL; each array may be NULL.
 * AMG_ERR_ARG for a level without factors. */
amg_status amg_level_get_ilu(amg_handle h, int level, int* n, long long* nnz_lower, long long* nnz_upper,
                             int* depth_lower, int* depth_upper, int* perm, int* lower_ptr, int* lower_col,
                             double* lower_val, int* upper_ptr, int* upper_col, double* upper_val, double* pivots);

/* The dense Gauss-Seidel map of a level of at most 4608 pressures: the n_p x n_p
 * matrix M (row-major) with dp = M g for the gs_iters Gauss-Seidel iterations on
 * S dp = g from dp = 0 in the order (strip parity, color, index) (Section 5.2's
 * Schur complement solve, as one linear map), formed at setup by running the sweep
 * on every unit vector (on the GPU with device_setup).  *n gets n_p; M may be NULL.
 * AMG_ERR_ARG for a level without a map (larger levels, the coarsest). */
amg_status amg_level_get_gs_map(amg_handle h, int level, int* n, double* M);

/* The coarsest level's FP64 pseudo-inverse X (N_c x N_c, row-major, N_c the N of
 * the last level), which the coarsest solve applies: the minimum-norm solution of
 * the (possibly singular) coarsest system, formed at setup by a one-sided Jacobi
 * SVD with singular values below 1e-12 of the largest dropped, then (N_c <= 512, so
 * always with the default max_coarse) refined by two Newton-Schulz steps
 * X <- X + X (I - A X) whose residual is summed in about twice the working
 * precision.  *n gets N_c; X (N_c * N_c doubles) may be NULL. */
amg_status amg_coarse_inverse(amg_handle h, int* n, double* X);

/* Bounded waits (the pipelined Gauss-Seidel kernel's waits on neighbouring strips,
 * the ILU(1) substitutions' waits on earlier rows) give up after this many polls,
 * set the cycle's error word and return, so a kernel always ends; the solve then
 * returns AMG_ERR_CUDA ("a bounded device wait timed out").  polls <= 0 restores
 * the default of 2^24 polls (seconds).  A low limit makes waits run out on purpose
 * (tests of the failure path); results of a cycle whose wait ran out are not
 * meaningful.  Applies to the handle's own cycles (not to a server's clones), and
 * every solve clears the error word when it starts.  Synchronous. */
amg_status amg_set_wait_limit(amg_handle h, long long polls);

/* The Gauss-Seidel variant the V-cycle (FP32 one if built, else FP64) uses on a
 * level for nrhs right-hand sides: -1 not chosen yet (the cycle for that K has
 * not run), 0 one block, 1 a cluster of *cluster blocks, 2 the pipelined strip
 * kernel, 3 one launch per phase, 4 the dense map (levels of at most 4608
 * pressures: the iterations' linear map formed at setup by the same sweeps and
 * applied as one dense product); *ms is the time the autotuner measured for one
 * launch (0 without autotuning).  Either output may be NULL. */
int amg_gs_variant(amg_handle h, int level, int nrhs, int* cluster, float* ms);

/* Fix the Gauss-Seidel variant (numbering of amg_gs_variant; `cluster` is the cluster
 * size or the pipelined kernel's shape 0-3, else 0) of a level for nrhs right-hand
 * sides in both of the handle's V-cycles, in place of the autotuner's choice.  Every
 * variant relaxes the same rows in the same order (the dense map applies the same
 * sweeps' linear map); they differ only in rounding.  A cycle already captured for that
 * nrhs is captured again on its next use.  Returns AMG_ERR_ARG if the level, nrhs or
 * variant does not apply (a dense map on a level without one, a cluster size the level
 * has no plan for, a pipelined shape outside 0-3).  Synchronises the device; not for a
 * handle whose request server is running. */
amg_status amg_set_gs_variant(amg_handle h, int level, int nrhs, int variant, int cluster);

/* The row mapping of a sparse kernel on a level for nrhs right-hand sides, as the
 * autotuner chose it (or by default): kernel = 0 velocity predictor, 1 Schur
 * right-hand side, 3 update, 4 residual, 5 restriction, 6 prolongation (the
 * classes of amg_profile_vcycle); result 0 one group of K/V threads per row with V
 * columns of 16 bytes each, 1 and 2 a row split over 2 or 4 such groups, 3 one
 * column per thread with several lanes per row; -1 for a bad argument. */
int amg_row_shape(amg_handle h, int level, int nrhs, int kernel);

void amg_hierarchy_destroy(amg_handle h);

const char* amg_last_error(void);

/* ------------------------------------------------------------------------
 * Request server: continuous batching of FGMRES solves on one device.
 *
 * The paper has no counterpart: it solves one system at a time.  The server
 * serves many solves (different hierarchies: mesh sizes, Reynolds numbers)
 * concurrently.  Each running request owns a slot: a clone of its hierarchy's
 * V-cycle (matrices shared with the hierarchy, vectors and CUDA graphs its own),
 * an FGMRES workspace for K = nrhs rounded up to a power of two, device copies of
 * b and x, and a stream.  amg_server_progress() advances every running request
 * whose last chunk of device work has finished by one more chunk (an Arnoldi
 * step or a cycle end) and admits queued requests as slots and memory free up,
 * so their kernels overlap on the device.
 *
 * Batching: a request starts together with the later queued requests on the
 * same hierarchy and rtol whose right-hand sides fit beside its own within
 * merge_k columns; the cohort's columns are stacked into one FGMRES solve (each
 * column keeps its own Krylov space, Hessenberg matrix and convergence test), so
 * one matrix pass of every V-cycle kernel serves all of them.  With merge_k <= 1 a
 * request runs alone and its result is bit-identical to amg_fgmres_solve_host()
 * of the same right-hand sides (restart and maxit set to the server's); in a
 * cohort of K columns its columns are computed by the K-column kernels, which
 * round differently from the kernels of its own width.
 *
 * Admission: a queued request takes an idle slot of the same (hierarchy, K), or
 * a new slot while fewer than max_active requests run and the slot's bytes fit
 * device_bytes (idle slots of other shapes are released, least recently used
 * first, to make room).  Requests are considered in submission order; one that
 * does not fit yet stays queued while later ones may start.
 *
 * One host thread drives a server.  Its hierarchies must outlive it, and must
 * not be used through the other entry points while the server has requests on
 * them (amg_fgmres_solve shares nothing with the server's slots, but the handle
 * is not thread safe).
 * ---------------------------------------------------------------------- */
typedef struct amg_server* amg_server_handle;

typedef struct {
  int max_active;      /* requests running at once (one stream each), 1..256; default 16 */
  size_t device_bytes; /* device memory the slots may hold; 0 = 80% of the free memory at creation */
  int restart;         /* FGMRES restart length of every request; default 100 */
  int maxit;           /* iteration limit per right-hand side; default 500 */
  int merge_k;         /* most columns stacked into one cohort, 0..32; default 8; <= 1: no batching */
  int policy;          /* admission order: 0 (default) submission order; 1 smallest work first
                          (N x columns rounded up), submission order among equals: lower median
                          latency under overload, but a large request can wait while smaller
                          ones keep arriving */
} amg_server_params;

typedef struct {
  int queued, running, slots; /* running: requests; slots: slots held (busy or idle) */
  int busy_slots;             /* slots running a cohort */
  size_t bytes_in_use, budget;
  long long kernel_launches; /* kernels launched for the server's requests (graph nodes counted) */
  long long slots_created, slots_released, errors;
  long long cohorts;          /* solves started (a cohort is one or more requests) */
} amg_server_stats;

void amg_server_params_default(amg_server_params* p);
amg_status amg_server_create(const amg_server_params* prm, amg_server_handle* out);

/* Queue one solve of A x = b with nrhs right-hand sides (1..32) to relative
 * residual rtol.  b_host and x_host are HOST arrays, N x nrhs row-major, owned
 * by the caller: b_host is read and x_host written while the request runs, so
 * both must stay valid until its result has been collected.  Page-locked
 * memory keeps the copies asynchronous (pageable x_host makes the final copy
 * wait for the request's own stream).  *ticket identifies the request. */
amg_status amg_server_submit(amg_server_handle sv, amg_handle h, const double* b_host, double* x_host, int nrhs,
                             double rtol, long long* ticket);

/* Create idle slots for requests of nrhs right-hand sides on h until count
 * slots of that shape exist, capturing their V-cycle graphs, so the first such
 * requests start without allocation or capture.  AMG_ERR_OOM when the budget is
 * exhausted first (the slots made so far stay).  Reserved slots are released
 * like any idle slot when room is needed for another shape. */
amg_status amg_server_reserve(amg_server_handle sv, amg_handle h, int nrhs, int count);

/* Never blocks: advances the running requests whose device work has finished,
 * admits queued requests, and writes up to cap tickets of requests that have
 * completed since they were last reported to done[] (count in *n_done). */
amg_status amg_server_progress(amg_server_handle sv, long long* done, int cap, int* n_done);

/* *state = 0 queued, 1 running, 2 done.  For a done request also fills iters
 * and relres (nrhs entries each, as amg_fgmres_solve), seconds[0] = queueing
 * time and seconds[1] = submission to completion (host clock; completion is
 * when progress() saw the last chunk finish), *status = the solve's status; the
 * request is then forgotten (a second call with its ticket is AMG_ERR_ARG).
 * Any output pointer may be NULL. */
amg_status amg_server_result(amg_server_handle sv, long long ticket, int* state, int* iters, double* relres,
                             double* seconds, amg_status* status);

/* *state of a request (0 queued, 1 running, 2 done) without collecting it. */
amg_status amg_server_state(amg_server_handle sv, long long ticket, int* state);

amg_status amg_server_get_stats(amg_server_handle sv, amg_server_stats* st);

/* Waits for the device work in flight, then frees every slot. */
void amg_server_destroy(amg_server_handle sv);

/* Message of the server's last asynchronous failure, else of the calling
 * thread's last failing amg_server_* call. */
const char* amg_server_last_error(amg_server_handle sv);

#ifdef __cplusplus
}
#endif
#endif /* EMIN_AMG_H */

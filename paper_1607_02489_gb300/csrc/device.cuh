// Device data and kernels of the V-cycle (Alg. 1's relaxation form, Section 5.2
// Braess-Sarazin, Section 4 transfers) and of flexible GMRES.
//
// Vectors hold K right-hand sides interleaved: entry (dof i, rhs k) at i*K + k,
// dofs ordered [u_x | u_y (| u_z) | p].  One thread computes one (row, rhs)
// pair; the K threads of a row read the row's matrix entries once (broadcast)
// and the K values of each column entry as one contiguous segment.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace emin {

constexpr int kBlock = 256;

template <typename T>
struct DCsr {
  int nrows = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const T* v = nullptr;
};

// Everything a level's kernels read; passed by value.
template <typename T>
struct LevelView {
  int dim, n_v, n_p, pinned;
  DCsr<T> A, B, Bt;
  // Schur complement with rows grouped by color: row r is pressure S_perm[r],
  // off-diagonal entries only, S_dinv[r] = 1 / S_ii.
  DCsr<T> S;
  const int* S_perm;
  const T* S_dinv;
  const T* w;  // 1 / (c D_i), 1 on Dirichlet rows
  // transfers to the next level: P (n_v x n_vc), Pp, R (n_vc x n_v), Rp
  DCsr<T> P, Pp, R, Rp;
  int n_vc, n_pc;
};

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

inline unsigned grid_for(long long items) { return (unsigned)((items + kBlock - 1) / kBlock); }

// y = x + w .* (b_u - A u - Bt p) on velocity rows; with zero_x, y = w .* b_u.
// (Braess-Sarazin step, first half: the Jacobi-like velocity predictor.)
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_bs_velocity(LevelView<T> L, const T* __restrict__ b,
                                                        const T* __restrict__ x, T* __restrict__ y, int zero_x) {
  const long long t = gtid();
  const int i = (int)(t / K), k = (int)(t % K);
  if (i >= L.n_v) return;
  const size_t nuK = (size_t)L.dim * L.n_v * K;
  T acc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    if (c < L.dim) acc[c] = b[((size_t)c * L.n_v + i) * K + k];
  if (!zero_x) {
    for (int e = L.A.rp[i]; e < L.A.rp[i + 1]; ++e) {
      const T a = L.A.v[e];
      const size_t j = (size_t)L.A.ci[e];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < L.dim) acc[c] -= a * x[((size_t)c * L.n_v + j) * K + k];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const int r = c * L.n_v + i;
        for (int e = L.Bt.rp[r]; e < L.Bt.rp[r + 1]; ++e) acc[c] -= L.Bt.v[e] * x[nuK + (size_t)L.Bt.ci[e] * K + k];
      }
  }
  const T wi = L.w[i];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    if (c < L.dim) {
      const size_t o = ((size_t)c * L.n_v + i) * K + k;
      y[o] = (zero_x ? T(0) : x[o]) + wi * acc[c];
    }
}

// Schur right-hand side g = c (B y - b_p) (= B D^-1 r_u - c r_p); pinned row g = r_p.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_schur_rhs(LevelView<T> L, const T* __restrict__ b,
                                                      const T* __restrict__ x, const T* __restrict__ y,
                                                      T* __restrict__ g, T cfac, int zero_x) {
  const long long t = gtid();
  const int i = (int)(t / K), k = (int)(t % K);
  if (i >= L.n_p) return;
  const size_t nuK = (size_t)L.dim * L.n_v * K;
  T acc = T(0);
  for (int e = L.B.rp[i]; e < L.B.rp[i + 1]; ++e) acc += L.B.v[e] * y[(size_t)L.B.ci[e] * K + k];
  const T bp = b[nuK + (size_t)i * K + k];
  if (i == L.pinned)
    g[(size_t)i * K + k] = bp - (zero_x ? T(0) : x[nuK + (size_t)i * K + k]);
  else
    g[(size_t)i * K + k] = cfac * (acc - bp);
}

// One color of a Gauss-Seidel iteration on S dp = g: rows of one color share no
// entry of S, so they are updated concurrently.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_gs_color(LevelView<T> L, const T* __restrict__ g, T* __restrict__ dp,
                                                     int r0, int r1) {
  const long long t = gtid();
  const int r = r0 + (int)(t / K), k = (int)(t % K);
  if (r >= r1) return;
  const int i = L.S_perm[r];
  T acc = g[(size_t)i * K + k];
  for (int e = L.S.rp[r]; e < L.S.rp[r + 1]; ++e) acc -= L.S.v[e] * dp[(size_t)L.S.ci[e] * K + k];
  dp[(size_t)i * K + k] = acc * L.S_dinv[r];
}

// u = y - w .* (Bt dp), p = p + dp (p = dp with zero_x): the velocity/pressure update.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_bs_update(LevelView<T> L, const T* __restrict__ y,
                                                      const T* __restrict__ dp, T* __restrict__ x, int zero_x) {
  const long long t = gtid();
  const int i = (int)(t / K), k = (int)(t % K);
  const size_t nuK = (size_t)L.dim * L.n_v * K;
  if (i < L.n_v) {
    const T wi = L.w[i];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const int r = c * L.n_v + i;
        T s = T(0);
        for (int e = L.Bt.rp[r]; e < L.Bt.rp[r + 1]; ++e) s += L.Bt.v[e] * dp[(size_t)L.Bt.ci[e] * K + k];
        const size_t o = (size_t)r * K + k;
        x[o] = y[o] - wi * s;
      }
  } else if (i < L.n_v + L.n_p) {
    const int q = i - L.n_v;
    const size_t o = nuK + (size_t)q * K + k;
    x[o] = (zero_x ? T(0) : x[o]) + dp[(size_t)q * K + k];
  }
}

// out = b - A x (HAS_B) or out = A x, for the whole block matrix [I(x)A, Bt; B, C].
template <typename T, typename TX, typename TO, int K, bool HAS_B>
__global__ void __launch_bounds__(kBlock) k_block_spmv(LevelView<T> L, const T* __restrict__ b,
                                                       const TX* __restrict__ x, TO* __restrict__ out) {
  const long long t = gtid();
  const int i = (int)(t / K), k = (int)(t % K);
  const size_t nuK = (size_t)L.dim * L.n_v * K;
  if (i < L.n_v) {
    T acc[3] = {T(0), T(0), T(0)};
    for (int e = L.A.rp[i]; e < L.A.rp[i + 1]; ++e) {
      const T a = L.A.v[e];
      const size_t j = (size_t)L.A.ci[e];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < L.dim) acc[c] += a * (T)x[((size_t)c * L.n_v + j) * K + k];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const int r = c * L.n_v + i;
        for (int e = L.Bt.rp[r]; e < L.Bt.rp[r + 1]; ++e) acc[c] += L.Bt.v[e] * (T)x[nuK + (size_t)L.Bt.ci[e] * K + k];
        const size_t o = (size_t)r * K + k;
        out[o] = (TO)(HAS_B ? b[o] - acc[c] : acc[c]);
      }
  } else if (i < L.n_v + L.n_p) {
    const int q = i - L.n_v;
    T acc = T(0);
    for (int e = L.B.rp[q]; e < L.B.rp[q + 1]; ++e) acc += L.B.v[e] * (T)x[(size_t)L.B.ci[e] * K + k];
    const size_t o = nuK + (size_t)q * K + k;
    if (q == L.pinned) acc += (T)x[o];
    out[o] = (TO)(HAS_B ? b[o] - acc : acc);
  }
}

// b_c = R r: velocity rows by R (each component), pressure rows by Rp.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_restrict(LevelView<T> L, const T* __restrict__ r, T* __restrict__ bc) {
  const long long t = gtid();
  const int I = (int)(t / K), k = (int)(t % K);
  if (I < L.n_vc) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        T s = T(0);
        for (int e = L.R.rp[I]; e < L.R.rp[I + 1]; ++e) s += L.R.v[e] * r[((size_t)c * L.n_v + L.R.ci[e]) * K + k];
        bc[((size_t)c * L.n_vc + I) * K + k] = s;
      }
  } else if (I < L.n_vc + L.n_pc) {
    const int q = I - L.n_vc;
    const size_t nuK = (size_t)L.dim * L.n_v * K;
    T s = T(0);
    for (int e = L.Rp.rp[q]; e < L.Rp.rp[q + 1]; ++e) s += L.Rp.v[e] * r[nuK + (size_t)L.Rp.ci[e] * K + k];
    bc[((size_t)L.dim * L.n_vc + q) * K + k] = s;
  }
}

// x += P x_c: velocity rows by P (each component), pressure rows by Pp.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_prolong(LevelView<T> L, const T* __restrict__ xc, T* __restrict__ x) {
  const long long t = gtid();
  const int i = (int)(t / K), k = (int)(t % K);
  if (i < L.n_v) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        T s = T(0);
        for (int e = L.P.rp[i]; e < L.P.rp[i + 1]; ++e) s += L.P.v[e] * xc[((size_t)c * L.n_vc + L.P.ci[e]) * K + k];
        x[((size_t)c * L.n_v + i) * K + k] += s;
      }
  } else if (i < L.n_v + L.n_p) {
    const int q = i - L.n_v;
    T s = T(0);
    for (int e = L.Pp.rp[q]; e < L.Pp.rp[q + 1]; ++e) s += L.Pp.v[e] * xc[((size_t)L.dim * L.n_vc + L.Pp.ci[e]) * K + k];
    x[((size_t)L.dim * L.n_v + q) * K + k] += s;
  }
}

// Coarsest level: x = A^+ b with the FP64 pseudo-inverse, whatever T is.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_coarse_solve(int Nc, const double* __restrict__ pinv,
                                                         const T* __restrict__ b, T* __restrict__ x) {
  const long long t = gtid();
  const int i = (int)(t / K), k = (int)(t % K);
  if (i >= Nc) return;
  double s = 0.0;
  const double* row = pinv + (size_t)i * Nc;
  for (int j = 0; j < Nc; ++j) s += row[j] * (double)b[(size_t)j * K + k];
  x[(size_t)i * K + k] = (T)s;
}

// dst (N x K) = src (N x ld, first nrhs columns, converted), zero padding.
template <typename TS, typename TD, int K>
__global__ void __launch_bounds__(kBlock) k_pack(long long N, const TS* __restrict__ src, int ld, int nrhs,
                                                 TD* __restrict__ dst) {
  const long long t = gtid();
  if (t >= N * K) return;
  const long long i = t / K;
  const int k = (int)(t % K);
  dst[t] = k < nrhs ? (TD)src[i * ld + k] : TD(0);
}

template <typename TS, typename TD, int K>
__global__ void __launch_bounds__(kBlock) k_unpack(long long N, const TS* __restrict__ src, int nrhs,
                                                   TD* __restrict__ dst, int ld) {
  const long long t = gtid();
  if (t >= N * nrhs) return;
  const long long i = t / nrhs;
  const int k = (int)(t % nrhs);
  dst[i * ld + k] = (TD)src[i * K + k];
}

}  // namespace emin

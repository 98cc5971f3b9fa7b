// Device data and kernels of the V-cycle (Alg. 1's relaxation form, Section 5.2
// Braess-Sarazin, Section 4 transfers) and of flexible GMRES.
//
// Vectors hold K right-hand sides interleaved: entry (dof i, rhs k) at i*K + k,
// dofs ordered [u_x | u_y (| u_z) | p].  A row is handled by K*G consecutive
// lanes of a warp: lane (k, g) takes right-hand side k and every G-th stored
// entry of the row starting at g, so one load instruction reads G consecutive
// matrix entries and, for each, the K contiguous values of its column; the G
// partial sums are combined with warp shuffles.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace emin {

constexpr int kBlock = 256;
constexpr int kGsBlock = 512;
constexpr int kGsPipeBlock = 512;
constexpr int kMaxColors = 255;  // colors of a Schur graph the pipelined kernel accepts

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

// Row mapping.  A row is handled by (K/V)*G threads: each takes V consecutive
// right-hand sides (one 16-byte vector load per matrix entry on large levels)
// and G lanes split the row's stored entries (small, latency-bound levels),
// combining their partial sums with warp shuffles.  Vector indices are 32-bit
// (the hierarchy checks N * K < 2^31 at creation).
template <int K>
struct RowLanes {
  static constexpr int G = K >= 32 ? 1 : (32 / K < 4 ? 32 / K : 4);
  static constexpr int W = K * G;
};
// Below this many (row, rhs) pairs a level is not wide enough for one thread per
// V right-hand sides to hide latency: it uses G > 1 lanes per row and V = 1.
constexpr long long kSmallLevelItems = 1LL << 20;

template <typename T, int K>
struct VecWidth {  // right-hand sides per thread on large levels: 16 bytes, at most K
  static constexpr int V = (int)(16 / sizeof(T)) < K ? (int)(16 / sizeof(T)) : K;
};

template <int K, int G, int V>
struct RowMap {
  static constexpr int KV = K / V;
  static constexpr int W = KV * G;
  unsigned row, k0, lane;
  __device__ __forceinline__ RowMap(long long t)
      : row((unsigned)(t / W)), k0((unsigned)(t % KV) * V), lane((unsigned)((t / KV) % G)) {}
};

// Mask of the W-lane group (aligned within the warp) of the calling thread.
template <int W>
__device__ __forceinline__ unsigned group_mask() {
  return W == 32 ? 0xffffffffu : (((1u << W) - 1u) << ((threadIdx.x & 31) & ~(unsigned)(W - 1)));
}

template <int K, int G, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
  for (int off = G / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(mask, v, off * K);
  return v;
}

// V consecutive values at p (aligned to V values) into / out of registers.
template <typename T, int V>
__device__ __forceinline__ void vld(T (&r)[V], const T* __restrict__ p) {
  if constexpr (sizeof(T) == 4 && V == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
  } else if constexpr (sizeof(T) == 4 && V == 2) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    r[0] = q.x; r[1] = q.y;
  } else if constexpr (sizeof(T) == 8 && V == 2) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    r[0] = q.x; r[1] = q.y;
  } else {
#pragma unroll
    for (int u = 0; u < V; ++u) r[u] = p[u];
  }
}
template <typename T, int V>
__device__ __forceinline__ void vst(T* __restrict__ p, const T (&r)[V]) {
  if constexpr (sizeof(T) == 4 && V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
  } else if constexpr (sizeof(T) == 4 && V == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(r[0], r[1]);
  } else if constexpr (sizeof(T) == 8 && V == 2) {
    *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
  } else {
#pragma unroll
    for (int u = 0; u < V; ++u) p[u] = r[u];
  }
}

// y = x + w .* (b_u - A u - Bt p) on velocity rows; with zero_x, y = w .* b_u.
// (Braess-Sarazin step, first half: the Jacobi-like velocity predictor.)
template <typename T, int K, int G, int V>
__global__ void __launch_bounds__(kBlock) k_bs_velocity(LevelView<T> L, const T* __restrict__ b,
                                                        const T* __restrict__ x, T* __restrict__ y, int zero_x) {
  using M = RowMap<K, G, V>;
  const M q(gtid());
  const unsigned i = q.row, k0 = q.k0;
  if (i >= (unsigned)L.n_v) return;
  const unsigned nvK = (unsigned)L.n_v * K, nuK = (unsigned)L.dim * nvK;
  T acc[3][V];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int u = 0; u < V; ++u) acc[c][u] = T(0);
  if (!zero_x) {
    for (int e = L.A.rp[i] + q.lane; e < L.A.rp[i + 1]; e += G) {
      const T a = L.A.v[e];
      const unsigned j = (unsigned)L.A.ci[e] * K + k0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < L.dim) {
          T xv[V];
          vld<T, V>(xv, x + c * nvK + j);
#pragma unroll
          for (int u = 0; u < V; ++u) acc[c][u] += a * xv[u];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const unsigned r = c * L.n_v + i;
        for (int e = L.Bt.rp[r] + q.lane; e < L.Bt.rp[r + 1]; e += G) {
          const T bv = L.Bt.v[e];
          T xv[V];
          vld<T, V>(xv, x + nuK + (unsigned)L.Bt.ci[e] * K + k0);
#pragma unroll
          for (int u = 0; u < V; ++u) acc[c][u] += bv * xv[u];
        }
      }
    if constexpr (G > 1) {
      const unsigned mask = group_mask<M::W>();
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int u = 0; u < V; ++u) acc[c][u] = group_sum<M::KV, G>(acc[c][u], mask);
    }
  }
  if (q.lane != 0) return;
  const T wi = L.w[i];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    if (c < L.dim) {
      const unsigned o = c * nvK + i * K + k0;
      T bv[V], xv[V], out[V];
      vld<T, V>(bv, b + o);
      if (!zero_x) vld<T, V>(xv, x + o);
#pragma unroll
      for (int u = 0; u < V; ++u) out[u] = (zero_x ? T(0) : xv[u]) + wi * (bv[u] - acc[c][u]);
      vst<T, V>(y + o, out);
    }
}

// Schur right-hand side g = c (B y - b_p) (= B D^-1 r_u - c r_p); pinned row g = r_p.
template <typename T, int K, int G, int V>
__global__ void __launch_bounds__(kBlock) k_schur_rhs(LevelView<T> L, const T* __restrict__ b,
                                                      const T* __restrict__ x, const T* __restrict__ y,
                                                      T* __restrict__ g, T cfac, int zero_x) {
  using M = RowMap<K, G, V>;
  const M q(gtid());
  const unsigned i = q.row, k0 = q.k0;
  if (i >= (unsigned)L.n_p) return;
  const unsigned nuK = (unsigned)L.dim * L.n_v * K;
  T acc[V];
#pragma unroll
  for (int u = 0; u < V; ++u) acc[u] = T(0);
  for (int e = L.B.rp[i] + q.lane; e < L.B.rp[i + 1]; e += G) {
    const T bv = L.B.v[e];
    T yv[V];
    vld<T, V>(yv, y + (unsigned)L.B.ci[e] * K + k0);
#pragma unroll
    for (int u = 0; u < V; ++u) acc[u] += bv * yv[u];
  }
  if constexpr (G > 1) {
    const unsigned mask = group_mask<M::W>();
#pragma unroll
    for (int u = 0; u < V; ++u) acc[u] = group_sum<M::KV, G>(acc[u], mask);
  }
  if (q.lane != 0) return;
  T bp[V], out[V];
  vld<T, V>(bp, b + nuK + i * K + k0);
  if ((int)i == L.pinned) {
    T xp[V];
    if (!zero_x) vld<T, V>(xp, x + nuK + i * K + k0);
#pragma unroll
    for (int u = 0; u < V; ++u) out[u] = bp[u] - (zero_x ? T(0) : xp[u]);
  } else {
#pragma unroll
    for (int u = 0; u < V; ++u) out[u] = cfac * (acc[u] - bp[u]);
  }
  vst<T, V>(g + i * K + k0, out);
}

// Bounded waits: a block polling a counter that another block publishes gives
// up after a limit of polls (by default kSpinLimit, seconds), sets *err and
// returns, so a wait can never hang the GPU; the host checks *err after the
// cycle.  The error word and the limit share one device allocation: err[0] is
// the error word, err[2..3] the limit as a 64-bit count (the host lowers it to
// make waits run out on purpose, for tests of the failure path).
constexpr unsigned long long kSpinLimit = 1ull << 24;
__device__ __forceinline__ unsigned long long wait_limit(const int* err) {
  return *reinterpret_cast<const volatile unsigned long long*>(err + 2);
}

// Strip-ordered Gauss-Seidel for the Schur system S dp = g, gs_iters iterations
// from dp = 0.  Rows are relaxed in the order (strip parity, color, index):
// strips are T consecutive rows and every entry of S couples rows of the same
// or adjacent strips, so the strips of one parity never share an entry of S and
// are relaxed concurrently, one block per strip; inside a strip the rows of one
// color are independent.  A strip reads only rows within T of itself, so its
// block stages that halo of dp (stage >= 1) and its own rows of S (stage == 2)
// in shared memory and runs the color sub-steps there with __syncthreads.
// k_gs_strips runs the phases [ph0, ph1) (phase = 2 * iteration + parity); a
// launch of several blocks runs exactly one phase, so no block ever waits for
// another.  G lanes share a row and combine their sums with warp shuffles.
struct GsStrips {
  const int* soff;  // nstrips x (ncol + 1): first sorted row of each (strip, color)
  int nstrips, ncol, T, iters, stage, max_strip_nnz;
};

// Asynchronous global -> shared copies (cp.async): every copy of a staging
// step is in flight at once and lands without a register round trip.
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copy n elements of type U from global to shared with cp.async, in 16-byte
// pieces when both addresses allow it.  COHERENT data (written by other blocks
// in the previous phase) is read only through L2: 16-byte cp.async.cg, or
// ld.global.cg for an unaligned remainder.
template <bool COHERENT, typename U>
__device__ __forceinline__ void stage_copy(U* sdst, const U* gsrc, int n) {
  const uintptr_t a = (uintptr_t)gsrc, b = (uintptr_t)__cvta_generic_to_shared(sdst);
  const int per16 = 16 / (int)sizeof(U);
  int done = 0;
  if (((a | b) & 15) == 0) {
    const int n16 = n / per16;
    for (int t = threadIdx.x; t < n16; t += blockDim.x) cp_async(sdst + t * per16, gsrc + t * per16, 16);
    done = n16 * per16;
  }
  for (int t = done + threadIdx.x; t < n; t += blockDim.x) {
    if (COHERENT)
      sdst[t] = __ldcg(gsrc + t);
    else
      cp_async(sdst + t, gsrc + t, (int)sizeof(U));
  }
}

template <typename T, int K, int G>
__global__ void __launch_bounds__(kGsBlock) k_gs_strips(LevelView<T> L, const T* __restrict__ g, T* dp, GsStrips P,
                                                        int ph0, int ph1) {
  static_assert(K * G <= 32, "a row group must fit in a warp");
  extern __shared__ __align__(16) unsigned char smem[];
  // layout: dp halo (3T x K), g (T x K), 1/S_ii (T), [S values], then ints:
  // row offsets (T+1), permutation (T), [S columns]
  T* s_dp = reinterpret_cast<T*>(smem);
  T* s_g = s_dp + (size_t)3 * P.T * K;
  T* s_dinv = s_g + (size_t)P.T * K;
  T* s_v = s_dinv + P.T;
  int* s_rp = reinterpret_cast<int*>(s_v + (P.stage == 2 ? P.max_strip_nnz : 0));
  int* s_perm = s_rp + P.T + 1;
  int* s_ci = s_perm + P.T;
  constexpr int kGroup = K * G;
  const int k = threadIdx.x % K;
  const int lane = (threadIdx.x / K) % G;
  const unsigned mask = kGroup == 32 ? 0xffffffffu
                                     : (((1u << kGroup) - 1u) << ((threadIdx.x & 31) & ~(unsigned)(kGroup - 1)));
  const int n_p = L.n_p;
  for (int ph = ph0; ph < ph1; ++ph) {
    const int bc = ph & 1;
    {
      for (int s = bc + 2 * blockIdx.x; s < P.nstrips; s += 2 * gridDim.x) {
        const int r_lo = s * P.T, r_hi = min(r_lo + P.T, n_p);
        const int h_lo = max(0, r_lo - P.T), h_hi = min(n_p, r_hi + P.T);
        const int* so = P.soff + (size_t)s * (P.ncol + 1);
        const int q0 = so[0], q1 = so[P.ncol];  // sorted rows of this strip
        const int e0 = L.S.rp[q0], e1 = L.S.rp[q1];
        if (P.stage >= 1) {
          stage_copy<true>(s_dp, dp + (size_t)h_lo * K, (h_hi - h_lo) * K);
          stage_copy<false>(s_g, g + (size_t)r_lo * K, (r_hi - r_lo) * K);
          stage_copy<false>(s_dinv, L.S_dinv + q0, q1 - q0);
          stage_copy<false>(s_perm, L.S_perm + q0, q1 - q0);
          stage_copy<false>(s_rp, L.S.rp + q0, q1 - q0 + 1);
          if (P.stage == 2) {
            stage_copy<false>(s_v, L.S.v + e0, e1 - e0);
            stage_copy<false>(s_ci, L.S.ci + e0, e1 - e0);
          }
          cp_async_wait_all();
        }
        __syncthreads();
        for (int pc = 0; pc < P.ncol; ++pc) {
          const int ra = so[pc], rb = so[pc + 1];
          const int items = (rb - ra) * kGroup;
          for (int t = threadIdx.x; t < items; t += blockDim.x) {
            const int r = ra + t / kGroup;
            T acc = T(0);
            if (P.stage == 2) {
              const int ea = s_rp[r - q0] - e0, eb = s_rp[r - q0 + 1] - e0;
              for (int e = ea + lane; e < eb; e += G) acc += s_v[e] * s_dp[(size_t)(s_ci[e] - h_lo) * K + k];
            } else if (P.stage == 1) {
              const int ea = s_rp[r - q0], eb = s_rp[r - q0 + 1];
              for (int e = ea + lane; e < eb; e += G) acc += L.S.v[e] * s_dp[(size_t)(L.S.ci[e] - h_lo) * K + k];
            } else {
              const int ea = L.S.rp[r], eb = L.S.rp[r + 1];
              for (int e = ea + lane; e < eb; e += G) acc += L.S.v[e] * dp[(size_t)L.S.ci[e] * K + k];
            }
#pragma unroll
            for (int off = G / 2; off >= 1; off >>= 1) acc += __shfl_xor_sync(mask, acc, off * K);
            if (lane == 0) {
              if (P.stage >= 1) {
                const int i = s_perm[r - q0];
                s_dp[(size_t)(i - h_lo) * K + k] = (s_g[(size_t)(i - r_lo) * K + k] - acc) * s_dinv[r - q0];
              } else {
                const int i = L.S_perm[r];
                dp[(size_t)i * K + k] = (g[(size_t)i * K + k] - acc) * L.S_dinv[r];
              }
            }
          }
          __syncthreads();
        }
        if (P.stage >= 1)
          for (int t = threadIdx.x; t < (r_hi - r_lo) * K; t += blockDim.x)
            dp[(size_t)r_lo * K + t] = s_dp[(size_t)(r_lo - h_lo) * K + t];
        __syncthreads();
      }
    }
  }
}

// Pipelined strip Gauss-Seidel: the same ordering as k_gs_strips in one launch
// and without grid barriers.  The work is cut into units (iteration it, strip s),
// numbered iteration by iteration with the even strips before the odd ones, which
// is a topological order of their dependencies: an even strip at iteration it
// needs its odd neighbours to have completed it iterations, an odd strip needs its
// even neighbours to have completed it + 1, and each strip needs its own previous
// unit.  (That is the sequential order's dependency, and it also keeps a strip from
// overwriting rows a neighbour has not read yet.)  Blocks take units from a ticket
// counter in that order, so a unit only ever waits for units already taken by
// running blocks: the kernel needs no co-residency, runs with any grid size and
// alongside any other work on the device.  Per-strip counters of completed
// iterations carry the dependencies (release / acquire).  A block stages the
// strip's rows of S, 1/S_ii and g while it waits, then the dp halo.  Waits are
// bounded (the wait_limit polls), set *err and return on timeout.
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// done[0..nstrips) are the per-strip counters and done[nstrips] the ticket
// counter; all are zero at launch, and dp is zero.
// In FP32 an entry of S is one 8-byte word (column relative to the strip's halo,
// value bits), pk: one shared-memory load per entry instead of two.
template <typename T, int K, int G, int V, int NT>
__global__ void __launch_bounds__(NT) k_gs_pipe(LevelView<T> L, const T* __restrict__ g, T* dp, GsStrips P,
                                                const int* __restrict__ ci_rel, const int2* __restrict__ pk,
                                                int* done, int* err) {
  static_assert((K / V) * G <= 32, "a row group must fit in a warp");
  constexpr bool PK = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smem[];
  T* s_dp = reinterpret_cast<T*>(smem);
  T* s_g = s_dp + (size_t)3 * P.T * K;
  T* s_dinv = s_g + (size_t)P.T * K;
  T* s_v = s_dinv + P.T;
  int* s_rp = reinterpret_cast<int*>(s_v + (!PK && P.stage == 2 ? P.max_strip_nnz : 0));
  int* s_perm = s_rp + P.T + 1;
  int* s_ci = s_perm + P.T;
  int2* s_pk = reinterpret_cast<int2*>(smem + ((reinterpret_cast<unsigned char*>(s_ci) - smem + 15) & ~(size_t)15));
  __shared__ int s_fail, s_unit;
  __shared__ int s_so[kMaxColors + 1];  // this strip's color offsets (sorted rows)
  constexpr int KV = K / V;
  constexpr int kGroup = KV * G;
  const int k = (threadIdx.x % KV) * V;
  const int lane = (threadIdx.x / KV) % G;
  const unsigned mask = group_mask<kGroup>();
  const int n_p = L.n_p;
  const int nunits = P.iters * P.nstrips;
  const int n_even = (P.nstrips + 1) / 2;
  int* ticket = done + P.nstrips;
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = atomicAdd(ticket, 1);
      s_fail = 0;
    }
    __syncthreads();
    const int u = s_unit;
    if (u >= nunits) return;
    const int it = u / P.nstrips, w = u - it * P.nstrips;
    const int s = w < n_even ? 2 * w : 2 * (w - n_even) + 1;
    const int par = s & 1;
    const int r_lo = s * P.T, r_hi = min(r_lo + P.T, n_p);
    const int h_lo = max(0, r_lo - P.T), h_hi = min(n_p, r_hi + P.T);
    const int* so_g = P.soff + (size_t)s * (P.ncol + 1);
    for (int t = threadIdx.x; t <= P.ncol; t += blockDim.x) s_so[t] = so_g[t];
    const int q0 = so_g[0], q1 = so_g[P.ncol];
    const int e0 = L.S.rp[q0], e1 = L.S.rp[q1];
    // data no other unit writes, in flight while this unit waits
    stage_copy<false>(s_g, g + (size_t)r_lo * K, (r_hi - r_lo) * K);
    stage_copy<false>(s_dinv, L.S_dinv + q0, q1 - q0);
    stage_copy<false>(s_perm, L.S_perm + q0, q1 - q0);
    stage_copy<false>(s_rp, L.S.rp + q0, q1 - q0 + 1);
    // packed entries land at the 16-byte phase of their global address: whole 16-byte copies
    int2* const s_pke = s_pk + (e0 & 1);
    if (P.stage == 2) {
      if constexpr (PK) {
        stage_copy<false>(s_pke, pk + e0, e1 - e0);
      } else {
        stage_copy<false>(s_v, L.S.v + e0, e1 - e0);
        stage_copy<false>(s_ci, ci_rel + e0, e1 - e0);
      }
    }
    const int need_nb = par == 0 ? it : it + 1;
    if (threadIdx.x == 0) {
      const unsigned long long limit = wait_limit(err);
      for (int nb = s - 1; nb <= s + 1; ++nb) {
        const int need = nb == s ? it : need_nb;
        if (nb < 0 || nb >= P.nstrips || need == 0) continue;
        unsigned long long spins = 0;
        while (ld_acquire(done + nb) < need) {
          if (++spins > limit || *(volatile int*)err) {
            atomicExch(err, 1);
            s_fail = 1;
            break;
          }
          __nanosleep(32);
        }
        if (s_fail) break;
      }
    }
    __syncthreads();
    if (s_fail) {
      cp_async_wait_all();
      return;
    }
    if (need_nb == 0) {
      // first unit of an even strip: dp is still zero around it
      for (int t = threadIdx.x; t < (h_hi - h_lo) * K; t += blockDim.x) s_dp[t] = T(0);
    } else {
      // the halo and this strip's rows as last written (through L2)
      stage_copy<true>(s_dp, dp + (size_t)h_lo * K, (h_hi - h_lo) * K);
    }
    cp_async_wait_all();
    __syncthreads();
    const int* so = s_so;
    for (int pc = 0; pc < P.ncol; ++pc) {
      const int ra = so[pc], rb = so[pc + 1];
      for (int t = threadIdx.x; t < (rb - ra) * kGroup; t += blockDim.x) {
        const int r = ra + t / kGroup;
        const int ea = s_rp[r - q0], eb = s_rp[r - q0 + 1];
        T acc[V];
        const T* sv = P.stage == 2 ? s_v - e0 : L.S.v;
        const int* sc = P.stage == 2 ? s_ci - e0 : ci_rel;
        const int2* sp = P.stage == 2 ? s_pke - e0 : pk;
        // entry e of S: relative column and value
        auto entry = [&](int e, int& c, T& v) {
          if constexpr (PK) {
            const int2 q = sp[e];
            c = q.x;
            v = __int_as_float(q.y);
          } else {
            c = sc[e];
            v = sv[e];
          }
        };
        if constexpr (V > 1 && G == 1) {
          // V columns per thread, whole row: two independent partial sums per column
          T a[V], b2[V];
#pragma unroll
          for (int uu = 0; uu < V; ++uu) a[uu] = b2[uu] = T(0);
          int e = ea;
          for (; e + 1 < eb; e += 2) {
            int c0, c1;
            T v0, v1;
            entry(e, c0, v0);
            entry(e + 1, c1, v1);
            T d0[V], d1[V];
            vld<T, V>(d0, s_dp + c0 * K + k);
            vld<T, V>(d1, s_dp + c1 * K + k);
#pragma unroll
            for (int uu = 0; uu < V; ++uu) {
              a[uu] += v0 * d0[uu];
              b2[uu] += v1 * d1[uu];
            }
          }
          if (e < eb) {
            int c0;
            T v0;
            entry(e, c0, v0);
            T d0[V];
            vld<T, V>(d0, s_dp + c0 * K + k);
#pragma unroll
            for (int uu = 0; uu < V; ++uu) a[uu] += v0 * d0[uu];
          }
#pragma unroll
          for (int uu = 0; uu < V; ++uu) acc[uu] = a[uu] + b2[uu];
        } else {
          // V columns per thread, G lanes per row, four independent partial sums
          T a1[V], a2[V], a3[V];
#pragma unroll
          for (int uu = 0; uu < V; ++uu) acc[uu] = a1[uu] = a2[uu] = a3[uu] = T(0);
          int e = ea + lane;
          for (; e + 3 * G < eb; e += 4 * G) {
            int c0, c1, c2, c3;
            T v0, v1, v2, v3;
            entry(e, c0, v0);
            entry(e + G, c1, v1);
            entry(e + 2 * G, c2, v2);
            entry(e + 3 * G, c3, v3);
            T d0[V], d1[V], d2[V], d3[V];
            vld<T, V>(d0, s_dp + c0 * K + k);
            vld<T, V>(d1, s_dp + c1 * K + k);
            vld<T, V>(d2, s_dp + c2 * K + k);
            vld<T, V>(d3, s_dp + c3 * K + k);
#pragma unroll
            for (int uu = 0; uu < V; ++uu) {
              acc[uu] += v0 * d0[uu];
              a1[uu] += v1 * d1[uu];
              a2[uu] += v2 * d2[uu];
              a3[uu] += v3 * d3[uu];
            }
          }
          for (; e < eb; e += G) {
            int c0;
            T v0;
            entry(e, c0, v0);
            T d0[V];
            vld<T, V>(d0, s_dp + c0 * K + k);
#pragma unroll
            for (int uu = 0; uu < V; ++uu) acc[uu] += v0 * d0[uu];
          }
#pragma unroll
          for (int uu = 0; uu < V; ++uu) acc[uu] = group_sum<KV, G>((acc[uu] + a1[uu]) + (a2[uu] + a3[uu]), mask);
        }
        if (lane == 0) {
          const int i = s_perm[r - q0];
          const T di = s_dinv[r - q0];
          T gv[V], out[V];
          vld<T, V>(gv, s_g + (size_t)(i - r_lo) * K + k);
#pragma unroll
          for (int uu = 0; uu < V; ++uu) out[uu] = (gv[uu] - acc[uu]) * di;
          vst<T, V>(s_dp + (size_t)(i - h_lo) * K + k, out);
        }
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < (r_hi - r_lo) * K; t += blockDim.x)
      dp[(size_t)r_lo * K + t] = s_dp[(size_t)(r_lo - h_lo) * K + t];
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(done + s, it + 1);
    }
  }
}

// Cluster Gauss-Seidel for a mid-size level: the same ordering, with the level's
// strips split over the C blocks of one thread-block cluster, each block holding
// its strips' rows of S, g, 1/S_ii and a dp window (its rows plus one strip on
// each side) in shared memory.  A phase (iteration, parity) relaxes every strip
// of that parity; phases are separated by the cluster barrier, after which a
// block copies the rows of the neighbouring strips that other blocks relaxed in
// the previous phase out of their shared memory (distributed shared memory), so
// nothing goes through global memory between phases.  The hardware schedules a
// cluster's blocks together, so the barrier needs no other guarantee.
// Block c owns strips [c*spc, min((c+1)*spc, nstrips)); plist holds, at each
// block's sorted rows, those rows grouped by (parity, color), poff[c] the offsets.
struct GsCluster {
  const int* soff;   // nstrips x (ncol + 1), as GsStrips
  const int* plist;  // n_p sorted rows, each block's segment grouped by (parity, color)
  const int* poff;   // C x (2 ncol + 1)
  int nstrips, ncol, T, iters, spc;
  int win_max, rows_max, nnz_max;  // shared-memory extents, equal in every block
};

template <typename T, int K, int G>
__global__ void __launch_bounds__(kGsBlock) k_gs_cluster(LevelView<T> L, const T* __restrict__ g, T* dp, GsCluster Q) {
  static_assert(K * G <= 32, "a row group must fit in a warp");
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem[];
  T* s_dp = reinterpret_cast<T*>(smem);
  T* s_g = s_dp + (size_t)Q.win_max * K;
  T* s_dinv = s_g + (size_t)Q.rows_max * K;
  T* s_v = s_dinv + Q.rows_max;
  int* s_rp = reinterpret_cast<int*>(s_v + Q.nnz_max);
  int* s_perm = s_rp + Q.rows_max + 1;
  int* s_ci = s_perm + Q.rows_max;
  int* s_plist = s_ci + Q.nnz_max;
  int* s_poff = s_plist + Q.rows_max;
  constexpr int kGroup = K * G;
  const int k = threadIdx.x % K;
  const int lane = (threadIdx.x / K) % G;
  const unsigned mask = group_mask<kGroup>();
  const int n_p = L.n_p, Ts = Q.T, ncol = Q.ncol;
  const int s0 = min(c * Q.spc, Q.nstrips), s1 = min(s0 + Q.spc, Q.nstrips);
  const int r_lo = min(s0 * Ts, n_p), r_hi = min(s1 * Ts, n_p);
  const int w_lo = max(0, r_lo - Ts), w_hi = min(n_p, r_hi + Ts);
  const int q0 = s1 > s0 ? Q.soff[(size_t)s0 * (ncol + 1)] : 0;
  const int q1 = s1 > s0 ? Q.soff[(size_t)(s1 - 1) * (ncol + 1) + ncol] : 0;
  const int e0 = L.S.rp[q0], e1 = s1 > s0 ? L.S.rp[q1] : e0;
  for (int t = threadIdx.x; t < (w_hi - w_lo) * K; t += blockDim.x) s_dp[t] = T(0);
  if (s1 > s0) {
    stage_copy<false>(s_g, g + (size_t)r_lo * K, (r_hi - r_lo) * K);
    stage_copy<false>(s_dinv, L.S_dinv + q0, q1 - q0);
    stage_copy<false>(s_perm, L.S_perm + q0, q1 - q0);
    stage_copy<false>(s_rp, L.S.rp + q0, q1 - q0 + 1);
    stage_copy<false>(s_v, L.S.v + e0, e1 - e0);
    stage_copy<false>(s_ci, L.S.ci + e0, e1 - e0);
    stage_copy<false>(s_plist, Q.plist + q0, q1 - q0);
  }
  stage_copy<false>(s_poff, Q.poff + (size_t)c * (2 * ncol + 1), 2 * ncol + 1);
  cp_async_wait_all();
  __syncthreads();
  for (int t = threadIdx.x; t < e1 - e0; t += blockDim.x) s_ci[t] -= w_lo;  // window-relative columns
  for (int t = threadIdx.x; t <= q1 - q0; t += blockDim.x) s_rp[t] -= e0;
  for (int t = threadIdx.x; t < q1 - q0; t += blockDim.x) s_plist[t] -= q0;
  // neighbouring strips held by other blocks, and where their windows start
  const bool has_left = s1 > s0 && s0 > 0, has_right = s1 > s0 && s1 < Q.nstrips;
  const T* left_dp = has_left ? cl.map_shared_rank(s_dp, c - 1) : nullptr;
  const T* right_dp = has_right ? cl.map_shared_rank(s_dp, c + 1) : nullptr;
  const int left_wlo = max(0, (s0 - Q.spc) * Ts - Ts);  // block c-1 owns spc strips ending at s0
  const int right_wlo = max(0, s1 * Ts - Ts);
  __syncthreads();
  for (int it = 0; it < Q.iters; ++it)
    for (int par = 0; par < 2; ++par) {
      cl.sync();  // every block finished the previous phase; its rows are visible
      if (has_left && ((s0 - 1) & 1) != par) {
        const int a = (s0 - 1) * Ts, b = min(s0 * Ts, n_p);
        for (int t = threadIdx.x; t < (b - a) * K; t += blockDim.x)
          s_dp[(size_t)(a - w_lo) * K + t] = left_dp[(size_t)(a - left_wlo) * K + t];
      }
      if (has_right && (s1 & 1) != par) {
        const int a = s1 * Ts, b = min((s1 + 1) * Ts, n_p);
        for (int t = threadIdx.x; t < (b - a) * K; t += blockDim.x)
          s_dp[(size_t)(a - w_lo) * K + t] = right_dp[(size_t)(a - right_wlo) * K + t];
      }
      __syncthreads();
      for (int pc = 0; pc < ncol; ++pc) {
        const int a = s_poff[par * ncol + pc], b = s_poff[par * ncol + pc + 1];
        for (int t = threadIdx.x; t < (b - a) * kGroup; t += blockDim.x) {
          const int r = s_plist[a + t / kGroup];
          const int ea = s_rp[r], eb = s_rp[r + 1];
          T a0 = T(0), a1 = T(0);
          int e = ea + lane;
          for (; e + G < eb; e += 2 * G) {
            a0 += s_v[e] * s_dp[(size_t)s_ci[e] * K + k];
            a1 += s_v[e + G] * s_dp[(size_t)s_ci[e + G] * K + k];
          }
          if (e < eb) a0 += s_v[e] * s_dp[(size_t)s_ci[e] * K + k];
          const T acc = group_sum<K, G>(a0 + a1, mask);
          if (lane == 0) {
            const int i = s_perm[r];
            s_dp[(size_t)(i - w_lo) * K + k] = (s_g[(size_t)(i - r_lo) * K + k] - acc) * s_dinv[r];
          }
        }
        __syncthreads();
      }
    }
  cl.sync();  // no block leaves while another may still read its window
  for (int t = threadIdx.x; t < (r_hi - r_lo) * K; t += blockDim.x)
    dp[(size_t)r_lo * K + t] = s_dp[(size_t)(r_lo - w_lo) * K + t];
}

// Dense form of the Gauss-Seidel call on a small level: the gs_iters iterations
// from dp = 0 in the (strip parity, color, index) order are a fixed linear map of
// g, dp = M g, with M (n_p x n_p, row-major, rows padded with zeros to ld, a
// multiple of 16 bytes) formed at setup by the same sweeps.
//
// k_gs_dense_tile (K <= 16): a block of kDenseWarps warps takes kDenseRows rows
// (kDenseRowsPerWarp per warp).  Lane t takes columns t, t + 32, ...: its reads of M
// are coalesced across the warp, and its K values of g are contiguous and adjacent to
// the next lane's, so g (small: it stays in L1) is read coalesced and serves all of
// the warp's rows.  Each step first issues the reads of M for kDenseSteps columns per
// lane, then reads g and accumulates, so the loads of M overlap.  No shared memory and
// no barrier.  Streaming M is the bound (about 71 MB in FP32 for 4225 pressures).
constexpr int kDenseWarps = 4, kDenseRowsPerWarp = 2, kDenseSteps = 16;
constexpr int kDenseRows = kDenseWarps * kDenseRowsPerWarp;
template <typename T, int K>
__global__ void __launch_bounds__(kDenseWarps * 32) k_gs_dense_tile(int n_p, int ld, const T* __restrict__ M,
                                                                    const T* __restrict__ g, T* __restrict__ dp) {
  constexpr int RW = kDenseRowsPerWarp, U = kDenseSteps;
  constexpr int VG = VecWidth<T, K>::V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * kDenseRows + warp * RW;
  if (i0 >= n_p) return;
  const T* Mr[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r) Mr[r] = M + (size_t)min(i0 + r, n_p - 1) * ld;  // rows past n_p: read, unused
  T acc[RW][K];
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[r][k] = T(0);
  for (int jb = lane; jb < n_p; jb += 32 * U) {
    T m[U][RW];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = jb + 32 * u;
#pragma unroll
      for (int r = 0; r < RW; ++r) m[u][r] = j < n_p ? Mr[r][j] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = jb + 32 * u;
      if (j < n_p) {
        const T* gj = g + (size_t)j * K;
#pragma unroll
        for (int k0 = 0; k0 < K; k0 += VG) {
          T gv[VG];
          vld<T, VG>(gv, gj + k0);
#pragma unroll
          for (int w = 0; w < VG; ++w)
#pragma unroll
            for (int r = 0; r < RW; ++r) acc[r][k0 + w] += m[u][r] * gv[w];
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RW; ++r)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      T a = acc[r][k];
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
      if (lane == (r * K + k) % 32 && i0 + r < n_p) dp[(size_t)(i0 + r) * K + k] = a;
    }
}

// k_gs_dense (any K, used for K = 32): one warp per row i, lane (jsplit, k) sums
// M[i, j] g[j, k] over j = jsplit, jsplit + 32/K, ..., then the 32/K partial sums of
// each column are combined.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_gs_dense(int n_p, int ld, const T* __restrict__ M,
                                                     const T* __restrict__ g, T* __restrict__ dp) {
  constexpr int J = 32 / K;  // row entries a column's lanes split
  const int i = (int)(gtid() >> 5);
  if (i >= n_p) return;
  const int lane = threadIdx.x & 31;
  const int k = lane % K, js = lane / K;
  const T* Mi = M + (size_t)i * ld;
  T a0 = T(0), a1 = T(0);
  int j = js;
  for (; j + J < n_p; j += 2 * J) {
    a0 += Mi[j] * g[(size_t)j * K + k];
    a1 += Mi[j + J] * g[(size_t)(j + J) * K + k];
  }
  if (j < n_p) a0 += Mi[j] * g[(size_t)j * K + k];
  T acc = a0 + a1;
#pragma unroll
  for (int off = 16; off >= K; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (js == 0) dp[(size_t)i * K + k] = acc;
}

// Vanka relaxation (Section 5.1) on one color of blocks: one thread block per
// Vanka block.  It gathers the block's residual rows r = f - A x (K columns), then
// adds omega * inv * r to x on the block's dofs, inv the block's local matrix
// inverted at setup; a warp takes one row at a time in both products.  Blocks of one color share no dof and no entry of A, so the
// blocks of a launch neither race nor see each other's updates.
template <typename T>
struct VankaView {
  const int* ptr;           // block b's dofs are dofs[ptr[b] .. ptr[b+1])
  const int* dofs;
  const T* inv;             // block b's inverse, row-major, at inv_off[b]
  const long long* inv_off;
  const int* order;         // blocks sorted by (color, index)
};

// Two forms, picked per level by the autotuner: k_vanka_color_pairs gives each
// thread one (row, column) pair and walks the row itself (small blocks, many per
// color); k_vanka_color gives each warp one row at a time, its lanes splitting the
// row's entries (large blocks, few per color).
template <typename T, int K>
__global__ void __launch_bounds__(128) k_vanka_color_pairs(LevelView<T> L, VankaView<T> V, int first,
                                                           const T* __restrict__ f, T* x, T omega) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int blk = V.order[first + blockIdx.x];
  const int p0 = V.ptr[blk], m = V.ptr[blk + 1] - p0;
  int* s_dof = reinterpret_cast<int*>(smem);
  T* s_r = reinterpret_cast<T*>(smem + ((size_t)m * sizeof(int) + 15) / 16 * 16);
  for (int j = threadIdx.x; j < m; j += blockDim.x) s_dof[j] = V.dofs[p0 + j];
  __syncthreads();
  const int nu = L.dim * L.n_v;
  for (int t = threadIdx.x; t < m * K; t += blockDim.x) {
    const int j = t / K, k = t % K;
    const int q = s_dof[j];
    T acc = T(0);
    if (q < nu) {
      const int c = q / L.n_v, i = q - c * L.n_v;
      const T* xc = x + (size_t)c * L.n_v * K;
      for (int e = L.A.rp[i]; e < L.A.rp[i + 1]; ++e) acc += L.A.v[e] * xc[(size_t)L.A.ci[e] * K + k];
      for (int e = L.Bt.rp[q]; e < L.Bt.rp[q + 1]; ++e) acc += L.Bt.v[e] * x[(size_t)(nu + L.Bt.ci[e]) * K + k];
    } else {
      const int i = q - nu;
      for (int e = L.B.rp[i]; e < L.B.rp[i + 1]; ++e) acc += L.B.v[e] * x[(size_t)L.B.ci[e] * K + k];
      if (i == L.pinned) acc += x[(size_t)q * K + k];
    }
    s_r[t] = f[(size_t)q * K + k] - acc;
  }
  __syncthreads();
  const T* Ib = V.inv + V.inv_off[blk];
  for (int t = threadIdx.x; t < m * K; t += blockDim.x) {
    const int j = t / K, k = t % K;
    const T* row = Ib + (size_t)j * m;
    T a0 = T(0), a1 = T(0);
    int l = 0;
    for (; l + 1 < m; l += 2) {
      a0 += row[l] * s_r[l * K + k];
      a1 += row[l + 1] * s_r[(l + 1) * K + k];
    }
    if (l < m) a0 += row[l] * s_r[l * K + k];
    x[(size_t)s_dof[j] * K + k] += omega * (a0 + a1);
  }
}

template <typename T, int K, int NT>
__global__ void __launch_bounds__(NT) k_vanka_color(LevelView<T> L, VankaView<T> V, int first,
                                                    const T* __restrict__ f, T* x, T omega) {
  // one warp per block row: lane (g, k) takes column k and every GL-th entry of the row from g
  constexpr int GL = K >= 32 ? 1 : 32 / K;
  extern __shared__ __align__(16) unsigned char smem[];
  const int blk = V.order[first + blockIdx.x];
  const int p0 = V.ptr[blk], m = V.ptr[blk + 1] - p0;
  int* s_dof = reinterpret_cast<int*>(smem);
  T* s_r = reinterpret_cast<T*>(smem + ((size_t)m * sizeof(int) + 15) / 16 * 16);
  for (int j = threadIdx.x; j < m; j += blockDim.x) s_dof[j] = V.dofs[p0 + j];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int k = lane % K, g = lane / K;
  const int nu = L.dim * L.n_v;
  for (int j = warp; j < m; j += nwarps) {
    const int q = s_dof[j];
    T acc = T(0);
    if (g < GL) {
      if (q < nu) {
        const int c = q / L.n_v, i = q - c * L.n_v;
        const T* xc = x + (size_t)c * L.n_v * K;
        for (int e = L.A.rp[i] + g; e < L.A.rp[i + 1]; e += GL) acc += L.A.v[e] * xc[(size_t)L.A.ci[e] * K + k];
        for (int e = L.Bt.rp[q] + g; e < L.Bt.rp[q + 1]; e += GL)
          acc += L.Bt.v[e] * x[(size_t)(nu + L.Bt.ci[e]) * K + k];
      } else {
        const int i = q - nu;
        for (int e = L.B.rp[i] + g; e < L.B.rp[i + 1]; e += GL) acc += L.B.v[e] * x[(size_t)L.B.ci[e] * K + k];
        if (i == L.pinned && g == 0) acc += x[(size_t)q * K + k];
      }
    }
#pragma unroll
    for (int off = 16; off >= K; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (g == 0 && k < K) s_r[j * K + k] = f[(size_t)q * K + k] - acc;
  }
  __syncthreads();
  const T* Ib = V.inv + V.inv_off[blk];
  for (int j = warp; j < m; j += nwarps) {
    const T* row = Ib + (size_t)j * m;
    T acc = T(0);
    if (g < GL)
      for (int l = g; l < m; l += GL) acc += row[l] * s_r[l * K + k];
#pragma unroll
    for (int off = 16; off >= K; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (g == 0 && k < K) x[(size_t)s_dof[j] * K + k] += omega * acc;
  }
}

// x = f on the listed (Dirichlet) dofs, all K columns.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_vanka_exact(int n, const int* __restrict__ dofs, const T* __restrict__ f,
                                                       T* __restrict__ x) {
  const long long t = gtid();
  if (t >= (long long)n * K) return;
  const size_t q = (size_t)dofs[t / K] * K + t % K;
  x[q] = f[q];
}

// ILU(1) relaxation (Section 5): x <- x + (L U)^-1 r, the factors' rows and columns
// in the smoother's order (position i holds dof perm[i]).  Each substitution is one
// launch with no grid-wide barrier.  Warps take rows from a ticket counter in
// (dependency level, position) order, so a row only ever waits for rows already
// taken by running warps: no co-residency is needed and any grid size works.  The
// substitution's output is filled with a sentinel (every bit set, a NaN) before the
// launch and the written values are their own signal: a lane polls each value it
// needs until it differs from the sentinel, so a row costs no fence and no flag.
// Values computed from finite data are never NaN; a NaN result that matched the
// sentinel would end in a timed-out wait, reported through *err.  Every wait is
// bounded (the wait_limit polls) and gives up at once when *err is set; a lane that
// gives up takes 0 and goes on, so the launch always ends.  The warp that takes
// the last ticket puts the counter back to zero for the next launch.
constexpr int kIluBlock = 256;
constexpr int kIluChunk = 8;  // entries a lane has in flight at once

template <typename T>
struct IluView {
  int n;
  const int* perm;    // position -> dof
  DCsr<T> L, U;       // strict lower / upper factor rows, columns in positions
  const T* dinv;      // 1 / pivot
  const int* schedL;  // ticket -> row of the forward substitution
  const int* schedU;  // ticket -> row of the backward substitution
};

__device__ __forceinline__ float ld_relaxed(const float* p) {
  float v;
  asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];\n" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_relaxed(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];\n" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
  asm volatile("st.relaxed.gpu.global.f32 [%0], %1;\n" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;\n" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ bool is_sentinel(float v) { return __float_as_uint(v) == 0xffffffffu; }
__device__ __forceinline__ bool is_sentinel(double v) { return __double_as_longlong(v) == -1ll; }

template <typename T>
__device__ __noinline__ T wait_value(const T* p, int* err) {
  T v = ld_relaxed(p);
  const unsigned long long limit = is_sentinel(v) ? wait_limit(err) : 0ull;
  for (unsigned long long spins = 1; is_sentinel(v); ++spins) {
    if (spins > limit || ((spins & 31) == 0 && *(volatile int*)err)) {
      atomicExch(err, 1);
      return T(0);
    }
    if (spins > 128) __nanosleep(64);
    v = ld_relaxed(p);
  }
  return v;
}

// sum over the row's entries of T.v[e] * z[T.ci[e]] for right-hand side k, the
// entries split over the G = 32 / K lane groups, z polled (written by this launch)
template <typename T, int K>
__device__ __forceinline__ T ilu_row_dot(const DCsr<T>& F, int i, const T* z, int k, int g, int* err) {
  constexpr int G = 32 / K;
  T acc = T(0);
  const int e1 = F.rp[i + 1];
  for (int e0 = F.rp[i] + g; e0 < e1; e0 += G * kIluChunk) {
    int j[kIluChunk];
    T a[kIluChunk], v[kIluChunk];
#pragma unroll
    for (int c = 0; c < kIluChunk; ++c) {
      const int e = e0 + c * G;
      j[c] = e < e1 ? F.ci[e] : -1;
      a[c] = e < e1 ? F.v[e] : T(0);
    }
#pragma unroll
    for (int c = 0; c < kIluChunk; ++c) v[c] = j[c] >= 0 ? ld_relaxed(z + (size_t)j[c] * K + k) : T(0);
#pragma unroll
    for (int c = 0; c < kIluChunk; ++c) {
      if (j[c] >= 0 && is_sentinel(v[c])) v[c] = wait_value(z + (size_t)j[c] * K + k, err);
      acc += a[c] * v[c];
    }
  }
#pragma unroll
  for (int o = K; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

__device__ __forceinline__ int ilu_ticket(int* ticket) {
  int t = 0;
  if ((threadIdx.x & 31) == 0) t = atomicAdd(ticket, 1);
  return __shfl_sync(0xffffffffu, t, 0);
}
__device__ __forceinline__ void ilu_release(int* ticket, int t, int n) {
  if ((threadIdx.x & 31) == 0 && t == n + (int)(gridDim.x * (blockDim.x / 32)) - 1) atomicExch(ticket, 0);
}

// forward substitution: y_i = r_{perm i} - sum_{j < i} L_ij y_j (y all sentinel at launch)
template <typename T, int K>
__global__ void __launch_bounds__(kIluBlock) k_ilu_lower(IluView<T> F, const T* __restrict__ r, T* y, int* ticket,
                                                         int* err) {
  static_assert(K >= 1 && K <= 32 && (32 % K) == 0, "K must divide a warp");
  const int lane = threadIdx.x & 31, k = lane % K, g = lane / K;
  for (;;) {
    const int t = ilu_ticket(ticket);
    if (t >= F.n) {
      ilu_release(ticket, t, F.n);
      return;
    }
    const int i = F.schedL[t];
    // the row's own operand first: its load overlaps the waits instead of following them
    const T ri = g == 0 ? r[(size_t)F.perm[i] * K + k] : T(0);
    const T acc = ilu_row_dot<T, K>(F.L, i, y, k, g, err);
    if (g == 0) st_relaxed(y + (size_t)i * K + k, ri - acc);
  }
}

// backward substitution: d_i = (y_i - sum_{j > i} U_ij d_j) / U_ii (d all sentinel at
// launch), then x_{perm i} += d_i (x_{perm i} = d_i when zero is set)
template <typename T, int K>
__global__ void __launch_bounds__(kIluBlock) k_ilu_upper(IluView<T> F, const T* __restrict__ y, T* d, T* x, int zero,
                                                         int* ticket, int* err) {
  const int lane = threadIdx.x & 31, k = lane % K, g = lane / K;
  for (;;) {
    const int t = ilu_ticket(ticket);
    if (t >= F.n) {
      ilu_release(ticket, t, F.n);
      return;
    }
    const int i = F.schedU[t];
    // the row's own operands first (overlapping the waits)
    T yi = T(0), dv = T(0), xq = T(0);
    size_t q = 0;
    if (g == 0) {
      yi = y[(size_t)i * K + k];
      dv = F.dinv[i];
      q = (size_t)F.perm[i] * K + k;
      if (!zero) xq = x[q];
    }
    const T acc = ilu_row_dot<T, K>(F.U, i, d, k, g, err);
    if (g == 0) {
      const T di = (yi - acc) * dv;
      st_relaxed(d + (size_t)i * K + k, di);
      x[q] = xq + di;
    }
  }
}

// Single-block Gauss-Seidel for a small level, same ordering: the whole level's
// S, g, 1/S_ii and dp sit in shared memory and the (parity, color) groups run one
// after another separated by __syncthreads, with no inter-block waits.
// plist holds the sorted rows of each (parity, color) group, poff its offsets.
template <typename T, int K, int G>
__global__ void __launch_bounds__(kGsBlock) k_gs_level(LevelView<T> L, const T* __restrict__ g, T* dp,
                                                       const int* __restrict__ plist, const int* __restrict__ poff,
                                                       int ncol, int iters) {
  static_assert(K * G <= 32, "a row group must fit in a warp");
  extern __shared__ __align__(16) unsigned char smem[];
  const int n_p = L.n_p;
  const int nnz = L.S.rp[n_p];
  T* s_dp = reinterpret_cast<T*>(smem);
  T* s_g = s_dp + (size_t)n_p * K;
  T* s_dinv = s_g + (size_t)n_p * K;
  T* s_v = s_dinv + n_p;
  int* s_rp = reinterpret_cast<int*>(s_v + nnz);
  int* s_ci = s_rp + n_p + 1;
  int* s_perm = s_ci + nnz;
  int* s_plist = s_perm + n_p;
  int* s_poff = s_plist + n_p;
  constexpr int kGroup = K * G;
  const int k = threadIdx.x % K;
  const int lane = (threadIdx.x / K) % G;
  const unsigned mask = group_mask<kGroup>();
  for (int t = threadIdx.x; t < n_p * K; t += blockDim.x) s_dp[t] = T(0);
  stage_copy<false>(s_g, g, n_p * K);
  stage_copy<false>(s_dinv, L.S_dinv, n_p);
  stage_copy<false>(s_v, L.S.v, nnz);
  stage_copy<false>(s_rp, L.S.rp, n_p + 1);
  stage_copy<false>(s_ci, L.S.ci, nnz);
  stage_copy<false>(s_perm, L.S_perm, n_p);
  stage_copy<false>(s_plist, plist, n_p);
  stage_copy<false>(s_poff, poff, 2 * ncol + 1);
  cp_async_wait_all();
  __syncthreads();
  for (int it = 0; it < iters; ++it)
    for (int grp = 0; grp < 2 * ncol; ++grp) {
      const int a = s_poff[grp], b = s_poff[grp + 1];
      for (int t = threadIdx.x; t < (b - a) * kGroup; t += blockDim.x) {
        const int r = s_plist[a + t / kGroup];
        const int ea = s_rp[r], eb = s_rp[r + 1];
        T a0 = T(0), a1 = T(0);
        int e = ea + lane;
        for (; e + G < eb; e += 2 * G) {
          a0 += s_v[e] * s_dp[(size_t)s_ci[e] * K + k];
          a1 += s_v[e + G] * s_dp[(size_t)s_ci[e + G] * K + k];
        }
        if (e < eb) a0 += s_v[e] * s_dp[(size_t)s_ci[e] * K + k];
        const T acc = group_sum<K, G>(a0 + a1, mask);
        if (lane == 0) {
          const int i = s_perm[r];
          s_dp[(size_t)i * K + k] = (s_g[(size_t)i * K + k] - acc) * s_dinv[r];
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < n_p * K; t += blockDim.x) dp[t] = s_dp[t];
}

// u = y - w .* (Bt dp), p = p + dp (p = dp with zero_x): the velocity/pressure update.
template <typename T, int K, int G, int V>
__global__ void __launch_bounds__(kBlock) k_bs_update(LevelView<T> L, const T* __restrict__ y,
                                                      const T* __restrict__ dp, T* __restrict__ x, int zero_x) {
  using M = RowMap<K, G, V>;
  const M q(gtid());
  const unsigned i = q.row, k0 = q.k0;
  const unsigned nvK = (unsigned)L.n_v * K, nuK = (unsigned)L.dim * nvK;
  if (i < (unsigned)L.n_v) {
    T sum[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int u = 0; u < V; ++u) sum[c][u] = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const unsigned r = c * L.n_v + i;
        for (int e = L.Bt.rp[r] + q.lane; e < L.Bt.rp[r + 1]; e += G) {
          const T bv = L.Bt.v[e];
          T dv[V];
          vld<T, V>(dv, dp + (unsigned)L.Bt.ci[e] * K + k0);
#pragma unroll
          for (int u = 0; u < V; ++u) sum[c][u] += bv * dv[u];
        }
      }
    if constexpr (G > 1) {
      const unsigned mask = group_mask<M::W>();
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int u = 0; u < V; ++u) sum[c][u] = group_sum<M::KV, G>(sum[c][u], mask);
    }
    if (q.lane != 0) return;
    const T wi = L.w[i];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const unsigned o = c * nvK + i * K + k0;
        T yv[V], out[V];
        vld<T, V>(yv, y + o);
#pragma unroll
        for (int u = 0; u < V; ++u) out[u] = yv[u] - wi * sum[c][u];
        vst<T, V>(x + o, out);
      }
  } else if (i < (unsigned)(L.n_v + L.n_p) && q.lane == 0) {
    const unsigned p = i - L.n_v;
    const unsigned o = nuK + p * K + k0;
    T xv[V], dv[V], out[V];
    vld<T, V>(dv, dp + p * K + k0);
    if (!zero_x) vld<T, V>(xv, x + o);
#pragma unroll
    for (int u = 0; u < V; ++u) out[u] = (zero_x ? T(0) : xv[u]) + dv[u];
    vst<T, V>(x + o, out);
  }
}

// out = b - A x (HAS_B) or out = A x, for the whole block matrix [I(x)A, Bt; B, C].
template <typename T, int K, int G, int V, bool HAS_B>
__global__ void __launch_bounds__(kBlock) k_block_spmv(LevelView<T> L, const T* __restrict__ b,
                                                       const T* __restrict__ x, T* __restrict__ out) {
  using M = RowMap<K, G, V>;
  const M q(gtid());
  const unsigned i = q.row, k0 = q.k0;
  const unsigned nvK = (unsigned)L.n_v * K, nuK = (unsigned)L.dim * nvK;
  const unsigned mask = group_mask<M::W>();
  if (i < (unsigned)L.n_v) {
    T acc[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int u = 0; u < V; ++u) acc[c][u] = T(0);
    for (int e = L.A.rp[i] + q.lane; e < L.A.rp[i + 1]; e += G) {
      const T a = L.A.v[e];
      const unsigned j = (unsigned)L.A.ci[e] * K + k0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < L.dim) {
          T xv[V];
          vld<T, V>(xv, x + c * nvK + j);
#pragma unroll
          for (int u = 0; u < V; ++u) acc[c][u] += a * xv[u];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const unsigned r = c * L.n_v + i;
        for (int e = L.Bt.rp[r] + q.lane; e < L.Bt.rp[r + 1]; e += G) {
          const T bv = L.Bt.v[e];
          T xv[V];
          vld<T, V>(xv, x + nuK + (unsigned)L.Bt.ci[e] * K + k0);
#pragma unroll
          for (int u = 0; u < V; ++u) acc[c][u] += bv * xv[u];
        }
      }
    if constexpr (G > 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int u = 0; u < V; ++u) acc[c][u] = group_sum<M::KV, G>(acc[c][u], mask);
    }
    if (q.lane != 0) return;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const unsigned o = c * nvK + i * K + k0;
        T r[V];
        if (HAS_B) {
          T bv[V];
          vld<T, V>(bv, b + o);
#pragma unroll
          for (int u = 0; u < V; ++u) r[u] = bv[u] - acc[c][u];
        } else {
#pragma unroll
          for (int u = 0; u < V; ++u) r[u] = acc[c][u];
        }
        vst<T, V>(out + o, r);
      }
  } else if (i < (unsigned)(L.n_v + L.n_p)) {
    const unsigned p = i - L.n_v;
    T acc[V];
#pragma unroll
    for (int u = 0; u < V; ++u) acc[u] = T(0);
    for (int e = L.B.rp[p] + q.lane; e < L.B.rp[p + 1]; e += G) {
      const T bv = L.B.v[e];
      T xv[V];
      vld<T, V>(xv, x + (unsigned)L.B.ci[e] * K + k0);
#pragma unroll
      for (int u = 0; u < V; ++u) acc[u] += bv * xv[u];
    }
    if constexpr (G > 1) {
#pragma unroll
      for (int u = 0; u < V; ++u) acc[u] = group_sum<M::KV, G>(acc[u], mask);
    }
    if (q.lane != 0) return;
    const unsigned o = nuK + p * K + k0;
    if ((int)p == L.pinned) {
      T xv[V];
      vld<T, V>(xv, x + o);
#pragma unroll
      for (int u = 0; u < V; ++u) acc[u] += xv[u];
    }
    T r[V];
    if (HAS_B) {
      T bv[V];
      vld<T, V>(bv, b + o);
#pragma unroll
      for (int u = 0; u < V; ++u) r[u] = bv[u] - acc[u];
    } else {
#pragma unroll
      for (int u = 0; u < V; ++u) r[u] = acc[u];
    }
    vst<T, V>(out + o, r);
  }
}

// b_c = R r: velocity rows by R (each component), pressure rows by Rp.
template <typename T, int K, int G, int V>
__global__ void __launch_bounds__(kBlock) k_restrict(LevelView<T> L, const T* __restrict__ r, T* __restrict__ bc) {
  using M = RowMap<K, G, V>;
  const M q(gtid());
  const unsigned I = q.row, k0 = q.k0;
  const unsigned mask = group_mask<M::W>();
  const unsigned nvK = (unsigned)L.n_v * K;
  if (I < (unsigned)L.n_vc) {
    T s[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int u = 0; u < V; ++u) s[c][u] = T(0);
    for (int e = L.R.rp[I] + q.lane; e < L.R.rp[I + 1]; e += G) {
      const T v = L.R.v[e];
      const unsigned j = (unsigned)L.R.ci[e] * K + k0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < L.dim) {
          T rv[V];
          vld<T, V>(rv, r + c * nvK + j);
#pragma unroll
          for (int u = 0; u < V; ++u) s[c][u] += v * rv[u];
        }
    }
    if constexpr (G > 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int u = 0; u < V; ++u) s[c][u] = group_sum<M::KV, G>(s[c][u], mask);
    }
    if (q.lane != 0) return;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) vst<T, V>(bc + ((unsigned)c * L.n_vc + I) * K + k0, s[c]);
  } else if (I < (unsigned)(L.n_vc + L.n_pc)) {
    const unsigned p = I - L.n_vc;
    const unsigned nuK = (unsigned)L.dim * nvK;
    T s[V];
#pragma unroll
    for (int u = 0; u < V; ++u) s[u] = T(0);
    for (int e = L.Rp.rp[p] + q.lane; e < L.Rp.rp[p + 1]; e += G) {
      const T v = L.Rp.v[e];
      T rv[V];
      vld<T, V>(rv, r + nuK + (unsigned)L.Rp.ci[e] * K + k0);
#pragma unroll
      for (int u = 0; u < V; ++u) s[u] += v * rv[u];
    }
    if constexpr (G > 1) {
#pragma unroll
      for (int u = 0; u < V; ++u) s[u] = group_sum<M::KV, G>(s[u], mask);
    }
    if (q.lane != 0) return;
    vst<T, V>(bc + ((unsigned)L.dim * L.n_vc + p) * K + k0, s);
  }
}

// x += P x_c: velocity rows by P (each component), pressure rows by Pp.
template <typename T, int K, int G, int V>
__global__ void __launch_bounds__(kBlock) k_prolong(LevelView<T> L, const T* __restrict__ xc, T* __restrict__ x) {
  using M = RowMap<K, G, V>;
  const M q(gtid());
  const unsigned i = q.row, k0 = q.k0;
  const unsigned mask = group_mask<M::W>();
  const unsigned ncK = (unsigned)L.n_vc * K;
  if (i < (unsigned)L.n_v) {
    T s[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int u = 0; u < V; ++u) s[c][u] = T(0);
    for (int e = L.P.rp[i] + q.lane; e < L.P.rp[i + 1]; e += G) {
      const T v = L.P.v[e];
      const unsigned j = (unsigned)L.P.ci[e] * K + k0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < L.dim) {
          T cv[V];
          vld<T, V>(cv, xc + c * ncK + j);
#pragma unroll
          for (int u = 0; u < V; ++u) s[c][u] += v * cv[u];
        }
    }
    if constexpr (G > 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int u = 0; u < V; ++u) s[c][u] = group_sum<M::KV, G>(s[c][u], mask);
    }
    if (q.lane != 0) return;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const unsigned o = ((unsigned)c * L.n_v + i) * K + k0;
        T xv[V];
        vld<T, V>(xv, x + o);
#pragma unroll
        for (int u = 0; u < V; ++u) xv[u] += s[c][u];
        vst<T, V>(x + o, xv);
      }
  } else if (i < (unsigned)(L.n_v + L.n_p)) {
    const unsigned p = i - L.n_v;
    T s[V];
#pragma unroll
    for (int u = 0; u < V; ++u) s[u] = T(0);
    for (int e = L.Pp.rp[p] + q.lane; e < L.Pp.rp[p + 1]; e += G) {
      const T v = L.Pp.v[e];
      T cv[V];
      vld<T, V>(cv, xc + (unsigned)L.dim * ncK + (unsigned)L.Pp.ci[e] * K + k0);
#pragma unroll
      for (int u = 0; u < V; ++u) s[u] += v * cv[u];
    }
    if constexpr (G > 1) {
#pragma unroll
      for (int u = 0; u < V; ++u) s[u] = group_sum<M::KV, G>(s[u], mask);
    }
    if (q.lane != 0) return;
    const unsigned o = ((unsigned)L.dim * L.n_v + p) * K + k0;
    T xv[V];
    vld<T, V>(xv, x + o);
#pragma unroll
    for (int u = 0; u < V; ++u) xv[u] += s[u];
    vst<T, V>(x + o, xv);
  }
}

// Block product in float-float arithmetic: out = A z for an FP32 vector z and the
// FP64 matrix split as a = hi + lo (two floats).  hi*z is formed exactly as
// p + e (e = fma(hi, z, -p)), lo*z in FP32 (its rounding is 2^-24 of a term
// already 2^-24 of a*z), and the sum is carried as a float-float pair with
// Knuth's two-sum, so the result matches FP64 to about 2^-44 relative to
// sum |a z| while using only FP32 instructions.
struct FFMat {
  const int* rp;
  const int* ci;
  const float* hi;
  const float* lo;
};
struct FFLevel {
  int dim, n_v, n_p, pinned;
  FFMat A, B, Bt;
};

struct FFAcc {
  float s, c;
  __device__ __forceinline__ void add(float a, float z) {
    const float p = a * z;
    const float e = fmaf(a, z, -p);
    const float t = s + p;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (p - bp);
    s = t;
    c += err + e;
  }
  __device__ __forceinline__ void add_small(float a, float z) { c = fmaf(a, z, c); }
};

// Sum of two float-float accumulators (two-sum of the leading parts).
__device__ __forceinline__ void ff_merge(FFAcc& a, float s2, float c2) {
  const float t = a.s + s2;
  const float bp = t - a.s;
  const float err = (a.s - (t - bp)) + (s2 - bp);
  a.s = t;
  a.c += c2 + err;
}

// G lanes per row (small problems: G = 4 keeps more gathers in flight per row), their
// float-float partial sums merged by shuffles at the end.
template <int K, int G, int V>
__global__ void __launch_bounds__(kBlock) k_block_spmv_ff(FFLevel L, const float* __restrict__ z,
                                                          double* __restrict__ out) {
  using M = RowMap<K, G, V>;
  const M q(gtid());
  const unsigned i = q.row, k0 = q.k0;
  const unsigned nvK = (unsigned)L.n_v * K, nuK = (unsigned)L.dim * nvK;
  auto merge = [&](FFAcc& a) {
    if constexpr (G > 1) {
      const unsigned mask = group_mask<M::W>();
#pragma unroll
      for (int off = G / 2; off >= 1; off >>= 1) {
        const float s2 = __shfl_xor_sync(mask, a.s, off * M::KV);
        const float c2 = __shfl_xor_sync(mask, a.c, off * M::KV);
        ff_merge(a, s2, c2);
      }
    }
  };
  if (i < (unsigned)L.n_v) {
    FFAcc acc[3][V];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int u = 0; u < V; ++u) acc[c][u] = {0.f, 0.f};
    for (int e = L.A.rp[i] + q.lane; e < L.A.rp[i + 1]; e += G) {
      const float h = L.A.hi[e], l = L.A.lo[e];
      const unsigned j = (unsigned)L.A.ci[e] * K + k0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < L.dim) {
          float zv[V];
          vld<float, V>(zv, z + c * nvK + j);
#pragma unroll
          for (int u = 0; u < V; ++u) {
            acc[c][u].add(h, zv[u]);
            acc[c][u].add_small(l, zv[u]);
          }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < L.dim) {
        const unsigned r = c * L.n_v + i;
        for (int e = L.Bt.rp[r] + q.lane; e < L.Bt.rp[r + 1]; e += G) {
          const float h = L.Bt.hi[e], l = L.Bt.lo[e];
          float zv[V];
          vld<float, V>(zv, z + nuK + (unsigned)L.Bt.ci[e] * K + k0);
#pragma unroll
          for (int u = 0; u < V; ++u) {
            acc[c][u].add(h, zv[u]);
            acc[c][u].add_small(l, zv[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < V; ++u) merge(acc[c][u]);
        if (q.lane == 0) {
          const unsigned o = c * nvK + i * K + k0;
#pragma unroll
          for (int u = 0; u < V; ++u) out[o + u] = (double)acc[c][u].s + (double)acc[c][u].c;
        }
      }
  } else if (i < (unsigned)(L.n_v + L.n_p)) {
    const unsigned p = i - L.n_v;
    FFAcc acc[V];
#pragma unroll
    for (int u = 0; u < V; ++u) acc[u] = {0.f, 0.f};
    for (int e = L.B.rp[p] + q.lane; e < L.B.rp[p + 1]; e += G) {
      const float h = L.B.hi[e], l = L.B.lo[e];
      float zv[V];
      vld<float, V>(zv, z + (unsigned)L.B.ci[e] * K + k0);
#pragma unroll
      for (int u = 0; u < V; ++u) {
        acc[u].add(h, zv[u]);
        acc[u].add_small(l, zv[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < V; ++u) merge(acc[u]);
    if (q.lane != 0) return;
    const unsigned o = nuK + p * K + k0;
#pragma unroll
    for (int u = 0; u < V; ++u) {
      double v = (double)acc[u].s + (double)acc[u].c;
      if ((int)p == L.pinned) v += (double)z[o + u];
      out[o + u] = v;
    }
  }
}

// Coarsest level: x = A^+ b with the FP64 pseudo-inverse, whatever T is.  One warp
// per row: the lanes split the row's columns (so the FP64 work of a row spreads over
// the SMs, not over one thread), then a shuffle tree per right-hand side.
template <typename T, int K>
__global__ void __launch_bounds__(kBlock) k_coarse_solve(int Nc, const double* __restrict__ pinv,
                                                         const T* __restrict__ b, T* __restrict__ x) {
  const long long i = gtid() >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= Nc) return;
  const double* row = pinv + (size_t)i * Nc;
  double s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.0;
  for (int j = lane; j < Nc; j += 32) {
    const double a = row[j];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] += a * (double)b[(size_t)j * K + k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], off);
    if (lane == k) x[(size_t)i * K + k] = (T)s[k];
  }
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

// Columns [col0, col0 + ncols) of dst (N x K) = src (N x ncols); other columns untouched.
template <int K>
__global__ void __launch_bounds__(kBlock) k_pack_cols(long long N, const double* __restrict__ src, int ncols,
                                                      double* __restrict__ dst, int col0) {
  const long long t = gtid();
  if (t >= N * ncols) return;
  const long long i = t / ncols;
  const int k = (int)(t % ncols);
  dst[i * K + col0 + k] = src[t];
}

// dst (N x ncols) = columns [col0, col0 + ncols) of src (N x K).
template <int K>
__global__ void __launch_bounds__(kBlock) k_unpack_cols(long long N, const double* __restrict__ src, int col0,
                                                        int ncols, double* __restrict__ dst) {
  const long long t = gtid();
  if (t >= N * ncols) return;
  const long long i = t / ncols;
  const int k = (int)(t % ncols);
  dst[t] = src[i * K + col0 + k];
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

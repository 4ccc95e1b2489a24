// recursion.cuh - device side of the pure-spectrum / partial-bicoherence
// recursion (Eq. pure): one pass over the lattice as a persistent
// cooperative kernel.  Included by plan.cu only.
#pragma once

#include <cuda/atomic>

#include "srm3_internal.cuh"

namespace srm3 {

// Rows of one work item: a point's row pairs (a, kk - a), a <= kk/2, are
// taken kRecRows at a time by one warp.
constexpr int kRecRows = 4;
constexpr int kRecThreads = 512;  // one CTA per SM
constexpr int kBarSlots0 = 32;    // first arrival slot of the grid barrier

struct RecArgs {
  int nk, nw, nlev, maxch, maxpts;
  long long nl;
  const int2 *items;    // (kk, chunk) of every level, level by level
  const int *lev_off;   // first item of each level
  const double *S;
  void *q;              // [nl][M] of T: q = S/S_p (0 where S = 0), plane fastest
  double *sb2;          // [M][nl]
  const void *G2;       // T[nk][nw]: g^2 = EkSq[|ik-jk|] EwSq[|iw-jw|]
  const double *scal;   // [M]: eps^2 dk dw per plane
  void *partial;        // [maxpts][maxch][M] of T
  unsigned int *ticket; // [maxpts]
  int *err;             // [M]: some S_p <= 0 on this plane
  unsigned int *bar;    // [0] release generation, [kBarSlots0 + b] arrival of CTA b
  unsigned int gen_base;  // generation of this launch's first barrier
  int *abort;           // barrier wait timed out
};

// Grid-wide barrier for a cooperative launch (all CTAs resident), without
// atomics: CTA b stores the barrier's generation number g in its own slot
// bar[kBarSlots0 + b]; warp 0 of CTA 0 polls every slot until all show g,
// then stores g into the release word bar[0], which the other CTAs poll.
// Generations never repeat across launches (the host advances the base),
// so a slot left over from an earlier pass cannot pass for an arrival.  The
// fences on both sides order every CTA's writes before the barrier with
// every read after it.  Waits are bounded: past ~2^22 polls a CTA raises
// *abort and every CTA returns false from this or its next barrier.
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, int *abort, unsigned int g) {
  __shared__ int s_ok;
  const long long limit = 1ll << 22;
  volatile unsigned int *vb = bar;
  volatile int *vab = abort;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    vb[kBarSlots0 + blockIdx.x] = g;
  }
  if (blockIdx.x == 0) {
    if (threadIdx.x < 32) {
      // each round reads all of this lane's slots with independent loads
      bool ok = true;
      long long spins = 0;
      for (;;) {
        bool mine = true;
        for (unsigned int i = threadIdx.x; i < gridDim.x; i += 32)
          mine &= vb[kBarSlots0 + i] == g;
        if (__all_sync(0xffffffffu, mine)) break;
        if (*vab || ++spins > limit) {
          ok = false;
          break;
        }
      }
      if (!__all_sync(0xffffffffu, ok)) {
        if (threadIdx.x == 0) atomicExch(abort, 1);
      } else if (threadIdx.x == 0) {
        __threadfence();
        vb[0] = g;
      }
    }
  } else if (threadIdx.x == 0) {
    long long spins = 0;
    while (vb[0] != g) {
      if (*vab) break;
      if (++spins > limit) {
        atomicExch(abort, 1);
        break;
      }
      __nanosleep(20);
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_ok = *vab == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T, int M>
struct PlaneVec;
template <>
struct PlaneVec<double, 1> {
  static __device__ __forceinline__ void load(const double *p, double (&v)[1]) { v[0] = *p; }
};
template <>
struct PlaneVec<double, 3> {
  static __device__ __forceinline__ void load(const double *p, double (&v)[3]) {
    v[0] = p[0];
    v[1] = p[1];
    v[2] = p[2];
  }
};
template <>
struct PlaneVec<float, 8> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[8]) {
    const float4 a = reinterpret_cast<const float4 *>(p)[0];
    const float4 b = reinterpret_cast<const float4 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
};

// One recursion pass over all anti-diagonal levels d = kk + kw.  Every part
// of a pair of Pi(k) lies on a lower level, so the points of a level are
// independent; the kernel walks the levels in order with a grid barrier in
// between.  A work item is one warp on up to kRecRows row pairs (a, kk - a)
// of one point: the rows' omega ranges are laid end to end and the lanes
// stride over the joined range with four independent accumulators.
// Canonical half: the centre row a = kk - a keeps iw <= kw/2; i = 0 is
// skipped.  Per plane m (one eps value each)
//   sum_b2(k) = eps_m^2 dk dw sum_{Pi(k)} g^2 q_i q_j,  q_k = 1/(1 - sum_b2)
// (b_p^2 = eps^2 g^2 dk dw q_i q_j for |B| = eps g sqrt(S_i S_j S_k)).
// Items of a point write their sums to scratch slots; the last to take the
// point's ticket (acq_rel atomic) adds the slots in chunk order, so results
// do not depend on scheduling.  T = double, M = 1 is the exact pass;
// T = float, M = 8 evaluates eight eps values at once to locate eps.
template <typename T, int M>
__global__ void __launch_bounds__(kRecThreads) k_rec_pass(RecArgs A) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const T *G2 = static_cast<const T *>(A.G2);
  T *q = static_cast<T *>(A.q);
  const int nw = A.nw;
  constexpr int UNR = 4;  // independent accumulators per lane
  // the first item of the next level (items and S are read-only, so they
  // are fetched before the barrier that ends the current level)
  int2 nx_it = make_int2(0, 0);
  double nx_S = 0.0;
  int nx_ok = 0;
  {
    const int i0 = A.lev_off[0], n = A.lev_off[1] - i0;
    if (gw < n) {
      nx_it = A.items[i0 + gw];
      nx_S = A.S[(long long)nx_it.x * nw + (0 - nx_it.x)];
      nx_ok = 1;
    }
  }
  for (int d = 0; d < A.nlev; ++d) {
    const int lo = max(0, d - nw + 1);
    const int i0 = A.lev_off[d], n = A.lev_off[d + 1] - i0;
    for (int w = gw; w < n; w += nwarps) {
      int2 it;
      double Sk;
      if (w == gw && nx_ok) {
        it = nx_it;
        Sk = nx_S;
      } else {
        it = A.items[i0 + w];
        Sk = A.S[(long long)it.x * nw + (d - it.x)];
      }
      const int kk = it.x, c = it.y, kw = d - kk;
      const long long k = (long long)kk * nw + kw;
      if (!(Sk > 0.0)) {
        if (c == 0 && lane < M) {
          A.sb2[lane * A.nl + k] = 0.0;
          q[k * M + lane] = (T)0;
        }
        continue;
      }
      const int nrow = kk / 2 + 1;
      const int nch = (nrow + kRecRows - 1) / kRecRows;
      const int a0 = c * kRecRows;
      // the item's rows laid end to end: row r covers [P[r], P[r+1])
      int lo_r[kRecRows], P[kRecRows + 1];
      P[0] = 0;
#pragma unroll
      for (int r = 0; r < kRecRows; ++r) {
        const int a = a0 + r;
        int len = 0;
        lo_r[r] = (a == 0) ? 1 : 0;  // i = 0 takes part in no pair
        if (a < nrow) {
          const int lim = (a == kk - a) ? kw / 2 : kw;
          len = max(0, lim - lo_r[r] + 1);
        }
        P[r + 1] = P[r] + len;
      }
      const int E = P[kRecRows];
      T acc[UNR][M];
#pragma unroll
      for (int j = 0; j < UNR; ++j)
#pragma unroll
        for (int m = 0; m < M; ++m) acc[j][m] = (T)0;
      for (int e0 = lane; e0 < E; e0 += 32 * UNR) {
#pragma unroll
        for (int j = 0; j < UNR; ++j) {
          const int e = e0 + 32 * j;
          if (e < E) {
            const int r = (e >= P[1]) + (e >= P[2]) + (e >= P[3]);
            const int a = a0 + r;
            const int pr = r == 0 ? P[0] : r == 1 ? P[1] : r == 2 ? P[2] : P[3];
            const int lr = r == 0 ? lo_r[0] : r == 1 ? lo_r[1] : r == 2 ? lo_r[2] : lo_r[3];
            const int iw = lr + (e - pr);
            const int dd = 2 * iw - kw;
            const T g2 = G2[(size_t)(kk - 2 * a) * nw + (dd < 0 ? -dd : dd)];
            T va[M], vb[M];
            PlaneVec<T, M>::load(q + ((size_t)a * nw + iw) * M, va);
            PlaneVec<T, M>::load(q + ((size_t)(kk - a) * nw + (kw - iw)) * M, vb);
#pragma unroll
            for (int m = 0; m < M; ++m) acc[j][m] = fma(g2, va[m] * vb[m], acc[j][m]);
          }
        }
      }
      T t[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        t[m] = (T)0;
#pragma unroll
        for (int j = 0; j < UNR; ++j) t[m] += acc[j][m];
        for (int o = 16; o > 0; o >>= 1) t[m] += __shfl_xor_sync(0xffffffffu, t[m], o);
      }
      if (lane == 0) {
        bool fin = true;
        if (nch > 1) {
          const int slot = kk - lo;
          volatile T *ps = static_cast<T *>(A.partial) + ((size_t)slot * A.maxch) * M;
#pragma unroll
          for (int m = 0; m < M; ++m) ps[c * M + m] = t[m];
          cuda::atomic_ref<unsigned int, cuda::thread_scope_device> tk(A.ticket[slot]);
          fin = tk.fetch_add(1u, cuda::memory_order_acq_rel) == (unsigned int)(nch - 1);
          if (fin) {
#pragma unroll
            for (int m = 0; m < M; ++m) t[m] = (T)0;
            for (int j = 0; j < nch; ++j)
#pragma unroll
              for (int m = 0; m < M; ++m) t[m] += ps[j * M + m];
            tk.store(0u, cuda::memory_order_relaxed);
          }
        }
        if (fin) {
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const T s2 = (T)A.scal[m] * t[m];
            A.sb2[m * A.nl + k] = (double)s2;
            if (s2 < (T)1) {
              q[k * M + m] = (T)1 / ((T)1 - s2);
            } else {
              q[k * M + m] = (T)0;
              atomicOr(A.err + m, 1);
            }
          }
        }
      }
    }
    if (d + 1 < A.nlev) {
      const int j0 = A.lev_off[d + 1], m1 = A.lev_off[d + 2] - j0;
      nx_ok = gw < m1;
      if (nx_ok) {
        nx_it = A.items[j0 + gw];
        nx_S = A.S[(long long)nx_it.x * nw + (d + 1 - nx_it.x)];
      }
    }
    if (!grid_barrier(A.bar, A.abort, A.gen_base + (unsigned int)d)) return;
  }
}

}  // namespace srm3

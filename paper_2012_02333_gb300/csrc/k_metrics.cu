// Distances between distributions (Eq. 16) and sampling from them.
//
// k_distance: chi^2 = sum_i (a_i - b_i)^2 / (a_i + b_i) (Eq. 16; a term with
//   a_i + b_i = 0 counts 0) and the total variation (1/2) sum_i |a_i - b_i|, in
//   one streaming pass.  FP32 inputs: each term in FP32, summed in compensated
//   FP32 (TwoSum) per thread and across the block; FP64 inputs in FP64.  Every
//   block writes its two partial sums; the block that finishes last adds them
//   in block order in FP64, so the result does not depend on scheduling.
// k_sample_chunks / k_sample_scan / k_sample_draw: inverse-transform sampling.
//   Weights w_i = max(p_i, 0) (negative entries are rounding residue and get
//   no weight).  The weights are cut into chunks of 1024 and the chunks into
//   tiles of 1024; a warp sums each chunk (compensated FP32, or FP64) and
//   each tile of chunk sums (FP64); one block scans the tile sums, and a warp
//   per tile turns them into the exclusive FP64 prefix of every chunk.  One
//   warp per draw takes t = u * total, finds the chunk by binary search over
//   the chunk prefixes, the lane of 32 weights by a warp scan and the outcome
//   by a scan of the lane's 32 weights: the first index whose running sum
//   exceeds what is left of t.  An
//   outcome with no weight is never drawn: where rounding leaves t past a
//   chunk's or lane's end, the last weighted index before it is taken; when no
//   outcome has weight every draw is -1.
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.h"

namespace cutqc {

namespace {

struct FF {
  float s, c;
};
__device__ __forceinline__ FF ff_add(FF a, float b) {
  const float s = a.s + b;
  const float bb = s - a.s;
  const float err = (a.s - (s - bb)) + (b - bb);
  return {s, a.c + err};
}
__device__ __forceinline__ FF ff_merge(FF a, FF b) {
  FF r = ff_add(a, b.s);
  r.c += b.c;
  return r;
}
__device__ __forceinline__ double ff_value(FF a) { return (double)a.s + (double)a.c; }

constexpr int DIST_BLOCKS = 152 * 8;
constexpr int CH = 1024;   // weights per chunk

template <typename T>
struct Acc {
  using type = typename std::conditional<sizeof(T) == 8, double, FF>::type;
};

template <typename T>
__device__ __forceinline__ void dist_term(T a, T b, typename Acc<T>::type& chi, typename Acc<T>::type& tv) {
  const T d = a - b, s = a + b;
  T c;
  if constexpr (sizeof(T) == 8)
    c = s != 0.0 ? d * d / s : 0.0;
  else
    c = s != 0.0f ? __fdividef(d * d, s) : 0.0f;   // within 2 ulp; the term is a summand
  if constexpr (sizeof(T) == 8) {
    chi += c;
    tv += fabs(d);
  } else {
    chi = ff_add(chi, c);
    tv = ff_add(tv, fabsf(d));
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_distance(const T* __restrict__ a, const T* __restrict__ b, int64_t n,
                                                  double* __restrict__ part, unsigned* __restrict__ counter,
                                                  double* __restrict__ chi2, double* __restrict__ tv_out) {
  using A = typename Acc<T>::type;
  A chi{}, tv{};
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const bool vec = sizeof(T) == 4 && (n % 4) == 0 && (reinterpret_cast<uintptr_t>(a) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(b) & 15) == 0;
  if constexpr (sizeof(T) == 4) {
    if (vec) {
      const float4* a4 = reinterpret_cast<const float4*>(a);
      const float4* b4 = reinterpret_cast<const float4*>(b);
      // two float4 of each input per step into two independent accumulator pairs
      A chi2_{}, tv2_{};
      const int64_t n4 = n / 4;
      int64_t i = tid;
      for (; i + nth < n4; i += 2 * nth) {
        const float4 x = __ldcs(a4 + i), y = __ldcs(b4 + i);
        const float4 x2 = __ldcs(a4 + i + nth), y2 = __ldcs(b4 + i + nth);
        dist_term<float>(x.x, y.x, chi, tv);
        dist_term<float>(x2.x, y2.x, chi2_, tv2_);
        dist_term<float>(x.y, y.y, chi, tv);
        dist_term<float>(x2.y, y2.y, chi2_, tv2_);
        dist_term<float>(x.z, y.z, chi, tv);
        dist_term<float>(x2.z, y2.z, chi2_, tv2_);
        dist_term<float>(x.w, y.w, chi, tv);
        dist_term<float>(x2.w, y2.w, chi2_, tv2_);
      }
      if (i < n4) {
        const float4 x = __ldcs(a4 + i), y = __ldcs(b4 + i);
        dist_term<float>(x.x, y.x, chi, tv);
        dist_term<float>(x.y, y.y, chi, tv);
        dist_term<float>(x.z, y.z, chi, tv);
        dist_term<float>(x.w, y.w, chi, tv);
      }
      chi = ff_merge(chi, chi2_);
      tv = ff_merge(tv, tv2_);
    }
  }
  if (!vec)
    for (int64_t i = tid; i < n; i += nth) dist_term<T>(__ldcs(a + i), __ldcs(b + i), chi, tv);
  // block reduction, then the last block adds the block partials in order
  __shared__ double red[2][8];
  __shared__ bool last;
  double cv, tvv;
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      chi += __shfl_xor_sync(0xffffffffu, chi, o);
      tv += __shfl_xor_sync(0xffffffffu, tv, o);
    }
    cv = chi;
    tvv = tv;
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      chi = ff_merge(chi, FF{__shfl_xor_sync(0xffffffffu, chi.s, o), __shfl_xor_sync(0xffffffffu, chi.c, o)});
      tv = ff_merge(tv, FF{__shfl_xor_sync(0xffffffffu, tv.s, o), __shfl_xor_sync(0xffffffffu, tv.c, o)});
    }
    cv = ff_value(chi);
    tvv = ff_value(tv);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = cv;
    red[1][threadIdx.x >> 5] = tvv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double c = 0.0, t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      c += red[0][w];
      t += red[1][w];
    }
    part[2 * blockIdx.x] = c;
    part[2 * blockIdx.x + 1] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double c = 0.0, t = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
      c += __ldcg(part + 2 * k);
      t += __ldcg(part + 2 * k + 1);
    }
    *chi2 = c;
    *tv_out = 0.5 * t;
    *counter = 0u;
  }
}

template <typename T>
__device__ __forceinline__ float weight32(T v) {
  return v > T(0) ? (float)v : 0.0f;
}

// a warp per chunk of CH weights: L1[c] = sum of the chunk's weights
template <typename T>
__global__ void k_sample_chunks(const T* __restrict__ p, int64_t n, double* __restrict__ L1, int64_t nch) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < nch; c += nw) {
    const int64_t i0 = c * CH;
    double sum;
    if constexpr (sizeof(T) == 8) {
      double acc = 0.0;
      for (int k = lane; k < CH; k += 32) {
        const int64_t i = i0 + k;
        if (i < n) acc += fmax(p[i], 0.0);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      sum = acc;
    } else {
      FF acc{};
      if (i0 + CH <= n && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        // a whole chunk: 8 float4 per lane, two accumulators
        const float4* p4 = reinterpret_cast<const float4*>(p + i0);
        FF acc2{};
#pragma unroll
        for (int k = 0; k < CH / 128; k += 2) {
          const float4 q = __ldcs(p4 + k * 32 + lane), q2 = __ldcs(p4 + (k + 1) * 32 + lane);
          acc = ff_add(acc, weight32(q.x));
          acc2 = ff_add(acc2, weight32(q2.x));
          acc = ff_add(acc, weight32(q.y));
          acc2 = ff_add(acc2, weight32(q2.y));
          acc = ff_add(acc, weight32(q.z));
          acc2 = ff_add(acc2, weight32(q2.z));
          acc = ff_add(acc, weight32(q.w));
          acc2 = ff_add(acc2, weight32(q2.w));
        }
        acc = ff_merge(acc, acc2);
      } else {
        for (int k = lane; k < CH; k += 32) {
          const int64_t i = i0 + k;
          if (i < n) acc = ff_add(acc, weight32(p[i]));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        acc = ff_merge(acc, FF{__shfl_xor_sync(0xffffffffu, acc.s, o), __shfl_xor_sync(0xffffffffu, acc.c, o)});
      sum = ff_value(acc);
    }
    if (lane == 0) L1[c] = sum;
  }
}

// a warp per tile of CH chunk sums: T2[g] = sum of the tile's chunk sums
__global__ void k_sample_tiles(const double* __restrict__ L1, int64_t nch, double* __restrict__ T2, int64_t nt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = warp; g < nt; g += nw) {
    double acc = 0.0;
    for (int k = lane; k < CH; k += 32) {
      const int64_t c = g * CH + k;
      if (c < nch) acc += L1[c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) T2[g] = acc;
  }
}

// one block of 1024 threads: P2 = exclusive prefix of the tile sums (FP64), *total
__global__ void __launch_bounds__(1024) k_sample_scan(const double* __restrict__ T2, int64_t nt,
                                                      double* __restrict__ P2, double* __restrict__ total) {
  __shared__ double seg[1024];
  const int t = threadIdx.x;
  const int64_t per = (nt + 1023) / 1024;
  const int64_t lo = t * per, hi = min(nt, lo + per);
  double s = 0.0;
  for (int64_t j = lo; j < hi; ++j) s += T2[j];
  seg[t] = s;
  __syncthreads();
  if (t == 0) {
    double run = 0.0;
    for (int k = 0; k < 1024; ++k) {
      const double v = seg[k];
      seg[k] = run;
      run += v;
    }
    *total = run;
  }
  __syncthreads();
  double run = seg[t];
  for (int64_t j = lo; j < hi; ++j) {
    P2[j] = run;
    run += T2[j];
  }
}

// a warp per tile: P1[c] = P2[g] + exclusive prefix of the tile's chunk sums
__global__ void k_sample_tile_scan(const double* __restrict__ L1, int64_t nch, const double* __restrict__ P2,
                                   int64_t nt, double* __restrict__ P1) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = warp; g < nt; g += nw) {
    double carry = P2[g];
    for (int k0 = 0; k0 < CH; k0 += 32) {
      const int64_t c = g * CH + k0 + lane;
      const double v = c < nch ? L1[c] : 0.0;
      double incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (c < nch) P1[c] = carry + (incl - v);
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// FF compare: a.s + a.c > r.s + r.c, evaluated as (a.s - r.s) + (a.c - r.c) > 0
// (the leading difference is exact when the two are close)
__device__ __forceinline__ bool ff_greater(FF a, FF r) { return (a.s - r.s) + (a.c - r.c) > 0.0f; }
__device__ __forceinline__ FF ff_of(double x) {
  const float hi = (float)x;
  return FF{hi, (float)(x - (double)hi)};
}

// Warps take the draws 32 at a time: each lane first binary-searches the chunk
// of its own draw (32 searches in flight per warp), then the warp resolves
// the 32 draws one after the other inside their chunks.  A draw's chunk is
// staged in a padded 32 x 33 shared-memory tile (row q = weights 32q .. 32q +
// 31): FP32 chunks come in with 16-byte loads (lane l takes weights 4l + 128i
// .. + 3), partial chunks, FP64 and unaligned inputs with coalesced scalar
// loads (weight l + 32i); lane q then reads its row without bank conflicts
// (33-word pitch).  The next draw's chunk is loaded into registers while the
// current one is resolved.
constexpr int DRAW_THREADS = 256;
// warps per block: the tile of one warp is 4.2 KB (FP32) or 8.4 KB (FP64),
// and a block's static shared memory stays at 33 KB either way
template <typename T>
constexpr int draw_warps() {
  return sizeof(T) == 4 ? DRAW_THREADS / 32 : DRAW_THREADS / 64;
}

template <typename T>
__global__ void __launch_bounds__(DRAW_THREADS) k_sample_draw(const T* __restrict__ p, int64_t n,
                                                              const double* __restrict__ P1,
                                                              const double* __restrict__ L1, int64_t nch,
                                                              const double* __restrict__ total,
                                                              const double* __restrict__ u, int64_t m,
                                                              int64_t* __restrict__ out, int vec_ok) {
  __shared__ T tile[draw_warps<T>()][32][33];
  const int lane = threadIdx.x & 31;
  T(*wb)[33] = tile[threadIdx.x >> 5];
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double tot = *total;
  const bool vec4 = sizeof(T) == 4 && vec_ok;
  // this lane's 32 weights of a chunk, in the load order of its form
  T v[32];
  bool vform = false;
  auto load = [&](int64_t c) {
    const int64_t base = c * CH;
    vform = vec4 && base + CH <= n;
    if (vform) {
      const float4* q = reinterpret_cast<const float4*>(p + base) + lane;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 x = __ldg(q + 32 * i);
        v[4 * i] = x.x;
        v[4 * i + 1] = x.y;
        v[4 * i + 2] = x.z;
        v[4 * i + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int64_t idx = base + lane + 32 * i;
        v[i] = idx < n ? __ldg(p + idx) : T(0);
      }
    }
  };
  auto stage = [&]() {
    if (vform) {
      // weight e = 4 lane + 128 i + k goes to row e / 32, column e % 32
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) wb[4 * i + (lane >> 3)][4 * (lane & 7) + k] = v[4 * i + k];
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) wb[i][lane] = v[i];
    }
  };
  for (int64_t k0 = warp * 32; k0 < m; k0 += nw * 32) {
    const int nd = (int)(m - k0 < 32 ? m - k0 : 32);
    if (!(tot > 0.0)) {   // no outcome carries weight
      if (lane < nd) out[k0 + lane] = -1;
      continue;
    }
    // this lane's draw: the largest chunk c with P1[c] <= t that carries weight
    const int64_t kl = k0 + lane;
    int64_t my_c = 0;
    double my_r = 0.0;
    if (kl < m) {
      const double t = u[kl] * tot;
      int64_t lo = 0, hi = nch - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (P1[mid] <= t) lo = mid;
        else hi = mid - 1;
      }
      while (lo > 0 && L1[lo] <= 0.0) --lo;   // rounding put t past the weighted chunks
      my_c = lo;
      my_r = t - P1[lo];
    }
    int64_t c_next = __shfl_sync(0xffffffffu, my_c, 0);
    load(c_next);
    for (int j = 0; j < nd; ++j) {
      const int64_t k = k0 + j;
      const int64_t c = c_next;
      const double r = __shfl_sync(0xffffffffu, my_r, j);
      __syncwarp();   // the previous draw has finished reading the tile
      stage();
      __syncwarp();
      if (j + 1 < nd) {
        c_next = __shfl_sync(0xffffffffu, my_c, j + 1);
        load(c_next);   // in flight while this draw is resolved
      }
      // lane sums of the chunk's 32 runs of 32 weights (row `lane` of the tile)
      const int64_t base = c * CH + 32 * lane;
      FF ls{};
      double ld = 0.0;
#pragma unroll 8
      for (int i = 0; i < 32; ++i) {
        if constexpr (sizeof(T) == 8)
          ld += fmax(wb[lane][i], 0.0);
        else
          ls = ff_add(ls, weight32(wb[lane][i]));
      }
      const double lsum = sizeof(T) == 8 ? ld : ff_value(ls);
      double incl = lsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const double excl = incl - lsum;
      const unsigned over = __ballot_sync(0xffffffffu, incl > r && lsum > 0.0);
      const unsigned weighted = __ballot_sync(0xffffffffu, lsum > 0.0);
      const int L = over ? __ffs(over) - 1 : (weighted ? 31 - __clz(weighted) : 0);
      if (lane == L) {
        const double r2 = r - excl;
        int64_t pick = -1, last_w = -1;
        if constexpr (sizeof(T) == 8) {
          double cd = 0.0;
          for (int i = 0; i < 32 && pick < 0; ++i) {
            const int64_t idx = base + i;
            if (idx >= n) break;
            const double w = fmax(wb[L][i], 0.0);
            if (w > 0.0) last_w = idx;
            cd += w;
            if (w > 0.0 && cd > r2) pick = idx;
          }
        } else {
          // running sum and remainder both as compensated FP32 pairs: no FP64 per weight
          const FF rr = ff_of(r2);
          FF cs{};
          for (int i = 0; i < 32 && pick < 0; ++i) {
            const int64_t idx = base + i;
            if (idx >= n) break;
            const float w = weight32(wb[L][i]);
            if (w > 0.0f) last_w = idx;
            cs = ff_add(cs, w);
            if (w > 0.0f && ff_greater(cs, rr)) pick = idx;
          }
        }
        if (pick < 0) pick = last_w >= 0 ? last_w : base;
        out[k] = pick;
      }
    }
  }
}

unsigned grid_for(int64_t work, int per_block, int cap) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

size_t distance_scratch_bytes() { return (size_t)DIST_BLOCKS * 2 * sizeof(double) + 256; }

void launch_distance(const void* a, const void* b, int64_t n, int dtype, double* chi2, double* tv, void* scratch,
                     cudaStream_t s) {
  double* part = static_cast<double*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(static_cast<char*>(scratch) + (size_t)DIST_BLOCKS * 16);
  const unsigned g = grid_for(n, 256 * 4, DIST_BLOCKS);
  if (dtype == CUTQC_F64)
    k_distance<double><<<g, 256, 0, s>>>(static_cast<const double*>(a), static_cast<const double*>(b), n, part,
                                         counter, chi2, tv);
  else
    k_distance<float><<<g, 256, 0, s>>>(static_cast<const float*>(a), static_cast<const float*>(b), n, part,
                                        counter, chi2, tv);
  count_launch();
  check_launch("k_distance");
}

size_t sample_scratch_bytes(int64_t n) {
  const int64_t nch = (n + CH - 1) / CH, nt = (nch + CH - 1) / CH;
  return (size_t)(2 * nch + 2 * nt + 1) * sizeof(double) + 256;
}

void launch_sample(const void* p, int64_t n, int dtype, const double* u, int64_t m, int64_t* out, void* scratch,
                   cudaStream_t s) {
  const int64_t nch = (n + CH - 1) / CH, nt = (nch + CH - 1) / CH;
  double* L1 = static_cast<double*>(scratch);
  double* P1 = L1 + nch;
  double* T2 = P1 + nch;
  double* P2 = T2 + nt;
  double* total = P2 + nt;
  const unsigned gc = grid_for(nch * 32, 256, 152 * 16);
  if (dtype == CUTQC_F64)
    k_sample_chunks<double><<<gc, 256, 0, s>>>(static_cast<const double*>(p), n, L1, nch);
  else
    k_sample_chunks<float><<<gc, 256, 0, s>>>(static_cast<const float*>(p), n, L1, nch);
  count_launch();
  check_launch("k_sample_chunks");
  const unsigned gt = grid_for(nt * 32, 256, 152 * 16);
  k_sample_tiles<<<gt, 256, 0, s>>>(L1, nch, T2, nt);
  count_launch();
  check_launch("k_sample_tiles");
  k_sample_scan<<<1, 1024, 0, s>>>(T2, nt, P2, total);
  count_launch();
  check_launch("k_sample_scan");
  k_sample_tile_scan<<<gt, 256, 0, s>>>(L1, nch, P2, nt, P1);
  count_launch();
  check_launch("k_sample_tile_scan");
  if (m == 0) return;
  const int vec_ok = (reinterpret_cast<uintptr_t>(p) & 15) == 0;
  if (dtype == CUTQC_F64) {
    constexpr int bt = 32 * draw_warps<double>();
    k_sample_draw<double><<<grid_for((m + 31) / 32 * 32, bt, 152 * 16), bt, 0, s>>>(
        static_cast<const double*>(p), n, P1, L1, nch, total, u, m, out, vec_ok);
  } else {
    constexpr int bt = 32 * draw_warps<float>();
    k_sample_draw<float><<<grid_for((m + 31) / 32 * 32, bt, 152 * 16), bt, 0, s>>>(
        static_cast<const float*>(p), n, P1, L1, nch, total, u, m, out, vec_ok);
  }
  count_launch();
  check_launch("k_sample_draw");
}

}  // namespace cutqc

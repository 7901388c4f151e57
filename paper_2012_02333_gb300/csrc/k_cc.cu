// CUDA-core reconstruction: the plain FP32 / FP64 baseline of the 4^K sum.
//
// The sum over cut assignments between two groups of subcircuits is a
// contraction over the Pauli index (Sec. 3.3: 4^K Kronecker products):
//   P[m][n] = 2^-K sum_e A[e][m] B[e][n],
// with A, B the groups' tensors addressed through row maps e -> row.  Terms
// whose A row or B row is all zero are skipped first (early termination,
// Sec. 4.2) by a stable compaction of the inner index.  The epilogue deposits
// (m, n) into the output index g = depA(m) + depB(n) (the Kronecker product's
// bit interleave; qubit 0 = most significant bit) and accumulates sum_x p(x)
// in FP64.  Register-tiled GEMM in general; a matrix-vector form when one side
// has at most 8 outputs (k_cc_skinny), which is then bound by reading the
// other side once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace cutqc {

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ uint64_t deposit(const uint64_t* __restrict__ tab, int nbytes, uint64_t v) {
  uint64_t g = 0;
  for (int b = 0; b < nbytes; ++b) g += __ldg(tab + b * 256 + ((v >> (8 * b)) & 255));
  return g;
}

// ---- row statistics (one block per row): non-zero flag and max |entry| ----
template <typename T>
__device__ __forceinline__ void row_stats_block(const T* __restrict__ row, int64_t cols, int32_t* flag, float* rmax) {
  __shared__ float red[32];
  using V = typename Vec<T>::type;
  constexpr int W = Vec<T>::W;
  constexpr int U = 4;   // vector loads per thread per step: a 256-thread block reads 4096 FP32 values at once
  float m = 0.0f;
  int nz = 0;
  auto take = [&](T x) {
    nz |= (x != T(0));
    // FP32 tensors stay on the FP32 pipes (the FP64 pipe is narrow here)
    if constexpr (sizeof(T) == 4)
      m = fmaxf(m, fabsf(x));
    else
      m = fmaxf(m, (float)fabs(x));
  };
  if (cols % W == 0 && (reinterpret_cast<uintptr_t>(row) % sizeof(V)) == 0) {
    const V* rv = reinterpret_cast<const V*>(row);
    const int64_t nv = cols / W;
    for (int64_t i0 = threadIdx.x; i0 < nv; i0 += (int64_t)blockDim.x * U) {
      V v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        if (i < nv) {
          v[u] = __ldg(rv + i);
        } else {
          T* z = reinterpret_cast<T*>(&v[u]);
#pragma unroll
          for (int w = 0; w < W; ++w) z[w] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const T* x = reinterpret_cast<const T*>(&v[u]);
#pragma unroll
        for (int w = 0; w < W; ++w) take(x[w]);
      }
    }
  } else {
    for (int64_t i0 = threadIdx.x; i0 < cols; i0 += (int64_t)blockDim.x * U) {
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        v[u] = i < cols ? row[i] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) take(v[u]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  nz = __syncthreads_or(nz);
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    *flag = nz;
    *rmax = m;
  }
}

// the block-wide stable compaction of one contraction's row pairs (batch 1),
// the a-priori bound S and the split count
__device__ void compact_block(const CompactJob& cj) {
  __shared__ int warp_tot[32];
  __shared__ float warp_s[32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  float s_acc = 0.0f;   // the bound in FP32 (a magnitude estimate; the FP64 pipe is narrow)
  const int32_t* ra = cj.rows;
  const int32_t* rb = cj.rows + cj.kmax;
  for (int k0 = 0; k0 < cj.kmax; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    int keep = 0, a = 0, b = 0;
    if (k < cj.kmax) {
      a = ra[k];
      b = rb[k];
      keep = cj.nzA[a] && cj.nzB[b];
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) off += warp_tot[w];
      tot += warp_tot[w];
    }
    if (keep) {
      const int ci = base + off + __popc(m & ((1u << lane) - 1u));
      cj.crow[ci] = a;
      cj.crow[cj.kmax + ci] = b;
      if (cj.bound) s_acc = fmaf(cj.rmaxA[a], cj.rmaxB[b], s_acc);
    }
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s_acc += __shfl_xor_sync(0xffffffffu, s_acc, o);
  if (lane == 0) warp_s[warp] = s_acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    *cj.kcount = base;
    if (cj.sum_zero) *cj.sum_zero = 0.0;
    if (cj.bound) {
      float Sf = 0.0f;
      for (int w = 0; w < nw; ++w) Sf += warp_s[w];
      // FP32 accumulation error is far below 1e-4 relative: inflate so S stays an upper bound
      const double S = (double)Sf * cj.scale * (1.0 + 1e-4);
      *cj.bound = S;
      // BF16 x3 drops terms of at most ~3 * 2^-18 relative to |a||b| per product
      *cj.nseg = cj.nseg_fixed ? cj.nseg_fixed : (3.0 * 3.814697265625e-06 * S <= cj.split_tol ? 3 : 6);
    }
  }
}

// Rows of at most 2048 values (tensors with many cut rows: 4^8 rows of 64
// values occur) are reduced by warps, not blocks: a warp task is one row, or
// for rows of at most 32 vectors one 32-vector chunk of consecutive rows,
// read with one coalesced vector load per lane and reduced over the lanes of
// each row by shuffles.  8 warp tasks per block.
template <typename T>
__device__ __forceinline__ void row_stats_warp(const T* __restrict__ t, int64_t rows, int64_t cols, int64_t task,
                                               int32_t* __restrict__ flags, float* __restrict__ rmax) {
  using V = typename Vec<T>::type;
  constexpr int W = Vec<T>::W;
  const int lane = (int)threadIdx.x & 31;
  float m = 0.0f;
  int nz = 0;
  auto take = [&](const V& v) {
    const T* x = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      nz |= (x[w] != T(0));
      if constexpr (sizeof(T) == 4)
        m = fmaxf(m, fabsf(x[w]));
      else
        m = fmaxf(m, (float)fabs(x[w]));
    }
  };
  const int64_t nv = cols / W;   // vectors per row
  if (nv <= 32) {
    // one chunk of 32 vectors holds 32 / nv whole rows
    const int64_t e = task * 32 + lane;          // vector index
    const int64_t row = e / nv;
    if (row < rows) take(__ldg(reinterpret_cast<const V*>(t) + e));
    for (int o = 1; o < (int)nv; o <<= 1) {
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      nz |= __shfl_xor_sync(0xffffffffu, nz, o);
    }
    if (row < rows && (lane % (int)nv) == 0) {
      flags[row] = nz;
      rmax[row] = m;
    }
  } else {
    const int64_t row = task;
    if (row < rows) {
      const V* rv = reinterpret_cast<const V*>(t + row * cols);
      for (int64_t i = lane; i < nv; i += 128) {
        V v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i + 32 * u < nv) v[u] = __ldg(rv + i + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (i + 32 * u < nv) take(v[u]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      nz |= __shfl_xor_sync(0xffffffffu, nz, o);
    }
    if (row < rows && lane == 0) {
      flags[row] = nz;
      rmax[row] = m;
    }
  }
}

// warp tasks of a tensor in the warp form
__host__ __device__ __forceinline__ int64_t row_stats_tasks(int64_t rows, int64_t cols, int W) {
  const int64_t nv = cols / W;
  return nv <= 32 ? (rows * nv + 31) / 32 : rows;
}

// up to two tensors: the blocks of job 0, then those of job 1 (one per row,
// per chunk of a long row, or per 8 warp tasks); with a compaction job, the
// block that finishes last (an atomic count after a fence: every other
// block's statistics are then visible) compacts
template <typename T>
__global__ void k_row_stats(RowStatsJobs jobs) {
  CUTQC_PDL_LAUNCH();   // the operand preparation may launch and wait on this grid
  __shared__ int is_last;
  __shared__ int32_t part_nz;
  __shared__ float part_max;
  int j = 0;
  int64_t u = blockIdx.x;
  if (u >= jobs.blocks0) {
    u -= jobs.blocks0;
    j = 1;
  }
  const T* t = static_cast<const T*>(jobs.t[j]);
  // select, not a dynamic index into the parameter arrays
  const int chunks = j ? jobs.chunks[1] : jobs.chunks[0];
  const int64_t cols = j ? jobs.cols[1] : jobs.cols[0];
  int32_t* flags = j ? jobs.flags[1] : jobs.flags[0];
  float* rmax = j ? jobs.rmax[1] : jobs.rmax[0];
  const int warp_form = j ? jobs.warp[1] : jobs.warp[0];
  if (warp_form) {
    const int64_t rows = j ? jobs.rows[1] : jobs.rows[0];
    row_stats_warp<T>(t, rows, cols, u * 8 + (threadIdx.x >> 5), flags, rmax);
  } else if (chunks == 1) {
    row_stats_block<T>(t + u * cols, cols, flags + u, rmax + u);
  } else {
    // a chunk of a long row: combined into the row's cleared flag and maximum
    const int64_t r = u / chunks, ch = u % chunks, cc = cols / chunks;
    row_stats_block<T>(t + r * cols + ch * cc, cc, &part_nz, &part_max);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (part_nz) atomicOr(flags + r, 1);
      atomicMax(reinterpret_cast<int*>(rmax + r), __float_as_int(part_max));   // maxima are >= 0
    }
  }
  if (!jobs.cj.active) return;
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(jobs.cj.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  compact_block(jobs.cj);
  if (threadIdx.x == 0) *jobs.cj.counter = 0u;
}

// ---- stable compaction of the inner index (one block per batch) ----------
__global__ void k_compact(const int32_t* __restrict__ rows, int kmax, const int32_t* __restrict__ nzA,
                          const int32_t* __restrict__ nzB, int32_t* __restrict__ crow,
                          int32_t* __restrict__ kcount, const float* __restrict__ rmaxA,
                          const float* __restrict__ rmaxB, double scale, double* __restrict__ bound,
                          int32_t* __restrict__ nseg, int nseg_fixed, double split_tol,
                          double* __restrict__ sum_zero) {
  __shared__ int warp_tot[32];
  __shared__ float warp_s[32];
  __shared__ int base;
  float s_acc = 0.0f;   // the bound in FP32 (a magnitude estimate; the FP64 pipe is narrow)
  const int b = blockIdx.x;
  const int32_t* ra = rows + (int64_t)b * 2 * kmax;
  const int32_t* rb = ra + kmax;
  int32_t* ca = crow + (int64_t)b * 2 * kmax;
  int32_t* cb = ca + kmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int k0 = 0; k0 < kmax; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    int keep = 0, a = 0, bb = 0;
    if (k < kmax) {
      a = ra[k];
      bb = rb[k];
      keep = (nzA ? nzA[a] : 1) && (nzB ? nzB[bb] : 1);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int before = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) off += warp_tot[w];
      tot += warp_tot[w];
    }
    if (keep) {
      ca[base + off + before] = a;
      cb[base + off + before] = bb;
      if (bound) s_acc = fmaf(rmaxA[a], rmaxB[bb], s_acc);
    }
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (bound) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s_acc += __shfl_xor_sync(0xffffffffu, s_acc, o);
    if (lane == 0) warp_s[warp] = s_acc;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (sum_zero && b == 0) *sum_zero = 0.0;
    kcount[b] = base;
    if (bound) {
      float Sf = 0.0f;
      for (int w = 0; w < nw; ++w) Sf += warp_s[w];
      // FP32 accumulation error is far below 1e-4 relative: inflate so S stays an upper bound
      const double S = (double)Sf * scale * (1.0 + 1e-4);
      bound[b] = S;
      // BF16 x3 drops terms of at most ~3 * 2^-18 relative to |a||b| per product
      const double err3 = 3.0 * 3.814697265625e-06 * S;
      *nseg = nseg_fixed ? nseg_fixed : (err3 <= split_tol ? 3 : 6);
    }
  }
}

// ---- the CUDA-core contraction ---------------------------------------------
template <typename T>
struct CCArgs {
  const T* A;
  const T* B;
  int64_t M, N;           // 2^fA, 2^fB (also the row strides)
  int kmax;
  const int32_t* crow;    // [batch][2][kmax]
  const int32_t* kcount;  // [batch]
  const uint64_t* depA;
  const uint64_t* depB;
  int nbA, nbB;
  uint64_t out_batch_stride;
  T* out;
  T scale;
  double* sum;
  int vecB;
  int64_t tilesN;
};

// Block tile BM x BN, inner step BK, 256 threads as 16 x 16, each thread a
// (TM x TN) micro-tile split in two halves per dimension (rows ty*TM/2 + i
// and BM/2 + ty*TM/2 + i), so shared-memory reads are conflict-free float4s.
// compensated FP32 running sum (TwoSum: the rounding error of each add is
// recovered exactly and carried in c); the FP64 pipe is narrow on this part,
// so per-row sums of FP32 outputs avoid FP64 instructions
struct FFs {
  float s, c;
};
__device__ __forceinline__ FFs ffs_add(FFs a, float b) {
  const float s = a.s + b;
  const float bb = s - a.s;
  return {s, a.c + ((a.s - (s - bb)) + (b - bb))};
}

template <typename T, int BM, int BN, int BK>
__global__ __launch_bounds__(256) void k_cc_gemm(const CCArgs<T> a) {
  constexpr int TM = BM / 16, TN = BN / 16, HM = TM / 2, HN = TN / 2;
  constexpr int W = Vec<T>::W;
  using V = typename Vec<T>::type;
  static_assert(BK * BM / W == 256 && BK * BN / W == 256, "one vector load per thread");
  __shared__ __align__(16) T As[2][BK][BM];
  __shared__ __align__(16) T Bs[2][BK][BN];
  __shared__ double red[8];

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int batch = blockIdx.y;
  const int64_t tile = blockIdx.x;
  const int64_t m0 = (tile / a.tilesN) * BM, n0 = (tile % a.tilesN) * BN;
  const int32_t* ra = a.crow + (int64_t)batch * 2 * a.kmax;
  const int32_t* rb = ra + a.kmax;
  const int kc = a.kcount[batch];

  // loader coordinates: one W-vector of A and one of B per thread per step
  const int lka = tid / (BM / W), lma = (tid % (BM / W)) * W;
  const int lkb = tid / (BN / W), lnb = (tid % (BN / W)) * W;
  const bool fullM = a.M >= BM, fullN = a.N >= BN;

  auto load_a = [&](int k0, T (&reg)[W]) {
    const int k = k0 + lka;
#pragma unroll
    for (int w = 0; w < W; ++w) reg[w] = T(0);
    if (k < kc) {
      const T* p = a.A + (int64_t)ra[k] * a.M + m0 + lma;
      if (fullM) {
        V v = *reinterpret_cast<const V*>(p);
        const T* vp = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int w = 0; w < W; ++w) reg[w] = vp[w];
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w)
          if (m0 + lma + w < a.M) reg[w] = p[w];
      }
    }
  };
  auto load_b = [&](int k0, T (&reg)[W]) {
    const int k = k0 + lkb;
#pragma unroll
    for (int w = 0; w < W; ++w) reg[w] = T(0);
    if (k < kc) {
      const T* p = a.B + (int64_t)rb[k] * a.N + n0 + lnb;
      if (fullN) {
        V v = *reinterpret_cast<const V*>(p);
        const T* vp = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int w = 0; w < W; ++w) reg[w] = vp[w];
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w)
          if (n0 + lnb + w < a.N) reg[w] = p[w];
      }
    }
  };

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  T ga[W], gb[W];
  load_a(0, ga);
  load_b(0, gb);
  int buf = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    As[0][lka][lma + w] = ga[w];
    Bs[0][lkb][lnb + w] = gb[w];
  }
  __syncthreads();
  for (int k0 = 0; k0 < kc; k0 += BK) {
    const bool more = k0 + BK < kc;
    if (more) {
      load_a(k0 + BK, ga);
      load_b(k0 + BK, gb);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T ra_[TM], rb_[TN];
#pragma unroll
      for (int i = 0; i < HM; ++i) {
        ra_[i] = As[buf][kk][ty * HM + i];
        ra_[HM + i] = As[buf][kk][BM / 2 + ty * HM + i];
      }
#pragma unroll
      for (int j = 0; j < HN; ++j) {
        rb_[j] = Bs[buf][kk][tx * HN + j];
        rb_[HN + j] = Bs[buf][kk][BN / 2 + tx * HN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(ra_[i], rb_[j], acc[i][j]);
    }
    if (more) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        As[buf ^ 1][lka][lma + w] = ga[w];
        Bs[buf ^ 1][lkb][lnb + w] = gb[w];
      }
    }
    __syncthreads();
    buf ^= 1;
  }

  // epilogue: scale, deposit into the output index; the sum accumulates each
  // row's TN values pairwise in T, then across rows compensated (FP32 tensors)
  // or in FP64
  FFs lsum{0.0f, 0.0f};
  double local = 0.0;
  T* out = a.out + (uint64_t)batch * a.out_batch_stride;
  uint64_t gB[TN];
  bool okB[TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int64_t n = n0 + (j < HN ? tx * HN + j : BN / 2 + tx * HN + (j - HN));
    okB[j] = n < a.N;
    gB[j] = okB[j] ? deposit(a.depB, a.nbB, (uint64_t)n) : 0;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t m = m0 + (i < HM ? ty * HM + i : BM / 2 + ty * HM + (i - HM));
    if (m >= a.M) continue;
    const uint64_t gA = deposit(a.depA, a.nbA, (uint64_t)m);
    T rowv[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) rowv[j] = okB[j] ? acc[i][j] * a.scale : T(0);
#pragma unroll
    for (int w = TN / 2; w > 0; w >>= 1)
#pragma unroll
      for (int j = 0; j < w; ++j) rowv[j] += rowv[j + w];
    if constexpr (sizeof(T) == 4)
      lsum = ffs_add(lsum, (float)rowv[0]);
    else
      local += (double)rowv[0];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (a.vecB >= HN && okB[h * HN + HN - 1] && (HN == 2 || HN == 4)) {
        T v[HN];
#pragma unroll
        for (int j = 0; j < HN; ++j) v[j] = acc[i][h * HN + j] * a.scale;
        if constexpr (sizeof(T) == 4 && HN == 4) {
          *reinterpret_cast<float4*>(out + gA + gB[h * HN]) = make_float4(v[0], v[1], v[2], v[3]);
        } else if constexpr (HN == 2) {
          if constexpr (sizeof(T) == 8)
            *reinterpret_cast<double2*>(out + gA + gB[h * HN]) = make_double2(v[0], v[1]);
          else
            *reinterpret_cast<float2*>(out + gA + gB[h * HN]) = make_float2(v[0], v[1]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < HN; ++j) {
          if (!okB[h * HN + j]) continue;
          out[gA + gB[h * HN + j]] = acc[i][h * HN + j] * a.scale;
        }
      }
    }
  }
  if (a.sum) {
    if constexpr (sizeof(T) == 4) local = (double)lsum.s + (double)lsum.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((tid & 31) == 0) red[tid >> 5] = local;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int w = 0; w < 8; ++w) s += red[w];
      atomicAdd(a.sum, s);
    }
  }
}

// Skinny contraction: one operand has NS <= 8 outputs (for example a
// subcircuit whose qubits are all merged), so the work is a batch of
// matrix-vector products bound by reading the long operand L once.  A thread
// owns W consecutive long outputs and all NS short ones; per pass the block
// stages 256 of the batch's kept row pairs (the short operand's values and the
// long operand's row numbers) in shared memory.  `swap`: A is the short side.
template <typename T, int NS>
__global__ __launch_bounds__(256) void k_cc_skinny(const CCArgs<T> a, int swap) {
  constexpr int W = Vec<T>::W;
  constexpr int KT = 256;
  using V = typename Vec<T>::type;
  __shared__ T Ss[KT][NS];
  __shared__ int32_t Rl[KT];
  __shared__ double red[8];
  const int tid = threadIdx.x, batch = blockIdx.y;
  const T* L = swap ? a.B : a.A;
  const T* S = swap ? a.A : a.B;
  const int64_t ML = swap ? a.N : a.M;
  const int32_t* rA = a.crow + (int64_t)batch * 2 * a.kmax;
  const int32_t* rB = rA + a.kmax;
  const int32_t* rl = swap ? rB : rA;
  const int32_t* rs = swap ? rA : rB;
  const int kc = a.kcount[batch];
  const int64_t m0 = ((int64_t)blockIdx.x * 256 + tid) * W;
  T acc[W][NS];
#pragma unroll
  for (int w = 0; w < W; ++w)
#pragma unroll
    for (int n = 0; n < NS; ++n) acc[w][n] = T(0);
  for (int k0 = 0; k0 < kc; k0 += KT) {
    __syncthreads();
    for (int i = tid; i < KT * NS; i += 256) {
      const int k = i / NS, n = i % NS;
      Ss[k][n] = k0 + k < kc ? S[(int64_t)rs[k0 + k] * NS + n] : T(0);
    }
    for (int i = tid; i < KT; i += 256) Rl[i] = k0 + i < kc ? rl[k0 + i] : 0;
    __syncthreads();
    const int kn = min(KT, kc - k0);
    if (m0 < ML) {
#pragma unroll 8
      for (int k = 0; k < kn; ++k) {
        const V v = __ldcs(reinterpret_cast<const V*>(L + (int64_t)Rl[k] * ML + m0));
        const T* vp = reinterpret_cast<const T*>(&v);
#pragma unroll
        for (int w = 0; w < W; ++w)
#pragma unroll
          for (int n = 0; n < NS; ++n) acc[w][n] = fma(vp[w], Ss[k][n], acc[w][n]);
      }
    }
  }
  FFs lsum{0.0f, 0.0f};
  double local = 0.0;
  if (m0 < ML) {
    T* out = a.out + (uint64_t)batch * a.out_batch_stride;
    const uint64_t* depL = swap ? a.depB : a.depA;
    const uint64_t* depS = swap ? a.depA : a.depB;
    const int nbL = swap ? a.nbB : a.nbA, nbS = swap ? a.nbA : a.nbB;
    uint64_t gS[NS];
#pragma unroll
    for (int n = 0; n < NS; ++n) gS[n] = deposit(depS, nbS, (uint64_t)n);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint64_t gL = deposit(depL, nbL, (uint64_t)(m0 + w));
      T v[NS];
#pragma unroll
      for (int n = 0; n < NS; ++n) {
        v[n] = acc[w][n] * a.scale;
        out[gL + gS[n]] = v[n];
      }
#pragma unroll
      for (int h = NS / 2; h > 0; h >>= 1)
#pragma unroll
        for (int n = 0; n < h; ++n) v[n] += v[n + h];
      if constexpr (sizeof(T) == 4)
        lsum = ffs_add(lsum, (float)v[0]);
      else
        local += (double)v[0];
    }
  }
  if (a.sum) {
    if constexpr (sizeof(T) == 4) local = (double)lsum.s + (double)lsum.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((tid & 31) == 0) red[tid >> 5] = local;
    __syncthreads();
    if (tid == 0) {
      double t = 0;
      for (int w = 0; w < 8; ++w) t += red[w];
      atomicAdd(a.sum, t);
    }
  }
}

template <typename T>
CCArgs<T> cc_args(const Contraction& c) {
  CCArgs<T> a;
  a.A = static_cast<const T*>(c.A);
  a.B = static_cast<const T*>(c.B);
  a.M = int64_t(1) << c.fA;
  a.N = int64_t(1) << c.fB;
  a.kmax = c.kmax;
  a.crow = c.crow;
  a.kcount = c.kcount;
  a.depA = c.depA;
  a.depB = c.depB;
  a.nbA = (c.fA + 7) / 8;
  a.nbB = (c.fB + 7) / 8;
  a.out_batch_stride = c.out_batch_stride;
  a.out = static_cast<T*>(c.out);
  a.scale = T(c.scale);
  a.sum = c.sum;
  a.vecB = c.vecB;
  a.tilesN = 1;
  return a;
}

template <typename T>
void launch_skinny(const Contraction& c, cudaStream_t s) {
  const CCArgs<T> a = cc_args<T>(c);
  const int swap = c.fA < c.fB ? 1 : 0;
  const int fS = swap ? c.fA : c.fB;
  const int64_t ML = int64_t(1) << (swap ? c.fB : c.fA);
  constexpr int W = Vec<T>::W;
  const dim3 grid((unsigned)((ML + 256 * W - 1) / (256 * W)), (unsigned)c.batch);
  cudaEvent_t ev = nullptr;
  if (c.profile) prof_begin(s, &ev);
  switch (fS) {
    case 0: k_cc_skinny<T, 1><<<grid, 256, 0, s>>>(a, swap); break;
    case 1: k_cc_skinny<T, 2><<<grid, 256, 0, s>>>(a, swap); break;
    case 2: k_cc_skinny<T, 4><<<grid, 256, 0, s>>>(a, swap); break;
    default: k_cc_skinny<T, 8><<<grid, 256, 0, s>>>(a, swap); break;
  }
  count_launch();
  check_launch("k_cc_skinny");
  if (c.profile) prof_end(s, ev);
}

template <typename T, int BM, int BN, int BK>
void launch_typed(const Contraction& c, cudaStream_t s) {
  CCArgs<T> a;
  a.A = static_cast<const T*>(c.A);
  a.B = static_cast<const T*>(c.B);
  a.M = int64_t(1) << c.fA;
  a.N = int64_t(1) << c.fB;
  a.kmax = c.kmax;
  a.crow = c.crow;
  a.kcount = c.kcount;
  a.depA = c.depA;
  a.depB = c.depB;
  a.nbA = (c.fA + 7) / 8;
  a.nbB = (c.fB + 7) / 8;
  a.out_batch_stride = c.out_batch_stride;
  a.out = static_cast<T*>(c.out);
  a.scale = T(c.scale);
  a.sum = c.sum;
  a.vecB = c.vecB;
  const int64_t tilesM = (a.M + BM - 1) / BM;
  a.tilesN = (a.N + BN - 1) / BN;
  dim3 grid((unsigned)(tilesM * a.tilesN), (unsigned)c.batch);
  cudaEvent_t ev = nullptr;
  if (c.profile) prof_begin(s, &ev);
  k_cc_gemm<T, BM, BN, BK><<<grid, 256, 0, s>>>(a);
  count_launch();
  check_launch("k_cc_gemm");
  if (c.profile) prof_end(s, ev);
}

// ---- low-rank contraction (at most 16 kept terms) --------------------------
// P[m][n] = scale * sum_{k < kc} A[ra[k]][m] B[rb[k]][n] for kc <= 16, the
// shape of circuits cut by one or two wires (4 or 16 terms) and of a
// disconnected subcircuit joined as an outer product (1 term), whose outputs
// run to 2^26 .. 2^28: the work is a few FMAs per output and the output
// stream is everything.  A thread keeps 4 consecutive columns of the kc B
// rows in registers (the N side owns the two lowest output bits) and walks
// the rows of 256-row panels of A staged in shared memory with the rows'
// output offsets; every 4 outputs go out as one 16-byte streaming store
// (FP32; two for FP64), four rows per unrolled step.  Work items are
// (problem, 256 rows, up to 1024 columns), listed per problem column-tile
// by column-tile; block b takes items b, b + G, b + 2G, ... (measured faster
// than contiguous ranges per block: the blocks then write neighbouring
// items at any time), and the next item's A panel is copied into the other
// half of a double-buffered panel while the current one is written (no DRAM
// round trip between items).  The FP64 sum is carried per thread in
// compensated FP32 (FP32 tensors) and added once per warp and problem.
template <typename T>
struct LRProblem {
  const T* A;
  const T* B;
  const int32_t* crow;     // [2][kmax]: compacted row pairs
  const int32_t* kcount;
  int kmax;
  int fA, fB, nbA, nbB;
  const uint64_t* depA;
  const uint64_t* depB;
  T* out;
  double* sum;
  double scale;
};
struct LRItem {
  int prob;
  int n0;
  int64_t m0;
};
constexpr int LR_MB = 256;     // rows per item (one staged panel)
constexpr int LR_NT = 1024;    // columns per item (256 threads x 4)

template <typename T>
struct LRArgs {
  const LRProblem<T>* probs;   // device list (batch) or null: `one` and an implicit item grid
  const LRItem* items;
  int64_t n_items;
  LRProblem<T> one;
  int64_t one_tiles_m;         // single problem: item it is column tile it / tiles_m, row tile it % tiles_m
};

// blocks per SM of each term class (register budget of the B columns)
template <typename T, int KC>
constexpr int lr_min_blocks() {
  return sizeof(T) == 8 ? (KC == 16 ? 1 : 2) : (KC == 16 ? 2 : (KC == 4 ? 4 : 6));
}
// two A panels, the output offsets of the low 8 row bits
template <typename T, int KC>
constexpr size_t lr_smem_bytes() {
  return 2 * (size_t)LR_MB * KC * sizeof(T) + 256 * sizeof(uint64_t);
}

__device__ __forceinline__ void lr_cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void lr_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void lr_cp_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// the thread's row of an item's A panel, copied to shared memory without
// passing through registers (so the copy stays in flight while the current
// item is written); zero beyond kc and beyond the last row
template <typename T, int KC>
__device__ __forceinline__ void lr_fetch(const LRProblem<T>& p, int kc, int64_t m0, T (*As)[KC]) {
  const int64_t M = int64_t(1) << p.fA;
  const int64_t m = m0 + threadIdx.x;
  const bool ok = m < M;
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    if (k < kc && ok)
      lr_cp_async(&As[threadIdx.x][k], p.A + (int64_t)__ldg(p.crow + k) * M + m, (int)sizeof(T));
    else
      As[threadIdx.x][k] = T(0);
  }
  lr_cp_commit();
}

// output offset of the rows m0 .. m0 + 255 beyond their low 8 bits (m0 is a
// multiple of 256, so the low byte of row m0 + i is i)
template <typename T>
__device__ __forceinline__ uint64_t lr_base(const LRProblem<T>& p, int64_t m0) {
  uint64_t g = 0;
  for (int b = 1; b < p.nbA; ++b) g += __ldg(p.depA + b * 256 + ((m0 >> (8 * b)) & 255));
  return g;
}

// this thread's 4 columns of the kc B rows, scaled by 2^-K (a power of two:
// exact), and their output offset
template <typename T, int KC>
__device__ __forceinline__ void lr_load_b(const LRProblem<T>& p, int kc, int n0, T (&b)[KC][4], uint64_t& gB) {
  const int N = 1 << p.fB;
  const int cols = N < LR_NT ? N : LR_NT;
  const int n = n0 + 4 * ((int)threadIdx.x % (cols / 4));
  const int32_t* rb = p.crow + p.kmax;
  const T sc = (T)p.scale;
#pragma unroll
  for (int k = 0; k < KC; ++k) {
#pragma unroll
    for (int j = 0; j < 4; ++j) b[k][j] = T(0);
    if (k < kc) {
      const T* src = p.B + (int64_t)__ldg(rb + k) * N + n;
      if constexpr (sizeof(T) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(src));
        b[k][0] = v.x * sc;
        b[k][1] = v.y * sc;
        b[k][2] = v.z * sc;
        b[k][3] = v.w * sc;
      } else {
        const double2 v0 = __ldg(reinterpret_cast<const double2*>(src));
        const double2 v1 = __ldg(reinterpret_cast<const double2*>(src) + 1);
        b[k][0] = v0.x * sc;
        b[k][1] = v0.y * sc;
        b[k][2] = v1.x * sc;
        b[k][3] = v1.y * sc;
      }
    }
  }
  gB = deposit(p.depB, p.nbB, (uint64_t)n);
}

template <typename T>
struct LRAcc {
  FFs f{0.0f, 0.0f};
  double d = 0.0;
};

// one output row of 4 columns: the row's panel values (16 bytes per
// shared-memory read, zero beyond kc), the store and the running sum
template <typename T, int KC>
__device__ __forceinline__ void lr_row(T* __restrict__ out, const T (*As)[KC], const uint64_t* tab0, uint64_t base,
                                       int i, const T (&b)[KC][4], uint64_t gB, LRAcc<T>& acc) {
  T v[4] = {T(0), T(0), T(0), T(0)};
  if constexpr (KC == 1) {
    const T a0 = As[i][0];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = a0 * b[0][j];
  } else {
#pragma unroll
    for (int k0 = 0; k0 < KC; k0 += 16 / (int)sizeof(T)) {
      T a[16 / sizeof(T)];
      if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(&As[i][k0]);
        a[0] = q.x;
        a[1] = q.y;
        a[2] = q.z;
        a[3] = q.w;
      } else {
        const double2 q = *reinterpret_cast<const double2*>(&As[i][k0]);
        a[0] = q.x;
        a[1] = q.y;
      }
#pragma unroll
      for (int kk = 0; kk < 16 / (int)sizeof(T); ++kk)
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = fma(a[kk], b[k0 + kk][j], v[j]);
    }
  }
  T* dst = out + (base + tab0[i] + gB);
  if constexpr (sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4*>(dst), make_float4(v[0], v[1], v[2], v[3]));
    acc.f = ffs_add(acc.f, (v[0] + v[1]) + (v[2] + v[3]));
  } else {
    __stcs(reinterpret_cast<double2*>(dst), make_double2(v[0], v[1]));
    __stcs(reinterpret_cast<double2*>(dst) + 1, make_double2(v[2], v[3]));
    acc.d += (v[0] + v[1]) + (v[2] + v[3]);
  }
}

// the rows of one item from a staged panel, four rows per step
template <typename T, int KC>
__device__ __forceinline__ void lr_rows(const LRProblem<T>& p, int64_t m0, const T (*As)[KC], const uint64_t* tab0,
                                        uint64_t base, const T (&b)[KC][4], uint64_t gB, LRAcc<T>& acc) {
  const int64_t M = int64_t(1) << p.fA;
  const int N = 1 << p.fB;
  const int cols = N < LR_NT ? N : LR_NT;
  const int tpr = cols / 4;                 // threads per row
  const int rpp = 256 / tpr;                // rows per pass
  const int rs = (int)threadIdx.x / tpr;
  const int rows = (int)((M - m0) < LR_MB ? (M - m0) : LR_MB);
  T* __restrict__ out = p.out;
  int i = rs;
  for (; i + 3 * rpp < rows; i += 4 * rpp) {
    lr_row<T, KC>(out, As, tab0, base, i, b, gB, acc);
    lr_row<T, KC>(out, As, tab0, base, i + rpp, b, gB, acc);
    lr_row<T, KC>(out, As, tab0, base, i + 2 * rpp, b, gB, acc);
    lr_row<T, KC>(out, As, tab0, base, i + 3 * rpp, b, gB, acc);
  }
  for (; i < rows; i += rpp) lr_row<T, KC>(out, As, tab0, base, i, b, gB, acc);
}

// the warp's share of the FP64 sum, added to the problem's sum
template <typename T>
__device__ __forceinline__ void lr_flush(double* sum, LRAcc<T>& acc) {
  if (sum) {
    double t = sizeof(T) == 4 ? (double)acc.f.s + (double)acc.f.c : acc.d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t != 0.0) atomicAdd(sum, t);
  }
  acc = LRAcc<T>{};
}

// KC = 1 (an outer product), 4 (one cut between the final groups) or 16
// (two): the register and shared-memory footprint of the smaller forms lets
// more blocks share an SM
template <typename T, int KC>
__global__ __launch_bounds__(256, lr_min_blocks<T, KC>()) void k_lowrank(const LRArgs<T> a) {
  extern __shared__ __align__(16) unsigned char lr_smem[];
  __shared__ LRProblem<T> sp;
  T(*As)[LR_MB][KC] = reinterpret_cast<T(*)[LR_MB][KC]>(lr_smem);
  uint64_t* tab0 = reinterpret_cast<uint64_t*>(lr_smem + 2 * (size_t)LR_MB * KC * sizeof(T));
  const int64_t it0 = blockIdx.x, it1 = a.n_items, step = gridDim.x;
  if (it0 >= it1) return;
  auto item_of = [&](int64_t it, int& prob, int64_t& m0, int& n0) {
    if (a.items) {
      const LRItem x = a.items[it];
      prob = x.prob;
      m0 = x.m0;
      n0 = x.n0;
    } else {
      prob = 0;
      m0 = (it % a.one_tiles_m) * LR_MB;
      n0 = (int)(it / a.one_tiles_m) * LR_NT;
    }
  };
  // the problem's parameters and its low-byte output offsets into shared memory
  // (the kept-term count is loaded beside the table)
  int kc;
  auto begin_problem = [&](int prob) {
    if (threadIdx.x == 0) sp = a.probs ? a.probs[prob] : a.one;
    __syncthreads();
    tab0[threadIdx.x] = __ldg(sp.depA + threadIdx.x);
    kc = *sp.kcount;
    __syncthreads();
  };
  int prob, n0;
  int64_t m0;
  item_of(it0, prob, m0, n0);
  begin_problem(prob);
  lr_fetch<T, KC>(sp, kc, m0, As[0]);
  T b[KC][4];
  uint64_t gB;
  lr_load_b<T, KC>(sp, kc, n0, b, gB);
  uint64_t base = lr_base(sp, m0);
  LRAcc<T> acc;
  lr_cp_wait();
  __syncthreads();
  int buf = 0;
  for (int64_t it = it0; it < it1; it += step) {
    const bool more = it + step < it1;
    int nprob = prob, nn0 = n0;
    int64_t nm0 = m0;
    if (more) item_of(it + step, nprob, nm0, nn0);
    const bool same = more && nprob == prob;
    // the next item's panel goes to the other buffer (last read before the
    // previous barrier) while this item is written
    if (same) lr_fetch<T, KC>(sp, kc, nm0, As[buf ^ 1]);
    lr_rows<T, KC>(sp, m0, As[buf], tab0, base, b, gB, acc);
    if (!same) lr_flush<T>(sp.sum, acc);
    if (more) {
      if (!same) {
        __syncthreads();   // every thread is done with the old problem's parameters
        begin_problem(nprob);
        lr_fetch<T, KC>(sp, kc, nm0, As[buf ^ 1]);
      }
      if (!same || nn0 != n0) lr_load_b<T, KC>(sp, kc, nn0, b, gB);
      base = lr_base(sp, nm0);
      prob = nprob;
      m0 = nm0;
      n0 = nn0;
    }
    lr_cp_wait();
    __syncthreads();
    buf ^= 1;
  }
}

// ---- every low-rank problem of a batch in three launches -----------------
// k_batch_rowstats: the row non-zero flags and max |.| of every problem's two
// operands, one block per chunk of at most 2^16 columns of a row over all
// problems (operands of one or two rows of 2^25-2^26 columns occur), each
// chunk's partial result to its own slot; k_batch_compact: one block per
// problem combines its rows' chunks into the flags and maxima, then compacts
// its row pairs (early termination, Sec. 4.2) and clears its FP64 sum;
// k_lowrank: the items of every problem.  No launch waits on another's
// blocks, so the three can run beside the batch's tensor-core problems.
struct BatchRowJob {
  const void* T;
  int64_t rows, cols;
  int64_t first;               // the job's first partial slot (row chunk) in the global slot order
  int64_t bfirst;              // the job's first block unit
  int chunks;                  // column chunks per row
  int warp;                    // rows of at most 2048 values: 8 warp tasks per block unit, one slot per row
  int32_t* flags;
  float* rmax;
};
constexpr int64_t BATCH_CHUNK = int64_t(1) << 16;   // columns per row chunk

template <typename T>
__global__ __launch_bounds__(256) void k_batch_rowstats(const BatchRowJob* __restrict__ rjobs, int nrjobs,
                                                        int64_t nblocks, int32_t* __restrict__ part_nz,
                                                        float* __restrict__ part_max) {
  for (int64_t u = blockIdx.x; u < nblocks; u += gridDim.x) {
    int j = 0;
    while (j + 1 < nrjobs && rjobs[j + 1].bfirst <= u) ++j;
    const BatchRowJob& rj = rjobs[j];
    if (rj.warp) {
      row_stats_warp<T>(static_cast<const T*>(rj.T), rj.rows, rj.cols, (u - rj.bfirst) * 8 + (threadIdx.x >> 5),
                        part_nz + rj.first, part_max + rj.first);
    } else {
      const int64_t unit = u - rj.bfirst;
      const int64_t row = unit / rj.chunks, ch = unit % rj.chunks;
      const int64_t cc = rj.cols / rj.chunks;
      row_stats_block<T>(static_cast<const T*>(rj.T) + row * rj.cols + ch * cc, cc, part_nz + rj.first + unit,
                         part_max + rj.first + unit);
      __syncthreads();   // the block's shared reduction buffer is reused by the next unit
    }
  }
}

__global__ __launch_bounds__(256) void k_batch_compact(const CompactJob* __restrict__ cjobs,
                                                       const BatchRowJob* __restrict__ rjobs, int nprob,
                                                       const int32_t* __restrict__ part_nz,
                                                       const float* __restrict__ part_max) {
  for (int p = blockIdx.x; p < nprob; p += gridDim.x) {
    for (int side = 0; side < 2; ++side) {
      const BatchRowJob& rj = rjobs[2 * p + side];
      for (int64_t r = threadIdx.x; r < rj.rows; r += blockDim.x) {
        int32_t nz = 0;
        float mx = 0.0f;
        for (int c = 0; c < rj.chunks; ++c) {
          nz |= part_nz[rj.first + r * rj.chunks + c];
          mx = fmaxf(mx, part_max[rj.first + r * rj.chunks + c]);
        }
        rj.flags[r] = nz;
        rj.rmax[r] = mx;
      }
    }
    __syncthreads();
    compact_block(cjobs[p]);
    __syncthreads();
  }
}

template <typename T>
LRProblem<T> lr_problem(const Contraction& c) {
  LRProblem<T> p{};
  p.A = static_cast<const T*>(c.A);
  p.B = static_cast<const T*>(c.B);
  p.crow = c.crow;
  p.kcount = c.kcount;
  p.kmax = c.kmax;
  p.fA = c.fA;
  p.fB = c.fB;
  p.nbA = std::max((c.fA + 7) / 8, 1);
  p.nbB = std::max((c.fB + 7) / 8, 1);
  p.depA = c.depA;
  p.depB = c.depB;
  p.out = static_cast<T*>(c.out);
  p.sum = c.sum;
  p.scale = c.scale;
  return p;
}

int lr_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    CUTQC_CUDA(cudaGetDevice(&dev));
    CUTQC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

int lr_grid(int64_t items, int per_sm) { return (int)std::min<int64_t>(items, (int64_t)lr_sms() * per_sm); }

// one launch of the low-rank kernel of term class KC (1, 4 or 16): as many
// blocks as fit, at most one per item (each walks several items, the next
// item's panel in flight; one block per item was measured slower in the
// batch, 3.25 against 3.08 ms of GPU time)
template <typename T, int KC>
void lr_launch(const LRArgs<T>& a, cudaStream_t s) {
  if (a.n_items == 0) return;
  constexpr size_t smem = lr_smem_bytes<T, KC>();
  if constexpr (smem > 48 * 1024) {
    static bool set = false;
    if (!set) {
      CUTQC_CUDA(cudaFuncSetAttribute(k_lowrank<T, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      set = true;
    }
  }
  k_lowrank<T, KC><<<lr_grid(a.n_items, lr_min_blocks<T, KC>()), 256, smem, s>>>(a);
  count_launch();
  check_launch("k_lowrank");
}

}  // namespace

bool lowrank_eligible(const Contraction& c) {
  return c.batch == 1 && c.kmax <= 16 && c.fB >= 2 && c.fB <= 30 && c.vecB >= 4 && c.fA <= 40;
}

static int64_t lr_tiles_n(const Contraction& c) { return c.fB >= 10 ? (int64_t(1) << (c.fB - 10)) : 1; }
static int64_t lr_tiles_m(const Contraction& c) { return ((int64_t(1) << c.fA) + LR_MB - 1) / LR_MB; }

int64_t lowrank_items(const Contraction& c) { return lr_tiles_n(c) * lr_tiles_m(c); }

// term class of a low-rank contraction: 0 (one term), 1 (up to 4), 2 (up to 16)
static int lr_class(const Contraction& c) { return c.kmax <= 1 ? 0 : (c.kmax <= 4 ? 1 : 2); }


// device tables of a batch: [problems][compaction jobs][row jobs][items]
// [chunk flags][chunk maxima]
struct BatchLayout {
  size_t probs, cjobs, rjobs, items, part_nz, part_max, bytes;
  int64_t n_items, nunits, nblocks;
  int64_t cls_items[3];
};
static size_t up256(size_t x) { return (x + 255) / 256 * 256; }

static int64_t row_chunks(int64_t cols) { return std::max<int64_t>(1, cols / BATCH_CHUNK); }

// the row-statistics geometry of one operand of a batch: warp form for rows
// of at most 2048 values, else a block per row chunk
static bool batch_warp_form(int64_t cols, int W) { return cols >= W && cols <= 2048; }
static int64_t batch_blocks(int64_t rows, int64_t cols, int W) {
  return batch_warp_form(cols, W) ? (row_stats_tasks(rows, cols, W) + 7) / 8 : rows * row_chunks(cols);
}

static BatchLayout batch_layout(const std::vector<Contraction>& cs) {
  BatchLayout L{};
  const size_t P = cs.size();
  for (const Contraction& c : cs) {
    const int W = c.dtype == CUTQC_F64 ? 2 : 4;
    L.n_items += lowrank_items(c);
    L.cls_items[lr_class(c)] += lowrank_items(c);
    L.nunits += (int64_t)c.rowsA * row_chunks(int64_t(1) << c.fA) + (int64_t)c.rowsB * row_chunks(int64_t(1) << c.fB);
    L.nblocks += batch_blocks(c.rowsA, int64_t(1) << c.fA, W) + batch_blocks(c.rowsB, int64_t(1) << c.fB, W);
  }
  L.probs = 0;
  L.cjobs = up256(P * std::max(sizeof(LRProblem<float>), sizeof(LRProblem<double>)));
  L.rjobs = L.cjobs + up256(P * sizeof(CompactJob));
  L.items = L.rjobs + up256(2 * P * sizeof(BatchRowJob));
  L.part_nz = L.items + up256((size_t)L.n_items * sizeof(LRItem));
  L.part_max = L.part_nz + up256((size_t)L.nunits * sizeof(int32_t));
  L.bytes = L.part_max + up256((size_t)L.nunits * sizeof(float));
  return L;
}

size_t lowrank_batch_bytes(const std::vector<Contraction>& cs) { return batch_layout(cs).bytes; }

void lowrank_batch_tables(const std::vector<Contraction>& cs, std::vector<char>& host, int64_t* n_items) {
  const BatchLayout L = batch_layout(cs);
  const bool f64 = !cs.empty() && cs[0].dtype == CUTQC_F64;
  const size_t psz = f64 ? sizeof(LRProblem<double>) : sizeof(LRProblem<float>);
  host.assign(L.bytes, 0);
  int64_t it = 0, unit0 = 0, block0 = 0;
  for (size_t i = 0; i < cs.size(); ++i) {
    const Contraction& c = cs[i];
    if ((c.dtype == CUTQC_F64) != f64) fail(CUTQC_ERR_ARG, "one dtype per low-rank batch");
    if (!c.rows || !c.nzA || !c.nzB || !c.rmaxA || !c.rmaxB) fail(CUTQC_ERR_ARG, "batched problem without its tables");
    if (f64) {
      const LRProblem<double> p = lr_problem<double>(c);
      std::memcpy(host.data() + L.probs + i * psz, &p, psz);
    } else {
      const LRProblem<float> p = lr_problem<float>(c);
      std::memcpy(host.data() + L.probs + i * psz, &p, psz);
    }
    CompactJob cj{};
    cj.active = 1;
    cj.rows = c.rows;
    cj.kmax = c.kmax;
    cj.nzA = c.nzA;
    cj.nzB = c.nzB;
    cj.crow = c.crow;
    cj.kcount = c.kcount;
    cj.sum_zero = c.sum;
    std::memcpy(host.data() + L.cjobs + i * sizeof(CompactJob), &cj, sizeof(CompactJob));
    for (int side = 0; side < 2; ++side) {
      BatchRowJob rj{};
      rj.T = side ? c.B : c.A;
      rj.rows = side ? c.rowsB : c.rowsA;
      rj.cols = int64_t(1) << (side ? c.fB : c.fA);
      rj.first = unit0;
      rj.bfirst = block0;
      rj.chunks = (int)row_chunks(rj.cols);
      rj.warp = batch_warp_form(rj.cols, f64 ? 2 : 4) ? 1 : 0;
      rj.flags = const_cast<int32_t*>(side ? c.nzB : c.nzA);
      rj.rmax = const_cast<float*>(side ? c.rmaxB : c.rmaxA);
      unit0 += rj.rows * rj.chunks;
      block0 += batch_blocks(rj.rows, rj.cols, f64 ? 2 : 4);
      std::memcpy(host.data() + L.rjobs + (2 * i + side) * sizeof(BatchRowJob), &rj, sizeof(BatchRowJob));
    }
  }
  // items by term class (one launch each), per problem column tile by
  // column tile
  for (int cls = 0; cls < 3; ++cls)
    for (size_t i = 0; i < cs.size(); ++i) {
      const Contraction& c = cs[i];
      if (lr_class(c) != cls) continue;
      for (int64_t tn = 0; tn < lr_tiles_n(c); ++tn)
        for (int64_t tm = 0; tm < lr_tiles_m(c); ++tm) {
          LRItem item{(int)i, (int)(tn * LR_NT), tm * LR_MB};
          std::memcpy(host.data() + L.items + (size_t)it * sizeof(LRItem), &item, sizeof(LRItem));
          ++it;
        }
    }
  *n_items = it;
}

void launch_lowrank_batch(const void* dev_tables, const std::vector<Contraction>& cs, int64_t n_items,
                          cudaStream_t s) {
  if (cs.empty()) return;
  const BatchLayout L = batch_layout(cs);
  if (L.n_items != n_items) fail(CUTQC_ERR_ARG, "batch tables do not match the problems");
  const char* t = static_cast<const char*>(dev_tables);
  const auto* rjobs = reinterpret_cast<const BatchRowJob*>(t + L.rjobs);
  int32_t* pnz = reinterpret_cast<int32_t*>(const_cast<char*>(t) + L.part_nz);
  float* pmx = reinterpret_cast<float*>(const_cast<char*>(t) + L.part_max);
  const int np = (int)cs.size();
  const unsigned g1 = (unsigned)std::min<int64_t>(L.nblocks, 152 * 8);
  if (cs[0].dtype == CUTQC_F64)
    k_batch_rowstats<double><<<g1, 256, 0, s>>>(rjobs, 2 * np, L.nblocks, pnz, pmx);
  else
    k_batch_rowstats<float><<<g1, 256, 0, s>>>(rjobs, 2 * np, L.nblocks, pnz, pmx);
  count_launch();
  check_launch("k_batch_rowstats");
  k_batch_compact<<<(unsigned)np, 256, 0, s>>>(reinterpret_cast<const CompactJob*>(t + L.cjobs), rjobs, np, pnz, pmx);
  count_launch();
  check_launch("k_batch_compact");
  auto run = [&](auto tag) {
    using T = decltype(tag);
    LRArgs<T> a{};
    a.probs = reinterpret_cast<const LRProblem<T>*>(t + L.probs);
    const LRItem* items = reinterpret_cast<const LRItem*>(t + L.items);
    for (int cls = 0; cls < 3; ++cls) {
      a.items = items;
      a.n_items = L.cls_items[cls];
      if (cls == 0) lr_launch<T, 1>(a, s);
      if (cls == 1) lr_launch<T, 4>(a, s);
      if (cls == 2) lr_launch<T, 16>(a, s);
      items += L.cls_items[cls];
    }
  };
  if (cs[0].dtype == CUTQC_F64)
    run(double{});
  else
    run(float{});
}

void launch_lowrank(const Contraction& c, cudaStream_t s) {
  if (!lowrank_eligible(c)) fail(CUTQC_ERR_UNSUPPORTED, "shape not supported by the low-rank contraction");
  cudaEvent_t ev = nullptr;
  if (c.profile) prof_begin(s, &ev);
  auto run = [&](auto tag) {
    using T = decltype(tag);
    LRArgs<T> a{};
    a.one = lr_problem<T>(c);
    a.n_items = lowrank_items(c);
    a.one_tiles_m = lr_tiles_m(c);
    const int cls = lr_class(c);
    if (cls == 0) lr_launch<T, 1>(a, s);
    if (cls == 1) lr_launch<T, 4>(a, s);
    if (cls == 2) lr_launch<T, 16>(a, s);
  };
  if (c.dtype == CUTQC_F64)
    run(double{});
  else
    run(float{});
  if (c.profile) prof_end(s, ev);
}

void launch_row_stats(const RowStatsJobs& jobs, int dtype, cudaStream_t s) {
  RowStatsJobs j = jobs;
  if (j.n < 2) j.rows[1] = 0;
  // tensors with fewer rows than SMs and long rows: a block per chunk of
  // 2^16 columns, combined with atomics into outputs cleared first; rows of
  // at most 2048 values (of vector-aligned tensors): 8 warp tasks per block;
  // other rows: a block each
  const int W = dtype == CUTQC_F64 ? 2 : 4;
  int64_t blocks = 0;
  bool block_rows = false;
  for (int k = 0; k < 2; ++k) {
    j.chunks[k] = 1;
    j.warp[k] = 0;
    int64_t bk = 0;
    if (k < j.n && j.rows[k] < 152 && j.cols[k] > (int64_t(1) << 18)) {
      j.chunks[k] = (int)(j.cols[k] >> 16);
      CUTQC_CUDA(cudaMemsetAsync(j.flags[k], 0, (size_t)j.rows[k] * sizeof(int32_t), s));
      CUTQC_CUDA(cudaMemsetAsync(j.rmax[k], 0, (size_t)j.rows[k] * sizeof(float), s));
      bk = j.rows[k] * j.chunks[k];
      block_rows = true;
    } else if (k < j.n && j.cols[k] >= W && j.cols[k] <= 2048 &&
               reinterpret_cast<uintptr_t>(j.t[k]) % (4 * (size_t)W) == 0) {
      j.warp[k] = 1;
      bk = (row_stats_tasks(j.rows[k], j.cols[k], W) + 7) / 8;
    } else {
      bk = j.rows[k];
      if (k < j.n && j.rows[k] > 0) block_rows = true;
    }
    if (k == 0) j.blocks0 = bk;
    blocks += bk;
  }
  const int64_t cmax = std::max(j.cols[0], j.n > 1 ? j.cols[1] : int64_t(0));
  const int threads = (cmax >= 256 || j.warp[0] || j.warp[1] || !block_rows) ? 256 : 32;
  if (dtype == CUTQC_F64)
    k_row_stats<double><<<(unsigned)blocks, threads, 0, s>>>(j);
  else
    k_row_stats<float><<<(unsigned)blocks, threads, 0, s>>>(j);
  count_launch();
  check_launch("k_row_stats");
}

void launch_row_stats(const void* T_, int dtype, int rows, int f, int32_t* flags, float* rmax, cudaStream_t s) {
  RowStatsJobs j{};
  j.n = 1;
  j.t[0] = T_;
  j.rows[0] = rows;
  j.cols[0] = int64_t(1) << f;
  j.flags[0] = flags;
  j.rmax[0] = rmax;
  launch_row_stats(j, dtype, s);
}

void launch_compact(const Contraction& c, cudaStream_t s) {
  int threads = 32;
  while (threads < c.kmax && threads < 1024) threads *= 2;
  if (c.bound && c.batch != 1) fail(CUTQC_ERR_UNSUPPORTED, "split-precision bound needs batch 1");
  k_compact<<<c.batch, threads, 0, s>>>(c.rows, c.kmax, c.nzA, c.nzB, c.crow, c.kcount, c.rmaxA, c.rmaxB,
                                        c.scale, c.bound, c.nseg, c.nseg_fixed, c.split_tol, c.sum_zero);
  count_launch();
  check_launch("k_compact");
}

// a short side of at most 8 outputs: the matrix-vector form (its long side
// needs at least one vector of 4 FP32 / 2 FP64 values per row)
bool cc_is_skinny(int fA, int fB) { return std::min(fA, fB) <= 3 && std::max(fA, fB) >= 2; }

void launch_cc_gemm(const Contraction& c, cudaStream_t s) {
  if (cc_is_skinny(c.fA, c.fB)) {
    if (c.dtype == CUTQC_F64)
      launch_skinny<double>(c, s);
    else
      launch_skinny<float>(c, s);
    return;
  }
  if (c.dtype == CUTQC_F64)
    launch_typed<double, 64, 64, 8>(c, s);
  else if (std::min(c.fA, c.fB) <= 6)
    launch_typed<float, 64, 64, 16>(c, s);   // a side of at most 64 outputs: a quarter of the idle tile
  else
    launch_typed<float, 128, 128, 8>(c, s);
}

void launch_fill_zero(void* p, size_t bytes, cudaStream_t s) {
  CUTQC_CUDA(cudaMemsetAsync(p, 0, bytes, s));
}

}  // namespace cutqc

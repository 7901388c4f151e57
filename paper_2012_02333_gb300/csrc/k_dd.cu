// Dynamic definition (Sec. 4.3, Algorithm 1): merging, bin ranking.
//
// k_dd_merge: for one subcircuit, groups the states that share the values of
//   its merged qubits (Algorithm 1: "group shots with common merged qubits"):
//   M[row][xa] = sum_{xm} T[row][dep_act(xa) | dep_mrg(xm) | zoom], where the
//   zoomed qubits are fixed at their bits.  Memory-bound: T is read once.
//   When the merged qubits are the lowest output bits (the usual case) each
//   output is a contiguous run read with 16-byte loads; otherwise, with >= 32
//   merged values per output, a warp owns an output (lanes stride the merged
//   index).  Runs of up to 32 values are summed pairwise in FP32 and folded
//   into FP64; the FP64 sums are kept for the bin ranking.
// k_topk_warps / k_topk_final: the 32 heaviest bins by their stored value
//   (ties to the lower index): every warp keeps a sorted list of 32 across its
//   lanes and inserts only values above its current minimum (ballot + shuffle);
//   a single block merges the warp lists.
// k_dd_gather64 / k_dd_eval: FP64 values of the candidate bins: the merge
//   kernels also keep their sums in FP64 (each run accumulated in FP64), the
//   candidate's merged values are gathered from there, then
//   2^-K sum_e prod_c M64_c[row_c(e)] in FP64.
#include <cuda_runtime.h>

#include <cfloat>

#include "internal.h"

namespace cutqc {

namespace {

__device__ __forceinline__ uint64_t dep_tab(const uint64_t* __restrict__ tab, int nbytes, uint64_t v) {
  uint64_t g = 0;
  for (int b = 0; b < nbytes; ++b) g += __ldg(tab + b * 256 + ((v >> (8 * b)) & 255));
  return g;
}

template <typename T>
__global__ void k_dd_merge_warp(const T* __restrict__ Tin, int64_t cols, int a, int mg,
                                const uint64_t* __restrict__ depAct, int nbA, const uint64_t* __restrict__ depMrg,
                                int nbM, uint64_t zoom, T* __restrict__ out, double* __restrict__ out64,
                                int64_t n_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nm = int64_t(1) << mg;
  for (int64_t o = warp; o < n_out; o += nwarps) {
    const int64_t row = o >> a;
    const uint64_t xa = (uint64_t)o & ((uint64_t(1) << a) - 1);
    const T* base = Tin + row * cols + (dep_tab(depAct, nbA, xa) | zoom);
    double acc = 0.0;
    for (int64_t x0 = lane; x0 < nm; x0 += 32 * 16) {
      T run = T(0);
#pragma unroll 4
      for (int r = 0; r < 16; ++r) {
        const int64_t xm = x0 + 32 * r;
        if (xm < nm) run += base[dep_tab(depMrg, nbM, (uint64_t)xm)];
      }
      acc += (double)run;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      out[o] = (T)acc;
      out64[o] = acc;
    }
  }
}

template <typename T>
__global__ void k_dd_merge_thread(const T* __restrict__ Tin, int64_t cols, int a, int mg,
                                  const uint64_t* __restrict__ depAct, int nbA,
                                  const uint64_t* __restrict__ depMrg, int nbM, uint64_t zoom,
                                  T* __restrict__ out, double* __restrict__ out64, int64_t n_out) {
  const int nm = 1 << mg;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_out; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = o >> a;
    const uint64_t xa = (uint64_t)o & ((uint64_t(1) << a) - 1);
    const T* base = Tin + row * cols + (dep_tab(depAct, nbA, xa) | zoom);
    T acc = T(0);
    for (int xm = 0; xm < nm; ++xm) acc += base[dep_tab(depMrg, nbM, (uint64_t)xm)];
    out[o] = acc;
    out64[o] = (double)acc;
  }
}

// Merged qubits on the lowest output bits: every output sums one contiguous
// run of 2^mg values.  Thread per output for runs of 4..256 values (16-byte
// loads, pairwise FP32 over groups of 32, FP64 across groups), warp per
// output for longer runs.
__device__ __forceinline__ float sum4(float4 v) { return (v.x + v.y) + (v.z + v.w); }

__global__ void k_dd_merge_run_thread(const float* __restrict__ Tin, int64_t cols, int a, int mg,
                                      const uint64_t* __restrict__ depAct, int nbA, uint64_t zoom,
                                      float* __restrict__ out, double* __restrict__ out64, int64_t n_out) {
  const int ng = 1 << (mg - 2);   // float4 groups in the run
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_out; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = o >> a;
    const uint64_t xa = (uint64_t)o & ((uint64_t(1) << a) - 1);
    const float4* p = reinterpret_cast<const float4*>(Tin + row * cols + (dep_tab(depAct, nbA, xa) | zoom));
    double acc = 0.0;
    for (int g0 = 0; g0 < ng; g0 += 8) {
      float t8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) t8[j] = g0 + j < ng ? sum4(p[g0 + j]) : 0.0f;
#pragma unroll
      for (int w = 4; w > 0; w >>= 1)
#pragma unroll
        for (int j = 0; j < w; ++j) t8[j] += t8[j + w];
      acc += (double)t8[0];
    }
    out[o] = (float)acc;
    out64[o] = acc;
  }
}

__global__ void k_dd_merge_run_warp(const float* __restrict__ Tin, int64_t cols, int a, int mg,
                                    const uint64_t* __restrict__ depAct, int nbA, uint64_t zoom,
                                    float* __restrict__ out, double* __restrict__ out64, int64_t n_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ng = int64_t(1) << (mg - 2);
  for (int64_t o = warp; o < n_out; o += nwarps) {
    const int64_t row = o >> a;
    const uint64_t xa = (uint64_t)o & ((uint64_t(1) << a) - 1);
    const float4* p = reinterpret_cast<const float4*>(Tin + row * cols + (dep_tab(depAct, nbA, xa) | zoom));
    double acc = 0.0;
    for (int64_t g0 = lane; g0 < ng; g0 += 32 * 8) {
      float t8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) t8[j] = g0 + 32 * j < ng ? sum4(p[g0 + 32 * j]) : 0.0f;
#pragma unroll
      for (int w = 4; w > 0; w >>= 1)
#pragma unroll
        for (int j = 0; j < w; ++j) t8[j] += t8[j + w];
      acc += (double)t8[0];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      out[o] = (float)acc;
      out64[o] = acc;
    }
  }
}

// ---- top-32 selection ------------------------------------------------------
constexpr int KC = 32;

__device__ __forceinline__ bool before(float v1, int64_t i1, float v2, int64_t i2) {
  return v1 > v2 || (v1 == v2 && i1 < i2);
}

// insert (v, idx) into the warp's list (lane j holds the j-th best)
__device__ __forceinline__ void warp_insert(float& lv, int64_t& li, float v, int64_t idx, int lane) {
  const unsigned ahead = __ballot_sync(0xffffffffu, before(lv, li, v, idx));
  const int pos = __popc(ahead);
  const float uv = __shfl_up_sync(0xffffffffu, lv, 1);
  const int64_t ui = __shfl_up_sync(0xffffffffu, li, 1);
  if (pos < 32) {
    if (lane > pos) {
      lv = uv;
      li = ui;
    } else if (lane == pos) {
      lv = v;
      li = idx;
    }
  }
}

template <typename T>
__global__ void k_topk_warps(const T* __restrict__ bins, int64_t n, int64_t per_warp, float* __restrict__ cv,
                             int64_t* __restrict__ ci) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  float lv = -FLT_MAX;
  int64_t li = INT64_MAX;
  const int64_t lo = warp * per_warp, hi = min(n, lo + per_warp);
  // 128 consecutive values per step, 4 per lane (lane-major within the step, so
  // candidates of one lane come in increasing index order and ties resolve low)
  for (int64_t b0 = lo; b0 < hi; b0 += 128) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = b0 + 32 * u + lane;
      v[u] = i < hi ? (float)bins[i] : -FLT_MAX;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = b0 + 32 * u + lane;
      const float thr = __shfl_sync(0xffffffffu, lv, 31);
      unsigned m = __ballot_sync(0xffffffffu, i < hi && v[u] > thr);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const float sv = __shfl_sync(0xffffffffu, v[u], src);
        const int64_t si = __shfl_sync(0xffffffffu, i, src);
        warp_insert(lv, li, sv, si, lane);
      }
    }
  }
  cv[warp * KC + lane] = lv;
  ci[warp * KC + lane] = li;
}

// one block of 1024 threads merges `m` candidate pairs into the best KC
__global__ void k_topk_final(const float* __restrict__ cv, const int64_t* __restrict__ ci, int64_t m,
                             float* __restrict__ ov, int64_t* __restrict__ oi) {
  __shared__ float sv[32 * KC];
  __shared__ int64_t si[32 * KC];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float lv = -FLT_MAX;
  int64_t li = INT64_MAX;
  for (int64_t b0 = (int64_t)w * 32; b0 < m; b0 += 32 * 32) {
    const int64_t j = b0 + lane;
    const float v = j < m ? cv[j] : -FLT_MAX;
    const int64_t idx = j < m ? ci[j] : INT64_MAX;
    unsigned msk = __ballot_sync(0xffffffffu, j < m && before(v, idx, __shfl_sync(0xffffffffu, lv, 31),
                                                              __shfl_sync(0xffffffffu, li, 31)));
    while (msk) {
      const int src = __ffs(msk) - 1;
      msk &= msk - 1;
      warp_insert(lv, li, __shfl_sync(0xffffffffu, v, src), __shfl_sync(0xffffffffu, idx, src), lane);
    }
  }
  sv[w * KC + lane] = lv;
  si[w * KC + lane] = li;
  __syncthreads();
  if (w == 0) {
    lv = -FLT_MAX;
    li = INT64_MAX;
    for (int j0 = 0; j0 < 32 * KC; j0 += 32) {
      const float v = sv[j0 + lane];
      const int64_t idx = si[j0 + lane];
      unsigned msk = __ballot_sync(0xffffffffu, before(v, idx, __shfl_sync(0xffffffffu, lv, 31),
                                                        __shfl_sync(0xffffffffu, li, 31)));
      while (msk) {
        const int src = __ffs(msk) - 1;
        msk &= msk - 1;
        warp_insert(lv, li, __shfl_sync(0xffffffffu, v, src), __shfl_sync(0xffffffffu, idx, src), lane);
      }
    }
    ov[lane] = lv;
    oi[lane] = li;
  }
}

// ---- FP64 re-evaluation of candidate bins ----------------------------------
// M64[cand][c][row] = the FP64 merged value of subcircuit c at the candidate's
// active bits (gathered from the merge kernels' FP64 output).  grid: (cand, c).
__global__ void k_dd_gather64(const DdEvalArgs a, double* __restrict__ m64) {
  const int cand = blockIdx.x, c = blockIdx.y;
  const DdEvalSub& s = a.sub[c];
  const int64_t bin = a.cand_idx[cand];
  if (bin < 0 || bin >= (int64_t(1) << a.n_active)) return;
  // active bits of this subcircuit: xa bit (a-1-i) = bin bit at rank act_rank[i]
  uint64_t xa = 0;
  for (int i = 0; i < s.a; ++i) {
    const uint64_t bit = (bin >> (a.n_active - 1 - s.act_rank[i])) & 1;
    xa |= bit << (s.a - 1 - i);
  }
  for (int64_t row = threadIdx.x; row < s.rows; row += blockDim.x)
    m64[((int64_t)cand * a.n_sub + c) * a.max_rows + row] = s.m64[(row << s.a) + xa];
}

// value[cand] = 2^-K sum_e prod_c M64[cand][c][row_c(e)].  grid: cand, block 256.
__global__ void k_dd_eval(const DdEvalArgs a, const double* __restrict__ m64, double* __restrict__ val) {
  const int cand = blockIdx.x;
  __shared__ double red[8];
  const int64_t nterms = int64_t(1) << (2 * a.n_cuts);
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < nterms; e += blockDim.x) {
    double prod = 1.0;
    for (int c = 0; c < a.n_sub; ++c) {
      const DdEvalSub& s = a.sub[c];
      int64_t row = 0;
      for (int j = 0; j < s.ncuts; ++j) row = 4 * row + ((e >> (2 * (a.n_cuts - 1 - s.cuts[j]))) & 3);
      prod *= m64[((int64_t)cand * a.n_sub + c) * a.max_rows + row];
    }
    acc += prod;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += red[w];
    val[cand] = tot * a.scale;
  }
}

unsigned grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

void launch_dd_merge(const void* T, int dtype, int64_t rows, int f, int a, int mg, const uint64_t* depAct,
                     const uint64_t* depMrg, uint64_t zoom, bool run, void* M, double* M64, cudaStream_t s) {
  const int64_t n_out = rows << a;
  const int64_t cols = int64_t(1) << f;
  const int nbA = (a + 7) / 8, nbM = (mg + 7) / 8;
  run = run && (reinterpret_cast<uintptr_t>(T) & 15) == 0;
  if (run && dtype == CUTQC_F32 && mg >= 2 && mg <= 8) {
    k_dd_merge_run_thread<<<grid_for(n_out, 256), 256, 0, s>>>(static_cast<const float*>(T), cols, a, mg, depAct,
                                                                nbA, zoom, static_cast<float*>(M), M64, n_out);
  } else if (run && dtype == CUTQC_F32 && mg > 8) {
    k_dd_merge_run_warp<<<grid_for(n_out * 32, 256), 256, 0, s>>>(static_cast<const float*>(T), cols, a, mg,
                                                                   depAct, nbA, zoom, static_cast<float*>(M), M64,
                                                                   n_out);
  } else if (mg >= 5) {
    const unsigned g = grid_for(n_out * 32, 256);
    if (dtype == CUTQC_F64)
      k_dd_merge_warp<double><<<g, 256, 0, s>>>(static_cast<const double*>(T), cols, a, mg, depAct, nbA, depMrg, nbM,
                                                zoom, static_cast<double*>(M), M64, n_out);
    else
      k_dd_merge_warp<float><<<g, 256, 0, s>>>(static_cast<const float*>(T), cols, a, mg, depAct, nbA, depMrg, nbM,
                                               zoom, static_cast<float*>(M), M64, n_out);
  } else {
    const unsigned g = grid_for(n_out, 256);
    if (dtype == CUTQC_F64)
      k_dd_merge_thread<double><<<g, 256, 0, s>>>(static_cast<const double*>(T), cols, a, mg, depAct, nbA, depMrg,
                                                  nbM, zoom, static_cast<double*>(M), M64, n_out);
    else
      k_dd_merge_thread<float><<<g, 256, 0, s>>>(static_cast<const float*>(T), cols, a, mg, depAct, nbA, depMrg, nbM,
                                                 zoom, static_cast<float*>(M), M64, n_out);
  }
  count_launch();
  check_launch("k_dd_merge");
}

size_t topk_workspace_bytes(int64_t n) {
  const int64_t warps = 152 * 8 * 4;
  return (size_t)warps * KC * (4 + 8) + 256;
}

void launch_topk(const void* bins, int dtype, int64_t n, void* ws, float* out_v, int64_t* out_i, cudaStream_t s) {
  const int64_t warps_max = 152 * 8 * 4;
  int64_t per_warp = ((n + warps_max - 1) / warps_max + 127) / 128 * 128;
  if (per_warp < 128) per_warp = 128;
  const int64_t warps = (n + per_warp - 1) / per_warp;
  const unsigned blocks = (unsigned)((warps + 7) / 8);
  float* cv = static_cast<float*>(ws);
  int64_t* ci = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + (size_t)warps_max * KC * 4);
  if (dtype == CUTQC_F64)
    k_topk_warps<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(bins), n, per_warp, cv, ci);
  else
    k_topk_warps<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(bins), n, per_warp, cv, ci);
  count_launch();
  check_launch("k_topk_warps");
  k_topk_final<<<1, 1024, 0, s>>>(cv, ci, (int64_t)blocks * 8 * KC, out_v, out_i);
  count_launch();
  check_launch("k_topk_final");
}

void launch_dd_rerank(const DdEvalArgs& a, int dtype, double* m64, double* val, cudaStream_t s) {
  k_dd_gather64<<<dim3(a.n_cand, a.n_sub), 256, 0, s>>>(a, m64);
  count_launch();
  check_launch("k_dd_gather64");
  k_dd_eval<<<a.n_cand, 256, 0, s>>>(a, m64, val);
  count_launch();
  check_launch("k_dd_eval");
}

}  // namespace cutqc

// Dynamic definition (Sec. 4.3, Algorithm 1): merging, bin ranking.
//
// k_dd_merge: for one subcircuit, groups the states that share the values of
//   its merged qubits (Algorithm 1: "group shots with common merged qubits"):
//   M[row][xa] = sum_{xm} T[row][dep_act(xa) | dep_mrg(xm) | zoom], where the
//   zoomed qubits are fixed at their bits.  Memory-bound: T is read once.
//   When the merged qubits are the lowest output bits (the usual case) each
//   output is a contiguous run read with 16-byte loads; otherwise, with >= 32
//   merged values per output, a warp owns an output (lanes stride the merged
//   index).  FP32 tensors are summed in compensated FP32 (runs of up to 32
//   values plainly, then TwoSum); the rounded sum feeds the contraction and
//   the compensation term is kept for the FP64 bin ranking.
// k_topk_warps / k_topk_final: the 32 heaviest bins by their stored value
//   (ties to the lower index): every warp keeps a sorted list of 32 across its
//   lanes and inserts only values above its current minimum (ballot + shuffle);
//   a single block merges the warp lists.
// k_dd_gather64 / k_dd_eval: FP64 values of the candidate bins: the
//   candidate's merged values (rounded sum + compensation) are gathered in
//   FP64, then 2^-K sum_e prod_c M64_c[row_c(e)] in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <type_traits>

#include "internal.h"

namespace cutqc {

namespace {

__device__ __forceinline__ uint64_t dep_tab(const uint64_t* __restrict__ tab, int nbytes, uint64_t v) {
  uint64_t g = 0;
  for (int b = 0; b < nbytes; ++b) g += __ldg(tab + b * 256 + ((v >> (8 * b)) & 255));
  return g;
}

// Compensated FP32 accumulation: a value is carried as s + c, s the rounded
// sum and c the accumulated rounding error.  ff_add is Knuth's TwoSum (the
// error of s = a + b is recovered exactly with six FP32 operations) plus the
// sum of the incoming error terms; ff_norm moves the error into s once at the
// end (Fast2Sum), so fl(s) is the rounded result and s + c holds the extra
// bits.  All of it runs on the FP32 pipes, which on this GPU outrun the FP64
// pipe by far more than the six-fold operation count.
struct FF {
  float s, c;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.s + b.s;
  const float bb = s - a.s;
  const float err = (a.s - (s - bb)) + (b.s - bb);
  return {s, (a.c + b.c) + err};
}

__device__ __forceinline__ FF ff_norm(FF a) {
  const float s = a.s + a.c;
  return {s, a.c - (s - a.s)};
}

__device__ __forceinline__ FF ff_shfl_xor(FF a, int off) {
  return {__shfl_xor_sync(0xffffffffu, a.s, off), __shfl_xor_sync(0xffffffffu, a.c, off)};
}

__device__ __forceinline__ void store_merged(float* out, float* outc, int64_t o, FF v) {
  v = ff_norm(v);
  out[o] = v.s;
  outc[o] = v.c;
}
__device__ __forceinline__ void store_merged(double* out, float*, int64_t o, double v) { out[o] = v; }

// Generic merge: a warp owns an output when there are >= 32 merged values
// (mg >= 5); lanes stride the merged index and sum runs of 16 in the
// tensor's type.
template <typename T>
__global__ void k_dd_merge_warp(const T* __restrict__ Tin, int64_t cols, int a, int mg,
                                const uint64_t* __restrict__ depAct, int nbA, const uint64_t* __restrict__ depMrg,
                                int nbM, uint64_t zoom, T* __restrict__ out, float* __restrict__ outc,
                                int64_t n_out) {
  using Acc = typename std::conditional<sizeof(T) == 4, FF, double>::type;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nm = int64_t(1) << mg;
  for (int64_t o = warp; o < n_out; o += nwarps) {
    const int64_t row = o >> a;
    const uint64_t xa = (uint64_t)o & ((uint64_t(1) << a) - 1);
    // the deposit is additive over disjoint index bits: the lane's part
    // (merged-index bits 0-4) once, the rest once per step and the same for
    // every lane (one broadcast load instead of a table lookup per value)
    const T* base = Tin + row * cols + (dep_tab(depAct, nbA, xa) | zoom) + dep_tab(depMrg, nbM, (uint64_t)lane);
    Acc acc{};
    for (int64_t x0 = 0; x0 < nm; x0 += 32 * 16) {
      T v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {   // 16 independent loads in flight per lane
        const int64_t xh = x0 + 32 * r;   // nm is a multiple of 32 (mg >= 5)
        v[r] = xh < nm ? base[dep_tab(depMrg, nbM, (uint64_t)xh)] : T(0);
      }
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if constexpr (sizeof(T) == 4)
          acc = ff_add(acc, FF{v[r], 0.0f});
        else
          acc += v[r];
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      if constexpr (sizeof(T) == 4)
        acc = ff_add(acc, ff_shfl_xor(acc, off));
      else
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
    }
    if (lane == 0) store_merged(out, outc, o, acc);
  }
}

// Generic merge with < 32 merged values: a thread per output.
template <typename T>
__global__ void k_dd_merge_thread(const T* __restrict__ Tin, int64_t cols, int a, int mg,
                                  const uint64_t* __restrict__ depAct, int nbA,
                                  const uint64_t* __restrict__ depMrg, int nbM, uint64_t zoom,
                                  T* __restrict__ out, float* __restrict__ outc, int64_t n_out) {
  const int nm = 1 << mg;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_out; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = o >> a;
    const uint64_t xa = (uint64_t)o & ((uint64_t(1) << a) - 1);
    const T* base = Tin + row * cols + (dep_tab(depAct, nbA, xa) | zoom);
    if constexpr (sizeof(T) == 4) {
      FF acc{};
      for (int xm = 0; xm < nm; ++xm) acc = ff_add(acc, FF{base[dep_tab(depMrg, nbM, (uint64_t)xm)], 0.0f});
      store_merged(out, outc, o, acc);
    } else {
      T acc = T(0);
      for (int xm = 0; xm < nm; ++xm) acc += base[dep_tab(depMrg, nbM, (uint64_t)xm)];
      out[o] = acc;
    }
  }
}

// Merged qubits on the lowest output bits: every output sums one contiguous
// run of 2^mg FP32 values.  A group of G = min(32, 2^mg / 4) lanes owns an
// output and reads its run with 16-byte loads, lane j taking float4 j, j + G,
// ... (one warp instruction covers 32 consecutive float4 of one run, or
// several whole runs).  With runs of at most 1024 values (PER = float4 per
// lane <= 8) a group takes 8 / PER outputs per step, so every lane has 8
// independent loads in flight.  Every addition is compensated (TwoSum), so
// the stored sum plus its compensation term carry the merged value to about
// FP64 accuracy: the FP64 re-ranking of candidate bins reads them.  `dense`: the active bits
// are the bits directly above the merged ones, so a run starts at
// row * cols + zoom + (xa << mg) without the deposit table.  Outputs too few
// to fill the GPU are split into 2^lnch chunks whose partial sums go to
// `part` and are combined in chunk order by k_dd_merge_finish.
__device__ __forceinline__ FF sum4(float4 v) {
  return ff_add(ff_add(FF{v.x, 0.0f}, FF{v.y, 0.0f}), ff_add(FF{v.z, 0.0f}, FF{v.w, 0.0f}));
}

template <int G, int PER>
__global__ void k_dd_merge_run(const float* __restrict__ Tin, int64_t cols, int a, int mg,
                               const uint64_t* __restrict__ depAct, int nbA, uint64_t zoom, int dense, int lnch,
                               float* __restrict__ out, float* __restrict__ outc, float2* __restrict__ part,
                               int64_t n_out) {
  constexpr int GPW = 32 / G;                    // groups per warp
  constexpr int U = PER == 0 ? 1 : 8 / PER;      // outputs per group per step
  const int lane = threadIdx.x & 31, gl = lane & (G - 1), gi = lane / G;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_units = n_out << lnch;
  const int64_t per = (int64_t(1) << (mg - 2 - lnch)) / G;   // float4 per lane in one chunk
  const uint64_t amask = (uint64_t(1) << a) - 1;
  const int64_t chmask = (int64_t(1) << lnch) - 1;
  auto unit_ptr = [&](int64_t u) {
    const int64_t o = u >> lnch, ch = u & chmask;
    const int64_t row = o >> a;
    const uint64_t xa = (uint64_t)o & amask;
    const uint64_t off = dense ? zoom + (xa << mg) : (dep_tab(depAct, nbA, xa) | zoom);
    return reinterpret_cast<const float4*>(Tin + row * cols + off) + ch * per * G + gl;
  };
  for (int64_t ub = warp * GPW * U; ub < n_units; ub += nwarps * GPW * U) {
    FF acc[U];
    if constexpr (PER > 0) {
      float4 q[8];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int64_t u = ub + k * GPW + gi;
        const bool ok = u < n_units;
        const float4* p = unit_ptr(ok ? u : 0);
#pragma unroll
        for (int e = 0; e < PER; ++e) q[k * PER + e] = ok ? __ldcs(p + e * G) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      FF t[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) t[j] = sum4(q[j]);
#pragma unroll
      for (int w = 1; w < PER; w <<= 1)
#pragma unroll
        for (int j = 0; j < 8; j += 2 * w) t[j] = ff_add(t[j], t[j + w]);
#pragma unroll
      for (int k = 0; k < U; ++k) acc[k] = t[k * PER];
    } else {
      const int64_t u = ub + gi;
      acc[0] = FF{0.0f, 0.0f};
      if (u < n_units) {
        const float4* p = unit_ptr(u);
        for (int64_t j0 = 0; j0 < per; j0 += 8) {   // per is a power of two >= 16 here
          float4 q[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) q[j] = __ldcs(p + (j0 + j) * G);
          FF t[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) t[j] = sum4(q[j]);
#pragma unroll
          for (int w = 4; w > 0; w >>= 1)
#pragma unroll
            for (int j = 0; j < w; ++j) t[j] = ff_add(t[j], t[j + w]);
          acc[0] = ff_add(acc[0], t[0]);
        }
      }
    }
    // across the group
#pragma unroll
    for (int off = 1; off < G; off <<= 1) {
#pragma unroll
      for (int k = 0; k < U; ++k) acc[k] = ff_add(acc[k], ff_shfl_xor(acc[k], off));
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t u = ub + k * GPW + gi;
      if (gl == 0 && u < n_units) {
        if (lnch == 0)
          store_merged(out, outc, u, acc[k]);
        else
          part[u] = make_float2(acc[k].s, acc[k].c);
      }
    }
  }
}

// Merged qubits below index bit T with R = 1 or 2 kept bits among them (T =
// mg + R; e.g. a subcircuit's measured cut qubits between merged outputs, or
// just below them): the 2^R outputs that differ only in those kept bits sum
// the values of one contiguous block of 2^T values, output l taking the
// values whose kept bits below T read l.  A group of G = min(32, 2^(T - 2))
// lanes owns such a unit and reads its block with 16-byte loads (lane j takes
// float4 j, j + G, ..., 8 in flight).  Within a float4 the kept bits among
// index bits 0-1 (`lo`) pair its components into one, two or four partial
// sums; the kept bits at or above bit 2 are bits `hb0`, `hb1` of the float4's
// index (-1: none) and pick the output; every output keeps its own
// compensated sum (TwoSum), adding zero where a partial sum is another
// output's (exact), as in the contiguous-run form.
template <int R>
__global__ void k_dd_merge_blk(const float* __restrict__ Tin, int64_t cols, int a, int T, int lo, int hb0, int hb1,
                               const uint64_t* __restrict__ depAct, int nbA, uint64_t zoom, float* __restrict__ out,
                               float* __restrict__ outc, int64_t n_units) {
  constexpr int NO = 1 << R;
  const int64_t F = int64_t(1) << (T - 2);      // float4 per block
  const int G = F < 32 ? (int)F : 32;
  const int64_t per = F / G;                    // float4 per lane
  const int lane = threadIdx.x & 31, gl = lane & (G - 1), gi = lane / G, upw = 32 / G;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t amask = (uint64_t(1) << a) - 1;
  const int nlo = __popc(lo);                   // kept bits among index bits 0-1
  // every lane of a warp runs the same number of steps (shuffles below)
  for (int64_t ub = warp * upw; ub < n_units; ub += nwarps * upw) {
    const int64_t u = ub + gi;
    const bool ok = u < n_units;
    const int64_t o0 = (ok ? u : 0) << R;       // the unit's first output (its R lowest kept bits zero)
    const uint64_t xa = (uint64_t)o0 & amask;
    const float4* p =
        reinterpret_cast<const float4*>(Tin + (o0 >> a) * cols + (dep_tab(depAct, nbA, xa) | zoom)) + gl;
    FF acc[NO];
#pragma unroll
    for (int l = 0; l < NO; ++l) acc[l] = FF{0.0f, 0.0f};
    if (ok) {
      for (int64_t j0 = 0; j0 < per; j0 += 8) {
        float4 q[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) q[e] = j0 + e < per ? __ldcs(p + (j0 + e) * G) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int64_t f = gl + (j0 + e) * G;  // the float4's index in the block
          const int lh = (hb0 >= 0 ? (int)((f >> hb0) & 1) : 0) | (hb1 >= 0 ? (int)((f >> hb1) & 1) << 1 : 0);
          FF ps[4];
          if (lo == 0) {
            ps[0] = sum4(q[e]);
          } else if (lo == 1) {        // index bit 0 kept: (x, z) and (y, w)
            ps[0] = ff_add(FF{q[e].x, 0.0f}, FF{q[e].z, 0.0f});
            ps[1] = ff_add(FF{q[e].y, 0.0f}, FF{q[e].w, 0.0f});
          } else if (lo == 2) {        // index bit 1 kept: (x, y) and (z, w)
            ps[0] = ff_add(FF{q[e].x, 0.0f}, FF{q[e].y, 0.0f});
            ps[1] = ff_add(FF{q[e].z, 0.0f}, FF{q[e].w, 0.0f});
          } else {                     // both kept: one output per component
            ps[0] = FF{q[e].x, 0.0f};
            ps[1] = FF{q[e].y, 0.0f};
            ps[2] = FF{q[e].z, 0.0f};
            ps[3] = FF{q[e].w, 0.0f};
          }
#pragma unroll
          for (int k = 0; k < NO; ++k) {
            // output k takes partial sum k mod 2^nlo when its higher kept bits read lh
            const int i = k & ((1 << nlo) - 1);
            const FF v = ps[i < (1 << nlo) ? i : 0];
            acc[k] = ff_add(acc[k], (k >> nlo) == lh ? v : FF{0.0f, 0.0f});
          }
        }
      }
    }
    for (int off = 1; off < G; off <<= 1)
#pragma unroll
      for (int l = 0; l < NO; ++l) acc[l] = ff_add(acc[l], ff_shfl_xor(acc[l], off));
    if (ok && gl == 0)
#pragma unroll
      for (int l = 0; l < NO; ++l) store_merged(out, outc, o0 + l, acc[l]);
  }
}

// warp per output: lanes take chunks lane, lane + 32, ... of its partial sums
__global__ void k_dd_merge_finish(const float2* __restrict__ part, int lnch, float* __restrict__ out,
                                  float* __restrict__ outc, int64_t n_out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nch = int64_t(1) << lnch;
  for (int64_t o = warp; o < n_out; o += nwarps) {
    FF acc{};
    for (int64_t c = lane; c < nch; c += 32) {
      const float2 v = part[(o << lnch) + c];
      acc = ff_add(acc, FF{v.x, v.y});
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = ff_add(acc, ff_shfl_xor(acc, off));
    if (lane == 0) store_merged(out, outc, o, acc);
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

// FP32 bins, 16-byte aligned, n a multiple of 4: each lane loads 4 float4 per
// step (512 consecutive values per warp), candidates filtered by the exact (value, index)
// order so the insertion order does not matter; at the end warp 0 of each
// block merges its warps' lists, so one list of KC per block is written.
__global__ void k_topk_warps4(const float4* __restrict__ bins4, int64_t n, int64_t per_warp,
                              float* __restrict__ cv, int64_t* __restrict__ ci) {
  __shared__ float sv[8 * KC];
  __shared__ int64_t si[8 * KC];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  float lv = -FLT_MAX;
  int64_t li = INT64_MAX;
  const int64_t lo = warp * per_warp, hi = min(n, lo + per_warp);
  for (int64_t b0 = lo; b0 < hi; b0 += 512) {
    float v[16];
    int64_t i0[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      i0[h] = b0 + 128 * h + 4 * lane;
      const float4 q = i0[h] < hi ? __ldcs(bins4 + (i0[h] >> 2)) : make_float4(-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX);
      v[4 * h + 0] = q.x;
      v[4 * h + 1] = q.y;
      v[4 * h + 2] = q.z;
      v[4 * h + 3] = q.w;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int64_t i = i0[u >> 2] + (u & 3);
      const float tv = __shfl_sync(0xffffffffu, lv, 31);
      const int64_t ti = __shfl_sync(0xffffffffu, li, 31);
      unsigned m = __ballot_sync(0xffffffffu, i < hi && before(v[u], i, tv, ti));
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        warp_insert(lv, li, __shfl_sync(0xffffffffu, v[u], src), __shfl_sync(0xffffffffu, i, src), lane);
      }
    }
  }
  sv[w * KC + lane] = lv;
  si[w * KC + lane] = li;
  __syncthreads();
  if (w == 0) {
    lv = -FLT_MAX;
    li = INT64_MAX;
    for (int j0 = 0; j0 < (int)(blockDim.x >> 5) * KC; j0 += 32) {
      const float v = sv[j0 + lane];
      const int64_t idx = si[j0 + lane];
      unsigned m = __ballot_sync(0xffffffffu, before(v, idx, __shfl_sync(0xffffffffu, lv, 31),
                                                      __shfl_sync(0xffffffffu, li, 31)));
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        warp_insert(lv, li, __shfl_sync(0xffffffffu, v, src), __shfl_sync(0xffffffffu, idx, src), lane);
      }
    }
    cv[(int64_t)blockIdx.x * KC + lane] = lv;
    ci[(int64_t)blockIdx.x * KC + lane] = li;
  }
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
// M64[cand][c][row] = the merged value of subcircuit c at the candidate's
// active bits in FP64: the FP64 merged tensor, or for FP32 tensors the merge's
// rounded sum plus its compensation term.  grid: (cand, c).
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
  for (int64_t row = threadIdx.x; row < s.rows; row += blockDim.x) {
    const int64_t i = (row << s.a) + xa;
    m64[((int64_t)cand * a.n_sub + c) * a.max_rows + row] =
        a.f64 ? static_cast<const double*>(s.m)[i] : (double)static_cast<const float*>(s.m)[i] + (double)s.mc[i];
  }
}

// part[cand][chunk] = sum over the chunk's terms e of prod_c M64[cand][c][row_c(e)];
// grid: (cand, chunk), block 256.  k_dd_eval_final adds the chunks in order and
// scales by 2^-K.
__global__ void k_dd_eval(const DdEvalArgs a, const double* __restrict__ m64, int nchunk,
                          double* __restrict__ part) {
  const int cand = blockIdx.x, chunk = blockIdx.y;
  __shared__ double red[8];
  const int64_t nterms = int64_t(1) << (2 * a.n_cuts);
  const int64_t per = nterms / nchunk;
  double acc = 0.0;
  for (int64_t e = chunk * per + threadIdx.x; e < (chunk + 1) * per; e += blockDim.x) {
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
    part[cand * nchunk + chunk] = tot;
  }
}

__global__ void k_dd_eval_final(const double* __restrict__ part, int n_cand, int nchunk, double scale,
                                double* __restrict__ val) {
  const int cand = threadIdx.x;
  if (cand >= n_cand) return;
  double tot = 0.0;
  for (int c = 0; c < nchunk; ++c) tot += part[cand * nchunk + c];
  val[cand] = tot * scale;
}

unsigned grid_for(int64_t work, int per_block) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int G, int PER>
void launch_run(const float* T, int64_t cols, int a, int mg, const uint64_t* depAct, int nbA, uint64_t zoom,
                int dense, int lnch, float* M, float* MC, float2* part, int64_t n_out, cudaStream_t s) {
  constexpr int U = PER == 0 ? 1 : 8 / PER;
  const int64_t threads = ((n_out << lnch) + U - 1) / U * G;
  k_dd_merge_run<G, PER><<<grid_for(threads, 256), 256, 0, s>>>(T, cols, a, mg, depAct, nbA, zoom, dense, lnch, M,
                                                                 MC, part, n_out);
}

// deposit tables built on the device from up to 32 bit values each (passed
// by value): table[b][v] = sum over set bits j of v of bits[8b + j]; a table
// for n bits has max(ceil(n / 8), 1) rows of 256
struct DepBits {
  uint64_t v[32];
  int n;
};
__global__ void k_deposit_tables(const DepBits A, const DepBits M, uint64_t* __restrict__ ta,
                                 uint64_t* __restrict__ tm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;   // (table, byte, v)
  const int nbA = max((A.n + 7) / 8, 1), nbM = max((M.n + 7) / 8, 1);
  const bool first = t < nbA * 256;
  const int i = first ? t : t - nbA * 256;
  if (!first && i >= nbM * 256) return;
  const int n = first ? A.n : M.n;
  const int b = i >> 8, v = i & 255;
  uint64_t g = 0;
  for (int j = 0; j < 8; ++j)
    if (((v >> j) & 1) && 8 * b + j < n) g += first ? A.v[8 * b + j] : M.v[8 * b + j];
  (first ? ta : tm)[i] = g;
}

}  // namespace

void launch_deposit_tables(const uint64_t* act, int na, const uint64_t* mrg, int nm, uint64_t* tab_act,
                           uint64_t* tab_mrg, cudaStream_t s) {
  if (na < 0 || na > 32 || nm < 0 || nm > 32) fail(CUTQC_ERR_UNSUPPORTED, "deposit tables take at most 32 bits");
  DepBits A{}, M{};
  for (int j = 0; j < na; ++j) A.v[j] = act[j];
  for (int j = 0; j < nm; ++j) M.v[j] = mrg[j];
  A.n = na;
  M.n = nm;
  const int total = (std::max((na + 7) / 8, 1) + std::max((nm + 7) / 8, 1)) * 256;
  k_deposit_tables<<<(total + 255) / 256, 256, 0, s>>>(A, M, tab_act, tab_mrg);
  count_launch();
  check_launch("k_deposit_tables");
}

uint64_t dd_merge_block(uint64_t merged_mask, int mg, uint64_t active_mask, uint64_t zoom) {
  if (mg <= 0 || merged_mask == 0) return 0;
  const int T = 64 - __builtin_clzll(merged_mask);   // the highest merged bit + 1
  if (T > 40) return 0;
  const uint64_t below = (uint64_t(1) << T) - 1;
  const uint64_t kept = active_mask & below;
  const int R = __builtin_popcountll(kept);
  // every bit below T merged or kept, none zoomed, at most two kept
  if (R < 1 || R > 2 || (zoom & below) || ((merged_mask | kept) != below) || T != mg + R) return 0;
  return kept;
}

int dd_merge_chunks(int64_t rows, int a, int mg) {
  if (mg < 2) return 0;
  const int64_t ng = int64_t(1) << (mg - 2), G = std::min<int64_t>(32, ng), n_out = rows << a;
  int lnch = 0;
  while ((n_out << lnch) * G < 152 * 2048 && (ng >> (lnch + 1)) >= 8 * G) ++lnch;
  return lnch;
}

void launch_dd_merge(const void* T_, int dtype, int64_t rows, int f, int a, int mg, const uint64_t* depAct,
                     const uint64_t* depMrg, uint64_t zoom, bool run, bool dense_bits, void* M, float* MC,
                     void* part, cudaStream_t s, uint64_t blk) {
  const void* T = T_;
  const int64_t n_out = rows << a;
  const int64_t cols = int64_t(1) << f;
  const int nbA = (a + 7) / 8, nbM = (mg + 7) / 8;
  run = run && dtype == CUTQC_F32 && mg >= 2 && (reinterpret_cast<uintptr_t>(T) & 15) == 0;
  // the block form needs its kept bits below T described (`blk`), whole
  // float4 blocks and enough units to fill the GPU (otherwise the warp form
  // below, a warp per output)
  const int R = blk ? __builtin_popcountll(blk) : 0;
  const int TB = mg + R;   // log2 of the block
  bool block = !run && (R == 1 || R == 2) && dtype == CUTQC_F32 && TB >= 2 && TB <= 40 &&
               (reinterpret_cast<uintptr_t>(T_) & 15) == 0 &&
               (n_out >> R) * std::min<int64_t>(32, int64_t(1) << (TB - 2)) >= 152 * 256;
  if (block) {
    const int64_t n_units = n_out >> R;
    const int64_t lanes = n_units * std::min<int64_t>(32, int64_t(1) << (TB - 2));
    const int lo = (int)(blk & 3);
    int hb[2] = {-1, -1}, nh = 0;
    for (int bit = 2; bit < TB; ++bit)
      if ((blk >> bit) & 1) hb[nh++] = bit - 2;
    const float* Tf = static_cast<const float*>(T_);
    float* Mf = static_cast<float*>(M);
    if (R == 2)
      k_dd_merge_blk<2><<<grid_for(lanes, 256), 256, 0, s>>>(Tf, cols, a, TB, lo, hb[0], hb[1], depAct, nbA, zoom, Mf,
                                                             MC, n_units);
    else
      k_dd_merge_blk<1><<<grid_for(lanes, 256), 256, 0, s>>>(Tf, cols, a, TB, lo, hb[0], hb[1], depAct, nbA, zoom, Mf,
                                                             MC, n_units);
  } else if (run) {
    const int lnch = dd_merge_chunks(rows, a, mg);
    const int dense = dense_bits ? 1 : 0;
    const float* Tf = static_cast<const float*>(T);
    float* Mf = static_cast<float*>(M);
    float2* pf = static_cast<float2*>(part);
    const int G = std::min(32, 1 << std::min(mg - 2, 5));
    const int64_t per = (int64_t(1) << (mg - 2 - lnch)) / G;
#define CUTQC_RUN(g, q) launch_run<g, q>(Tf, cols, a, mg, depAct, nbA, zoom, dense, lnch, Mf, MC, pf, n_out, s)
    if (G < 32) {
      switch (G) {
        case 1: CUTQC_RUN(1, 1); break;
        case 2: CUTQC_RUN(2, 1); break;
        case 4: CUTQC_RUN(4, 1); break;
        case 8: CUTQC_RUN(8, 1); break;
        default: CUTQC_RUN(16, 1); break;
      }
    } else {
      switch (per) {
        case 1: CUTQC_RUN(32, 1); break;
        case 2: CUTQC_RUN(32, 2); break;
        case 4: CUTQC_RUN(32, 4); break;
        case 8: CUTQC_RUN(32, 8); break;
        default: CUTQC_RUN(32, 0); break;
      }
    }
#undef CUTQC_RUN
    if (lnch > 0) {
      count_launch();
      check_launch("k_dd_merge_run");
      k_dd_merge_finish<<<grid_for(n_out * 32, 256), 256, 0, s>>>(pf, lnch, Mf, MC, n_out);
    }
  } else if (mg >= 5) {
    const unsigned g = grid_for(n_out * 32, 256);
    if (dtype == CUTQC_F64)
      k_dd_merge_warp<double><<<g, 256, 0, s>>>(static_cast<const double*>(T), cols, a, mg, depAct, nbA, depMrg, nbM,
                                                zoom, static_cast<double*>(M), nullptr, n_out);
    else
      k_dd_merge_warp<float><<<g, 256, 0, s>>>(static_cast<const float*>(T), cols, a, mg, depAct, nbA, depMrg, nbM,
                                               zoom, static_cast<float*>(M), MC, n_out);
  } else {
    const unsigned g = grid_for(n_out, 256);
    if (dtype == CUTQC_F64)
      k_dd_merge_thread<double><<<g, 256, 0, s>>>(static_cast<const double*>(T), cols, a, mg, depAct, nbA, depMrg,
                                                  nbM, zoom, static_cast<double*>(M), nullptr, n_out);
    else
      k_dd_merge_thread<float><<<g, 256, 0, s>>>(static_cast<const float*>(T), cols, a, mg, depAct, nbA, depMrg, nbM,
                                                 zoom, static_cast<float*>(M), MC, n_out);
  }
  count_launch();
  check_launch("k_dd_merge");
}

size_t topk_workspace_bytes(int64_t n) {
  const int64_t warps = 152 * 8 * 4;
  return (size_t)warps * KC * (4 + 8) + 256;
}

void launch_topk(const void* bins, int dtype, int64_t n, void* ws, float* out_v, int64_t* out_i, cudaStream_t s) {
  const int64_t lists_max = 152 * 8 * 4;   // capacity of the workspace in lists of KC
  float* cv = static_cast<float*>(ws);
  int64_t* ci = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + (size_t)lists_max * KC * 4);
  int64_t lists;
  if (dtype == CUTQC_F32 && n % 4 == 0 && (reinterpret_cast<uintptr_t>(bins) & 15) == 0) {
    // up to 64 warps per SM, one list per block of 8 warps
    const int64_t warps_max = 152 * 64;
    int64_t per_warp = ((n + warps_max - 1) / warps_max + 511) / 512 * 512;
    const int64_t warps = (n + per_warp - 1) / per_warp;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    k_topk_warps4<<<blocks, 256, 0, s>>>(static_cast<const float4*>(bins), n, per_warp, cv, ci);
    lists = blocks;
  } else {
    const int64_t warps_max = lists_max;
    int64_t per_warp = ((n + warps_max - 1) / warps_max + 127) / 128 * 128;
    if (per_warp < 128) per_warp = 128;
    const int64_t warps = (n + per_warp - 1) / per_warp;
    const unsigned blocks = (unsigned)((warps + 7) / 8);
    if (dtype == CUTQC_F64)
      k_topk_warps<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(bins), n, per_warp, cv, ci);
    else
      k_topk_warps<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(bins), n, per_warp, cv, ci);
    lists = (int64_t)blocks * 8;
  }
  count_launch();
  check_launch("k_topk_warps");
  k_topk_final<<<1, 1024, 0, s>>>(cv, ci, lists * KC, out_v, out_i);
  count_launch();
  check_launch("k_topk_final");
}

void launch_topk_lists(void* ws, int64_t nlists, float* out_v, int64_t* out_i, cudaStream_t s) {
  const int64_t lists_max = 152 * 8 * 4;
  if (nlists > lists_max) fail(CUTQC_ERR_UNSUPPORTED, "too many candidate lists");
  float* cv = static_cast<float*>(ws);
  int64_t* ci = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + (size_t)lists_max * KC * 4);
  k_topk_final<<<1, 1024, 0, s>>>(cv, ci, nlists * KC, out_v, out_i);
  count_launch();
  check_launch("k_topk_final");
}

int dd_eval_chunks(int n_cuts) {
  const int64_t nterms = int64_t(1) << (2 * n_cuts);
  int64_t c = nterms / 2048;
  return (int)std::max<int64_t>(1, std::min<int64_t>(64, c));
}

void launch_dd_rerank(const DdEvalArgs& a, int dtype, double* m64, double* part, double* val, cudaStream_t s) {
  k_dd_gather64<<<dim3(a.n_cand, a.n_sub), 256, 0, s>>>(a, m64);
  count_launch();
  check_launch("k_dd_gather64");
  const int nchunk = dd_eval_chunks(a.n_cuts);
  k_dd_eval<<<dim3(a.n_cand, nchunk), 256, 0, s>>>(a, m64, nchunk, part);
  count_launch();
  check_launch("k_dd_eval");
  k_dd_eval_final<<<1, 32, 0, s>>>(part, a.n_cand, nchunk, a.scale, val);
  count_launch();
  check_launch("k_dd_eval_final");
}

}  // namespace cutqc

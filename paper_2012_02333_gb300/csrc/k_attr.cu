// Attribution of measured variant distributions (Sec. 3.2.2, Eq. 2 and Eq. 3).
//
// A subcircuit with k_in init slots and k_out measurement slots is run in
// 4^k_in x 3^k_out physical variants (Fig. 3: every init slot prepared in
// |0>, |1>, |+>, |+i>; every measured cut qubit measured in the Z, X or Y
// basis).  Given the measured output distribution of every variant (from a
// device's shot counts or from simulation), the Pauli-indexed tensor is
//
//   T[a][b][x] = sum_s C(a, s) sum_m W(b, m) p_s,mb(b)(y(x, m))
//
// with, per slot, C the Eq. 2 coefficients (I = |0><0| + |1><1|,
// Z = |0><0| - |1><1|, X = 2|+><+| - I, Y = 2|+i><+i| - I), mb(b) the basis
// that serves Pauli b (I and Z: the Z-basis circuit, X: X, Y: Y), W the Eq. 3
// factor of outcome m (basis I: +1 for both outcomes; X, Y, Z: 0 -> +1,
// 1 -> -1), and y(x, m) the subcircuit's local bit string holding the output
// bits x and the measured cut-qubit outcomes m.
//
// Two streaming passes over memory, no scratch (a single-pass form that
// applies both equations per output was measured slower: its threads each
// hold all inits of one basis combination, too few to keep the loads in
// flight): k_attr_outcomes applies Eq. 3
// (one thread per (s, b, x): the 2^k_out outcomes of the variant that serves
// b, read where consecutive threads take consecutive x) and writes the
// result into the output buffer; k_attr_inits then applies Eq. 2 in place
// (one thread per (b, x) holding the 4^k_in values of all physical inits in
// registers and combining them slot by slot into the Pauli operators).  With
// more than 3 init slots (4^k_in values no longer fit in registers) a single
// kernel does both per entry.  FP64 inputs sum in FP64; FP32 inputs in
// compensated FP32 (TwoSum), the FP64 pipe being narrow on this part.
// Entries below 2^-40 in magnitude become exactly 0, as at input preparation
// (they are rounding residue of terms that vanish exactly).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>

#include "internal.h"

namespace cutqc {

namespace {

struct AttrArgs {
  int d, k_in, k_out, n_eff;
  int meas_pos[12];   // bit of y (from the least significant) holding measurement slot j
  int out_pos[32];    // bit of y holding output i (output 0 = most significant bit of x)
  int64_t pow3_kout;
};

struct FF {
  float s, c;
};
__device__ __forceinline__ FF ff_add(FF a, float b) {
  const float s = a.s + b;
  const float bb = s - a.s;
  const float err = (a.s - (s - bb)) + (b - bb);
  return {s, a.c + err};
}

// |r| < 2^-40 -> 0, compared in the entry's own type (2^-40 is exact in both)
__device__ __forceinline__ float snap_small(float r) { return fabsf(r) < 9.094947017729282e-13f ? 0.0f : r; }
__device__ __forceinline__ double snap_small(double r) { return fabs(r) < 9.094947017729282e-13 ? 0.0 : r; }

// Eq. 2: physical inits (0 = |0>, 1 = |1>, 2 = |+>, 3 = |+i>) with non-zero
// coefficient in Pauli a (0 = I, 1 = X, 2 = Y, 3 = Z)
__device__ __forceinline__ int init_terms(int pauli, int (&s)[3], float (&c)[3]) {
  switch (pauli) {
    case 0: s[0] = 0; c[0] = 1.f; s[1] = 1; c[1] = 1.f; return 2;
    case 1: s[0] = 0; c[0] = -1.f; s[1] = 1; c[1] = -1.f; s[2] = 2; c[2] = 2.f; return 3;
    case 2: s[0] = 0; c[0] = -1.f; s[1] = 1; c[1] = -1.f; s[2] = 3; c[2] = 2.f; return 3;
    default: s[0] = 0; c[0] = 1.f; s[1] = 1; c[1] = -1.f; return 2;
  }
}

template <typename T>
__global__ void k_attribute(const T* __restrict__ P, const AttrArgs a, T* __restrict__ out, int64_t n_out) {
  const int f = a.n_eff;
  const int64_t nb = int64_t(1) << (2 * a.k_out);
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_out; o += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t x = (uint64_t)o & ((uint64_t(1) << f) - 1);
    const int64_t rest = o >> f;
    const int64_t b = rest & (nb - 1), av = rest >> (2 * a.k_out);
    // the output bits' place in y
    uint64_t yx = 0;
    for (int i = 0; i < f; ++i) yx |= ((x >> (f - 1 - i)) & 1) << a.out_pos[i];
    // Eq. 3: the basis each measurement slot was measured in, and which slots sign their outcome
    int64_t mb = 0;
    unsigned signed_slots = 0;
    for (int j = 0; j < a.k_out; ++j) {
      const int bj = (int)((b >> (2 * (a.k_out - 1 - j))) & 3);
      mb = 3 * mb + (bj == 1 ? 1 : bj == 2 ? 2 : 0);
      if (bj != 0) signed_slots |= 1u << j;
    }
    // Eq. 2: per init slot the physical inits that contribute, as an odometer
    int ns[12], idx[12], sj[12][3];
    float cj[12][3];
    for (int j = 0; j < a.k_in; ++j) {
      const int aj = (int)((av >> (2 * (a.k_in - 1 - j))) & 3);
      int s3[3];
      float c3[3];
      ns[j] = init_terms(aj, s3, c3);
      for (int t = 0; t < 3; ++t) {
        sj[j][t] = s3[t];
        cj[j][t] = c3[t];
      }
      idx[j] = 0;
    }
    using Acc = typename std::conditional<sizeof(T) == 8, double, FF>::type;
    Acc acc{};
    for (;;) {
      int64_t s = 0;
      float coef = 1.f;
      for (int j = 0; j < a.k_in; ++j) {
        s = 4 * s + sj[j][idx[j]];
        coef *= cj[j][idx[j]];
      }
      const T* base = P + ((s * a.pow3_kout + mb) << a.d);
      for (uint32_t m = 0; m < (1u << a.k_out); ++m) {
        uint64_t y = yx;
        for (int j = 0; j < a.k_out; ++j) y |= (uint64_t)((m >> j) & 1) << a.meas_pos[j];
        const float sign = (__popc(m & signed_slots) & 1) ? -1.f : 1.f;
        const T v = __ldg(base + y) * (T)(coef * sign);
        if constexpr (sizeof(T) == 8)
          acc += v;
        else
          acc = ff_add(acc, v);
      }
      int j = a.k_in - 1;
      while (j >= 0 && ++idx[j] == ns[j]) idx[j--] = 0;
      if (j < 0) break;
    }
    T r;
    if constexpr (sizeof(T) == 8)
      r = acc;
    else
      r = acc.s + acc.c;
    out[o] = snap_small(r);
  }
}

// Eq. 3: Q[s][b][x] = sum_m W(b, m) P[s][mb(b)][y(x, m)]; snap when it is final.
// y(x, m) comes from per-block shared tables: for each byte of x and of m, the
// bits of y its set bits stand for (the deposit is additive over bytes).
template <typename T>
__device__ __forceinline__ void fill_tables(const AttrArgs& a, uint64_t (&tab_x)[4][256], uint64_t (&tab_m)[2][256]) {
  const int f = a.n_eff;
  for (int i = threadIdx.x; i < 6 * 256; i += blockDim.x) {
    const int t = i >> 8, v = i & 255;
    uint64_t dep = 0;
    for (int k = 0; k < 8; ++k) {
      if (!((v >> k) & 1)) continue;
      if (t < 4) {
        const int xb = 8 * t + k;                       // bit of x, from the least significant
        if (xb < f) dep |= uint64_t(1) << a.out_pos[f - 1 - xb];
      } else {
        const int slot = 8 * (t - 4) + k;               // bit of m = measurement slot
        if (slot < a.k_out) dep |= uint64_t(1) << a.meas_pos[slot];
      }
    }
    if (t < 4)
      tab_x[t][v] = dep;
    else
      tab_m[t - 4][v] = dep;
  }
  __syncthreads();
}

// the Eq. 3 basis and sign pattern of Pauli row b
__device__ __forceinline__ void basis_of(uint32_t b, int k_out, int64_t& mb, unsigned& signed_slots) {
  mb = 0;
  signed_slots = 0;
  for (int j = 0; j < k_out; ++j) {
    const int bj = (int)((b >> (2 * (k_out - 1 - j))) & 3);
    mb = 3 * mb + (bj == 1 ? 1 : bj == 2 ? 2 : 0);
    if (bj != 0) signed_slots |= 1u << j;
  }
}

// G consecutive x per thread (G = 4 when n_eff >= 2): the index arithmetic and
// the table lookups are shared, and with VEC (FP32, the two lowest output bits
// on the two lowest local bits, aligned buffers) each outcome is one 16-byte
// load and each result one 16-byte store.
template <typename T, int G, bool VEC>
__global__ void k_attr_outcomes(const T* __restrict__ P, const AttrArgs a, T* __restrict__ Q, int64_t n_out,
                                int snap) {
  __shared__ uint64_t tab_x[4][256];
  __shared__ uint64_t tab_m[2][256];
  fill_tables<T>(a, tab_x, tab_m);
  const int f = a.n_eff;
  const int lg_nb = 2 * a.k_out;
  const int64_t n_grp = n_out / G;
  uint64_t dlow[G];
#pragma unroll
  for (int k = 0; k < G; ++k) dlow[k] = tab_x[0][k];
  for (int64_t og = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; og < n_grp;
       og += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = og * G;
    const uint32_t x = (uint32_t)((uint64_t)o & ((uint64_t(1) << f) - 1));
    const int64_t rest = o >> f;
    const uint32_t b = (uint32_t)(rest & ((int64_t(1) << lg_nb) - 1));
    const int64_t sv = rest >> lg_nb;
    const uint64_t yx = tab_x[0][x & 255] | tab_x[1][(x >> 8) & 255] | tab_x[2][(x >> 16) & 255] | tab_x[3][x >> 24];
    int64_t mb;
    unsigned signed_slots;
    basis_of(b, a.k_out, mb, signed_slots);
    const T* base = P + ((sv * a.pow3_kout + mb) << a.d) + yx;
    using Acc = typename std::conditional<sizeof(T) == 8, double, FF>::type;
    Acc acc[G];
#pragma unroll
    for (int k = 0; k < G; ++k) acc[k] = Acc{};
    for (uint32_t m = 0; m < (1u << a.k_out); ++m) {
      const T* pm = base + (tab_m[0][m & 255] | tab_m[1][m >> 8]);
      const bool neg = __popc(m & signed_slots) & 1;
      T v[G];
      if constexpr (VEC) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(pm));
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
      } else {
#pragma unroll
        for (int k = 0; k < G; ++k) v[k] = __ldg(pm + dlow[k]);
      }
#pragma unroll
      for (int k = 0; k < G; ++k) {
        const T t = neg ? -v[k] : v[k];
        if constexpr (sizeof(T) == 8)
          acc[k] += t;
        else
          acc[k] = ff_add(acc[k], t);
      }
    }
    T r[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
      if constexpr (sizeof(T) == 8)
        r[k] = acc[k];
      else
        r[k] = acc[k].s + acc[k].c;
      if (snap) r[k] = snap_small(r[k]);
    }
    if constexpr (VEC) {
      *reinterpret_cast<float4*>(Q + o) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
#pragma unroll
      for (int k = 0; k < G; ++k) Q[o + k] = r[k];
    }
  }
}

// Eq. 3, variant-centred (k_out <= 4, n_eff >= 2): one thread per (variant s,
// basis combination mb, 4 consecutive x) loads the 4 * 2^KOUT outcomes of
// that variant once and takes, by a Walsh-Hadamard butterfly over the slots,
// every signed sum sum_m (-1)^{popc(m & p)} v[m] at once; then it writes the
// rows b that mb serves (a Z-basis slot serves I, unsigned, and Z, signed;
// X and Y serve themselves), 4 consecutive x per 16-byte store.  P is read
// exactly once.  The butterfly's adds are pairwise over at most 16 values.
// CONTIG (FP32, k_out <= 2, aligned): the measured cut qubits are the lowest
// local bits, in any order, and x bits 0-1 sit right above them, so a
// thread's 4 * 2^KOUT values are contiguous: 2^KOUT 16-byte loads, each value
// then picked by its measured-bit offset (a select over 2^KOUT registers).
template <typename T, int KOUT, bool CONTIG>
__global__ void k_attr_variants(const T* __restrict__ P, const AttrArgs a, T* __restrict__ Q, int64_t n_grp,
                                int snap) {
  __shared__ uint64_t tab_x[4][256];
  __shared__ uint64_t tab_m[2][256];
  fill_tables<T>(a, tab_x, tab_m);
  constexpr int NM = 1 << KOUT;
  const int f = a.n_eff;
  const int lg_xg = f - 2;
  uint64_t dlow[4], dm[NM];
#pragma unroll
  for (int k = 0; k < 4; ++k) dlow[k] = tab_x[0][k];
#pragma unroll
  for (int m = 0; m < NM; ++m) dm[m] = tab_m[0][m];
  // the first outcome of group g (4 consecutive x of one variant row)
  auto group_base = [&](int64_t g) {
    const uint32_t gx = (uint32_t)(g & ((int64_t(1) << lg_xg) - 1)) << 2;
    const uint64_t yx =
        tab_x[0][gx & 255] | tab_x[1][(gx >> 8) & 255] | tab_x[2][(gx >> 16) & 255] | tab_x[3][gx >> 24];
    return P + ((int64_t)(g >> lg_xg) << a.d) + yx;
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t og = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // CONTIG: the next group's 2^KOUT 16-byte loads are in flight while the
  // current one is processed (the grid is one wave of resident blocks, so a
  // thread takes several groups)
  float4 nxt[CONTIG ? NM : 1];
  if constexpr (CONTIG) {
    if (og < n_grp) {
      const float4* b4 = reinterpret_cast<const float4*>(group_base(og));
#pragma unroll
      for (int j = 0; j < NM; ++j) nxt[j] = __ldg(b4 + j);
    }
  }
  for (; og < n_grp; og += stride) {
    const uint32_t x = (uint32_t)(og & ((int64_t(1) << lg_xg) - 1)) << 2;
    const uint32_t rest = (uint32_t)(og >> lg_xg);          // s * 3^KOUT + mb
    const uint32_t sv = rest / (uint32_t)a.pow3_kout, mb = rest - sv * (uint32_t)a.pow3_kout;
    T v[NM][4];
    if constexpr (CONTIG) {
      // entry e of the 4 * NM contiguous values is measured offset e % NM
      // (dm[m] for outcome m) of output x + e / NM
      T w[4 * NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        const float4 q = nxt[j];
        w[4 * j] = q.x;
        w[4 * j + 1] = q.y;
        w[4 * j + 2] = q.z;
        w[4 * j + 3] = q.w;
      }
      if (og + stride < n_grp) {
        const float4* b4 = reinterpret_cast<const float4*>(group_base(og + stride));
#pragma unroll
        for (int j = 0; j < NM; ++j) nxt[j] = __ldg(b4 + j);
      }
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const int o = (int)dm[m];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          T r = w[NM * k];
#pragma unroll
          for (int t = 1; t < NM; ++t) r = o == t ? w[NM * k + t] : r;
          v[m][k] = r;
        }
      }
    } else {
      const T* base = group_base(og);
#pragma unroll
      for (int m = 0; m < NM; ++m)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[m][k] = __ldg(base + dm[m] + dlow[k]);
    }
    // butterfly over slot j (m bit j): (u, w) -> (u + w, u - w); afterwards
    // v[p] = sum_m (-1)^{popc(m & p)} v_in[m]
#pragma unroll
    for (int j = 0; j < KOUT; ++j)
#pragma unroll
      for (int m = 0; m < NM; ++m)
        if (!((m >> j) & 1))
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const T u = v[m][k], w = v[m | (1 << j)][k];
            v[m][k] = u + w;
            v[m | (1 << j)][k] = u - w;
          }
    // basis digit of every slot (slot 0 = most significant base-3 digit)
    int dig[KOUT > 0 ? KOUT : 1];
    {
      uint32_t r = mb;
#pragma unroll
      for (int j = KOUT - 1; j >= 0; --j) {
        dig[j] = (int)(r % 3);
        r /= 3;
      }
    }
    // sign pattern p (bit j: slot j signed) serves one row when every
    // unsigned slot was measured in the Z basis (it is then I); a signed slot
    // is Z, X or Y by its basis
#pragma unroll
    for (int p = 0; p < NM; ++p) {
      bool valid = true;
      uint32_t b = 0;
#pragma unroll
      for (int j = 0; j < KOUT; ++j) {
        int pauli;
        if (!((p >> j) & 1)) {
          if (dig[j] != 0) valid = false;
          pauli = 0;
        } else {
          pauli = dig[j] == 0 ? 3 : dig[j];
        }
        b = 4 * b + (uint32_t)pauli;
      }
      if (!valid) continue;
      T r[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = snap ? snap_small(v[p][k]) : v[p][k];
      T* q = Q + (((int64_t)sv << (2 * KOUT)) + b) * (int64_t(1) << f) + x;
      if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(q) = make_float4(r[0], r[1], r[2], r[3]);
      } else {
        *reinterpret_cast<double2*>(q) = make_double2(r[0], r[1]);
        *reinterpret_cast<double2*>(q + 2) = make_double2(r[2], r[3]);
      }
    }
  }
}

// Eq. 2 in place: for every (b, x) the 4^KIN values over physical inits s
// (slot 0 most significant) become the 4^KIN Pauli operators a
template <typename T, int KIN>
__global__ void k_attr_inits(T* __restrict__ TQ, int64_t inner) {
  constexpr int NV = 1 << (2 * KIN);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < inner; i += (int64_t)gridDim.x * blockDim.x) {
    T v[NV];
#pragma unroll
    for (int s = 0; s < NV; ++s) v[s] = TQ[s * inner + i];
#pragma unroll
    for (int j = 0; j < KIN; ++j) {
      const int stride = 1 << (2 * (KIN - 1 - j));   // slot j's digit weight
#pragma unroll
      for (int g = 0; g < NV; ++g) {
        if ((g / stride) % 4 != 0) continue;        // g = the member with digit 0 of its group
        const T v0 = v[g], v1 = v[g + stride], v2 = v[g + 2 * stride], v3 = v[g + 3 * stride];
        const T s01 = v0 + v1;
        v[g] = s01;                                  // I = |0><0| + |1><1|
        v[g + stride] = (v2 + v2) - s01;             // X = 2|+><+| - I
        v[g + 2 * stride] = (v3 + v3) - s01;         // Y = 2|+i><+i| - I
        v[g + 3 * stride] = v0 - v1;                 // Z = |0><0| - |1><1|
      }
    }
#pragma unroll
    for (int s = 0; s < NV; ++s) {
      TQ[s * inner + i] = snap_small(v[s]);
    }
  }
}

// blocks of 256 threads for n threads of work, at most one wave of resident
// blocks of `fn` on the device
unsigned resident_grid(const void* fn, int64_t n) {
  static std::mutex mu;
  static std::map<const void*, int> cap;
  int c;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cap.find(fn);
    if (it == cap.end()) {
      int dev = 0, sms = 0, per = 0;
      CUTQC_CUDA(cudaGetDevice(&dev));
      CUTQC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      CUTQC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 256, 0));
      it = cap.emplace(fn, std::max(per, 1) * sms).first;
    }
    c = it->second;
  }
  const int64_t g = (n + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, c));
}

template <typename T>
void launch_two_pass(const T* P, const AttrArgs& a, T* out, cudaStream_t s) {
  const int64_t n_out = (int64_t(1) << (2 * (a.k_in + a.k_out))) << a.n_eff;
  const int64_t inner = (int64_t(1) << (2 * a.k_out)) << a.n_eff;
  auto grid = [](int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)(g > 152 * 16 ? 152 * 16 : g);
  };
  const int snap = a.k_in == 0 ? 1 : 0;
  const bool aligned = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  if (a.n_eff >= 2 && a.k_out <= 4 && aligned) {
    const int64_t n_grp = (((int64_t(1) << (2 * a.k_in)) * a.pow3_kout) << a.n_eff) / 4;
    // measured cut qubits on y bits 0 .. k_out-1 (any order), x bits 0-1 right above
    bool contig = sizeof(T) == 4 && a.k_out <= 2 && (reinterpret_cast<uintptr_t>(P) & 15) == 0 &&
                  a.out_pos[a.n_eff - 1] == a.k_out && a.out_pos[a.n_eff - 2] == a.k_out + 1;
    for (int j = 0; j < a.k_out; ++j) contig = contig && a.meas_pos[j] < a.k_out;
    if constexpr (sizeof(T) == 4) {
      if (contig) {
        // one wave of resident blocks (the loads are pipelined across a
        // thread's groups, and each block fills its tables once)
        auto go = [&](auto kern) {
          kern<<<resident_grid(reinterpret_cast<const void*>(kern), n_grp), 256, 0, s>>>(P, a, out, n_grp, snap);
        };
        switch (a.k_out) {
          case 0: go(k_attr_variants<T, 0, true>); break;
          case 1: go(k_attr_variants<T, 1, true>); break;
          default: go(k_attr_variants<T, 2, true>); break;
        }
      }
    }
    if (!contig) {
      switch (a.k_out) {
        case 0: k_attr_variants<T, 0, false><<<grid(n_grp), 256, 0, s>>>(P, a, out, n_grp, snap); break;
        case 1: k_attr_variants<T, 1, false><<<grid(n_grp), 256, 0, s>>>(P, a, out, n_grp, snap); break;
        case 2: k_attr_variants<T, 2, false><<<grid(n_grp), 256, 0, s>>>(P, a, out, n_grp, snap); break;
        case 3: k_attr_variants<T, 3, false><<<grid(n_grp), 256, 0, s>>>(P, a, out, n_grp, snap); break;
        default: k_attr_variants<T, 4, false><<<grid(n_grp), 256, 0, s>>>(P, a, out, n_grp, snap); break;
      }
    }
  } else if (a.n_eff >= 2) {
    // x bits 0 and 1 on y bits 0 and 1: four consecutive x are four consecutive y
    const bool low = a.out_pos[a.n_eff - 1] == 0 && a.out_pos[a.n_eff - 2] == 1;
    const bool vec = sizeof(T) == 4 && low && (reinterpret_cast<uintptr_t>(P) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    if constexpr (sizeof(T) == 4) {
      if (vec) {
        k_attr_outcomes<T, 4, true><<<grid(n_out / 4), 256, 0, s>>>(P, a, out, n_out, snap);
      } else {
        k_attr_outcomes<T, 4, false><<<grid(n_out / 4), 256, 0, s>>>(P, a, out, n_out, snap);
      }
    } else {
      (void)vec;
      k_attr_outcomes<T, 4, false><<<grid(n_out / 4), 256, 0, s>>>(P, a, out, n_out, snap);
    }
  } else {
    k_attr_outcomes<T, 1, false><<<grid(n_out), 256, 0, s>>>(P, a, out, n_out, snap);
  }
  count_launch();
  check_launch("k_attr_outcomes");
  switch (a.k_in) {
    case 0: return;
    case 1: k_attr_inits<T, 1><<<grid(inner), 256, 0, s>>>(out, inner); break;
    case 2: k_attr_inits<T, 2><<<grid(inner), 256, 0, s>>>(out, inner); break;
    default: k_attr_inits<T, 3><<<grid(inner), 256, 0, s>>>(out, inner); break;
  }
  count_launch();
  check_launch("k_attr_inits");
}

}  // namespace

void launch_attribute(const void* P, int dtype, int d, int k_in, const int* meas_q, int k_out, const int* out_q,
                      int n_eff, void* tensor, cudaStream_t s) {
  AttrArgs a{};
  a.d = d;
  a.k_in = k_in;
  a.k_out = k_out;
  a.n_eff = n_eff;
  for (int j = 0; j < k_out; ++j) a.meas_pos[j] = d - 1 - meas_q[j];
  for (int i = 0; i < n_eff; ++i) a.out_pos[i] = d - 1 - out_q[i];
  a.pow3_kout = 1;
  for (int j = 0; j < k_out; ++j) a.pow3_kout *= 3;
  if (k_in <= 3) {
    if (dtype == CUTQC_F64)
      launch_two_pass(static_cast<const double*>(P), a, static_cast<double*>(tensor), s);
    else
      launch_two_pass(static_cast<const float*>(P), a, static_cast<float*>(tensor), s);
    return;
  }
  const int64_t n_out = (int64_t(1) << (2 * (k_in + k_out))) << n_eff;
  int64_t g = (n_out + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (dtype == CUTQC_F64)
    k_attribute<double><<<(unsigned)g, 256, 0, s>>>(static_cast<const double*>(P), a, static_cast<double*>(tensor),
                                                    n_out);
  else
    k_attribute<float><<<(unsigned)g, 256, 0, s>>>(static_cast<const float*>(P), a, static_cast<float*>(tensor),
                                                   n_out);
  count_launch();
  check_launch("k_attribute");
}

}  // namespace cutqc

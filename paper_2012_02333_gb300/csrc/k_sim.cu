// GPU subcircuit simulator: input preparation for the reconstruction.
//
// For one subcircuit it simulates every physical variant (state stored in
// complex FP64, gates evaluated in double-float arithmetic, see below)
// (Fig. 3: each init slot prepared in |0>, |1>, |+>, |+i>; each measured cut
// qubit measured in the Z, X or Y basis), attributes the measured cut qubits'
// outcomes with the +-1 factors of Eq. 3 (basis I: both outcomes +1; X, Y, Z:
// outcome 0 -> +1, outcome 1 -> -1; I and Z share the Z-basis circuit), and
// combines the init variants into Pauli operators as in Eq. 2 (I = |0><0| +
// |1><1|, Z = |0><0| - |1><1|, X = 2|+><+| - I, Y = 2|+i><+i| - I).  The
// result is the tensor T[a][b][x] of the ABI.
//
// State layout: [variant][2^d] complex doubles, local qubit 0 = most
// significant bit of the index.  One kernel launch per run of consecutive
// gates over at most 10 index bits (k_gates_tile), over all variants of a
// chunk.  Attribution accumulates in FP64, entries below
// 2^-40 in magnitude are set to 0, then the tensor is cast to its dtype.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <vector>

#include "internal.h"

namespace cutqc {

namespace {

constexpr int kMaxSlots = 12;
constexpr int kMaxMeasSim = 8;   // measured cut qubits per subcircuit in the simulator
constexpr int kMaxRotSim = 4;    // ... whose basis changes the attribution applies itself
constexpr int kMaxOut = 40;

struct SimArgs {
  int d, k_in, k_out, n_eff;
  int init_bit[kMaxSlots];   // index bit position of each init slot's qubit
  int meas_bit[kMaxSlots];
  int out_bit[kMaxOut];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__global__ void k_sim_init(double2* __restrict__ psi, SimArgs a, int s0, int nb) {
  const int64_t dim = int64_t(1) << a.d;
  const int64_t tot = dim * nb;
  const double r = 0.70710678118654752440;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    // every extent here is a power of two: shifts and masks, no 64-bit division
    const int s = s0 + (int)(t >> a.d);
    const int64_t y = t & (dim - 1);
    int64_t init_mask = 0;
    double2 amp = make_double2(1.0, 0.0);
    for (int j = 0; j < a.k_in; ++j) {
      const int bit = a.init_bit[j];
      init_mask |= int64_t(1) << bit;
      const int digit = (s >> (2 * (a.k_in - 1 - j))) & 3;
      const int v = (y >> bit) & 1;
      double2 c;
      if (digit == 0) c = make_double2(v ? 0.0 : 1.0, 0.0);          // |0>
      else if (digit == 1) c = make_double2(v ? 1.0 : 0.0, 0.0);     // |1>
      else if (digit == 2) c = make_double2(r, 0.0);                 // |+>
      else c = v ? make_double2(0.0, r) : make_double2(r, 0.0);      // |+i>
      amp = cmul(amp, c);
    }
    if (y & ~init_mask) amp = make_double2(0.0, 0.0);   // other qubits start in |0>
    psi[t] = amp;
  }
}

__global__ void k_gate1(double2* __restrict__ psi, int d, int nb, int bit, double2 u00, double2 u01, double2 u10,
                        double2 u11) {
  const int64_t half = int64_t(1) << (d - 1);
  const int64_t tot = half * nb;
  const int64_t lo = (int64_t(1) << bit) - 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t >> (d - 1), i = t & (half - 1);
    const int64_t i0 = ((i & ~lo) << 1) | (i & lo);
    const int64_t i1 = i0 | (int64_t(1) << bit);
    double2* p = psi + (v << d);
    const double2 a0 = p[i0], a1 = p[i1];
    p[i0] = cadd(cmul(u00, a0), cmul(u01, a1));
    p[i1] = cadd(cmul(u10, a0), cmul(u11, a1));
  }
}

// Gate fusion: a run of consecutive gates that together touch at most
// kTileBits of the state's index bits is applied in one pass.  The tile bits
// are those bits plus the lowest other ones (so a tile's first 8 amplitudes
// are contiguous in memory); a block owns one tile (one variant, one value
// of the other bits), loads its 2^L amplitudes into shared memory, applies
// every gate of the run there (one barrier between gates) and writes them
// back.
//
// Inside a pass the amplitudes are double-float numbers (an unevaluated sum
// hi + lo of two FP32 values, about 48 significant bits) and the gates are
// evaluated with error-free transformations on the FP32 pipes: Knuth's
// TwoSum for additions, the FMA form of Dekker's product for
// multiplications (the pair renormalised with Dekker's fast two-sum after
// each operation).  FP64 runs at 1/64 of the FP32 rate on this part, and
// the gates were FP64-bound (53 % of the FP64 peak in the fused kernel).
// Between passes the state is stored in FP64.  Each operation's relative
// error is about 2^-48 (against 2^-53 in FP64), so amplitudes of a
// 100-gate circuit carry relative errors of order 1e-13 and the attributed
// tensor entries (sums of probabilities of magnitude at most 2) absolute
// errors of order 1e-13: entries that vanish exactly stay far below the
// 2^-40 (9.1e-13) zero threshold only if the accumulation stays below it,
// which the simulator tests check against the FP64 oracle at 1e-12.
constexpr int kTileBits = 10;

struct FusedGate {
  int nq;        // 1 or 2
  int diag;      // the matrix is diagonal (entries 0, 3 or 0, 5, 10, 15 of the table)
  int p0, p1;    // positions among the tile bits (p0: the matrix's more significant qubit)
  int mat;       // first entry of its matrix in the matrix table (4 or 16 entries)
};

struct TileBits {
  int L;
  int tb[kTileBits];   // index bit of tile position k, ascending
  int64_t tmask;       // the tile bits as a mask
};

struct DF {
  float hi, lo;
};
// (the _rn intrinsics are never contracted into an FMA, which would break
// the error-free transformations)
// Dekker's fast two-sum (|a| >= |b| or a == 0)
__device__ __forceinline__ DF df_fast(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// Knuth's TwoSum
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  const DF t = df_two_sum(a.lo, b.lo);
  s = df_fast(s.hi, __fadd_rn(s.lo, t.hi));
  return df_fast(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);   // exact rounding error of the product
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast(p, e);
}
__device__ __forceinline__ DF df_of(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double df_val(DF a) { return (double)a.hi + (double)a.lo; }

struct CDF {
  DF re, im;
};
__device__ __forceinline__ CDF cdf_of(double2 z) { return {df_of(z.x), df_of(z.y)}; }
__device__ __forceinline__ double2 cdf_val(CDF z) { return make_double2(df_val(z.re), df_val(z.im)); }
__device__ __forceinline__ CDF cdf_mul(CDF u, CDF a) {
  return {df_add(df_mul(u.re, a.re), df_neg(df_mul(u.im, a.im))), df_add(df_mul(u.re, a.im), df_mul(u.im, a.re))};
}
__device__ __forceinline__ CDF cdf_add(CDF a, CDF b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ float4 cdf_pack(CDF z) { return make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo); }
__device__ __forceinline__ CDF cdf_unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }

__global__ __launch_bounds__(256, 3) void k_gates_tile(double2* __restrict__ psi, int d, TileBits t,
                                                    const FusedGate* __restrict__ gates, int ng,
                                                    const float4* __restrict__ mats) {
  __shared__ float4 tile[1 << kTileBits];
  const int L = t.L, n = 1 << L, tid = threadIdx.x;
  const int64_t v = (int64_t)blockIdx.x >> (d - L);
  const int64_t r = (int64_t)blockIdx.x & ((int64_t(1) << (d - L)) - 1);
  // the other bits of this tile's amplitudes: r deposited into the non-tile bits
  int64_t base = 0;
  for (int b = 0, rb = 0; b < d; ++b)
    if (!((t.tmask >> b) & 1)) base |= ((r >> rb++) & 1) << b;
  double2* p = psi + (v << d);
  auto at = [&](int j) {
    int64_t y = base;
#pragma unroll
    for (int k = 0; k < kTileBits; ++k)
      if (k < L) y |= (int64_t)((j >> k) & 1) << t.tb[k];
    return y;
  };
  for (int j = tid; j < n; j += 256) tile[j] = cdf_pack(cdf_of(p[at(j)]));
  __syncthreads();
  for (int gi = 0; gi < ng; ++gi) {
    const FusedGate G = gates[gi];
    if (G.nq == 1) {
      const int lo = (1 << G.p0) - 1;
      if (G.diag) {
        const CDF u00 = cdf_unpack(mats[G.mat]), u11 = cdf_unpack(mats[G.mat + 3]);
        for (int q = tid; q < (n >> 1); q += 256) {
          const int i0 = ((q & ~lo) << 1) | (q & lo), i1 = i0 | (1 << G.p0);
          tile[i0] = cdf_pack(cdf_mul(u00, cdf_unpack(tile[i0])));
          tile[i1] = cdf_pack(cdf_mul(u11, cdf_unpack(tile[i1])));
        }
      } else {
        const CDF u00 = cdf_unpack(mats[G.mat]), u01 = cdf_unpack(mats[G.mat + 1]);
        const CDF u10 = cdf_unpack(mats[G.mat + 2]), u11 = cdf_unpack(mats[G.mat + 3]);
        for (int q = tid; q < (n >> 1); q += 256) {
          const int i0 = ((q & ~lo) << 1) | (q & lo), i1 = i0 | (1 << G.p0);
          const CDF a0 = cdf_unpack(tile[i0]), a1 = cdf_unpack(tile[i1]);
          tile[i0] = cdf_pack(cdf_add(cdf_mul(u00, a0), cdf_mul(u01, a1)));
          tile[i1] = cdf_pack(cdf_add(cdf_mul(u10, a0), cdf_mul(u11, a1)));
        }
      }
    } else {
      const int lo_b = G.p0 < G.p1 ? G.p0 : G.p1, hi_b = G.p0 < G.p1 ? G.p1 : G.p0;
      for (int q = tid; q < (n >> 2); q += 256) {
        int i = q;
        int m = (1 << lo_b) - 1;
        i = ((i & ~m) << 1) | (i & m);
        m = (1 << hi_b) - 1;
        i = ((i & ~m) << 1) | (i & m);
        int idx[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) idx[k] = i | (((k >> 1) & 1) << G.p0) | ((k & 1) << G.p1);
        if (G.diag) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tile[idx[k]] = cdf_pack(cdf_mul(cdf_unpack(mats[G.mat + 5 * k]), cdf_unpack(tile[idx[k]])));
        } else {
          CDF a[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) a[k] = cdf_unpack(tile[idx[k]]);
#pragma unroll 1
          for (int rr = 0; rr < 4; ++rr) {
            CDF acc = cdf_mul(cdf_unpack(mats[G.mat + 4 * rr]), a[0]);
#pragma unroll
            for (int k = 1; k < 4; ++k) acc = cdf_add(acc, cdf_mul(cdf_unpack(mats[G.mat + 4 * rr + k]), a[k]));
            tile[idx[rr]] = cdf_pack(acc);
          }
        }
      }
    }
    __syncthreads();
  }
  for (int j = tid; j < n; j += 256) p[at(j)] = cdf_val(cdf_unpack(tile[j]));
}

// Generic form (any number of measured qubits up to 8): phi is a copy of
// the state already rotated into the measurement bases of combination mb.
__global__ void k_attr_meas(const double2* __restrict__ phi, SimArgs a, int s0, int nb, int mb,
                            double* __restrict__ P) {
  const int64_t nx = int64_t(1) << a.n_eff;
  const int64_t tot = nx * nb;
  const int nm = 1 << a.k_out;
  const int64_t rows_b = int64_t(1) << (2 * a.k_out);
  int basis[kMaxMeasSim];
  int zmask = 0;
  for (int j = 0; j < a.k_out; ++j) {
    int t = mb;
    for (int r = 0; r < a.k_out - 1 - j; ++r) t /= 3;
    basis[j] = t % 3;
    if (basis[j] == 0) zmask |= 1 << j;
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int sl = (int)(t >> a.n_eff);
    const int64_t x = t & (nx - 1);
    int64_t ybase = 0;
    for (int i = 0; i < a.n_eff; ++i)
      if ((x >> (a.n_eff - 1 - i)) & 1) ybase |= int64_t(1) << a.out_bit[i];
    const double2* p = phi + ((int64_t)sl << a.d);
    double pr[1 << kMaxMeasSim];
    for (int m = 0; m < nm; ++m) {
      int64_t y = ybase;
      for (int j = 0; j < a.k_out; ++j)
        if ((m >> (a.k_out - 1 - j)) & 1) y |= int64_t(1) << a.meas_bit[j];
      const double2 v = p[y];
      pr[m] = v.x * v.x + v.y * v.y;
    }
    // enumerate the b rows served: for Z-basis slots choose I or Z
    for (int sub = 0; sub < nm; ++sub) {
      if (sub & ~zmask) continue;   // only subsets of the Z-basis slots
      int64_t b = 0;
      int sign_mask = 0;            // slots whose outcome flips the sign (bit j = slot j)
      for (int j = 0; j < a.k_out; ++j) {
        int digit;
        if (basis[j] == 0) digit = ((sub >> j) & 1) ? 3 : 0;
        else digit = basis[j];      // X = 1, Y = 2
        b = 4 * b + digit;
        if (digit != 0) sign_mask |= 1 << (a.k_out - 1 - j);
      }
      double val = 0.0;
      for (int m = 0; m < nm; ++m) val += (__popc(m & sign_mask) & 1) ? -pr[m] : pr[m];
      P[((int64_t)(s0 + sl) * rows_b + b) * nx + x] = val;
    }
  }
}

// KO <= 4 measured qubits: the state is the one before measurement and the
// kernel applies the basis changes itself (H for X, S^dagger then H for Y)
// to the 2^KO amplitudes of each output it holds, with the arithmetic of the
// gate kernels, for every basis combination mb = blockIdx.y in one launch
// (no rotated copy of the state per combination); the sizes are compile-time
// so the amplitudes and probabilities stay in registers.  Same results as
// the generic form on a rotated copy.
template <int KO>
__global__ void k_attr_meas_rot(const double2* __restrict__ psi, SimArgs a, int s0, int nb,
                                double* __restrict__ P) {
  constexpr int NM = 1 << KO;
  const int mb = (int)blockIdx.y;
  const int64_t nx = int64_t(1) << a.n_eff;
  const int64_t tot = nx * nb;
  constexpr int64_t rows_b = int64_t(1) << (2 * KO);
  int basis[KO > 0 ? KO : 1];
  int zmask = 0;
#pragma unroll
  for (int j = 0; j < KO; ++j) {
    int t = mb;
    for (int r = 0; r < KO - 1 - j; ++r) t /= 3;
    basis[j] = t % 3;
    if (basis[j] == 0) zmask |= 1 << j;
  }
  const double r = 0.70710678118654752440;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int sl = (int)(t >> a.n_eff);
    const int64_t x = t & (nx - 1);
    int64_t ybase = 0;
    for (int i = 0; i < a.n_eff; ++i)
      if ((x >> (a.n_eff - 1 - i)) & 1) ybase |= int64_t(1) << a.out_bit[i];
    const double2* p = psi + ((int64_t)sl << a.d);
    double2 amp[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      int64_t y = ybase;
#pragma unroll
      for (int j = 0; j < KO; ++j)
        if ((m >> (KO - 1 - j)) & 1) y |= int64_t(1) << a.meas_bit[j];
      amp[m] = p[y];
    }
#pragma unroll
    for (int j = 0; j < KO; ++j) {
      if (basis[j] == 0) continue;
      // X: (1/sqrt2) [[1, 1], [1, -1]]; Y: (1/sqrt2) [[1, -i], [1, i]]
      const double2 u00 = make_double2(r, 0.0), u10 = make_double2(r, 0.0);
      const double2 u01 = basis[j] == 1 ? make_double2(r, 0.0) : make_double2(0.0, -r);
      const double2 u11 = basis[j] == 1 ? make_double2(-r, 0.0) : make_double2(0.0, r);
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const int bit = 1 << (KO - 1 - j);
        if (m & bit) continue;
        const double2 a0 = amp[m], a1 = amp[m | bit];
        amp[m] = cadd(cmul(u00, a0), cmul(u01, a1));
        amp[m | bit] = cadd(cmul(u10, a0), cmul(u11, a1));
      }
    }
    double pr[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) pr[m] = amp[m].x * amp[m].x + amp[m].y * amp[m].y;
#pragma unroll
    for (int sub = 0; sub < NM; ++sub) {
      if (sub & ~zmask) continue;
      int64_t b = 0;
      int sign_mask = 0;
#pragma unroll
      for (int j = 0; j < KO; ++j) {
        int digit;
        if (basis[j] == 0) digit = ((sub >> j) & 1) ? 3 : 0;
        else digit = basis[j];
        b = 4 * b + digit;
        if (digit != 0) sign_mask |= 1 << (KO - 1 - j);
      }
      double val = 0.0;
#pragma unroll
      for (int m = 0; m < NM; ++m) val += (__popc(m & sign_mask) & 1) ? -pr[m] : pr[m];
      P[((int64_t)(s0 + sl) * rows_b + b) * nx + x] = val;
    }
  }
}

// Eq. 2 along init slot j: for every fixed rest of the index, the 4 physical
// variants (|0>, |1>, |+>, |+i>) become the 4 Pauli operators (I, X, Y, Z).
__global__ void k_attr_init(double* __restrict__ P, int k_in, int j, int64_t inner) {
  // inner = 4^k_out * 2^n_eff; index = ((hi * 4 + digit) * stride + lo)
  const int64_t stride = (int64_t(1) << (2 * (k_in - 1 - j))) * inner;   // a power of two
  const int ls = __ffsll((long long)stride) - 1;
  const int64_t hi_n = int64_t(1) << (2 * j);
  const int64_t tot = hi_n * stride;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t hi = t >> ls, lo = t & (stride - 1);
    double* base = P + hi * 4 * stride + lo;
    const double p0 = base[0], p1 = base[stride], pp = base[2 * stride], pi = base[3 * stride];
    base[0] = p0 + p1;                     // I
    base[stride] = 2.0 * pp - p0 - p1;     // X
    base[2 * stride] = 2.0 * pi - p0 - p1; // Y
    base[3 * stride] = p0 - p1;            // Z
  }
}

template <typename T>
__global__ void k_sim_finish(const double* __restrict__ P, T* __restrict__ out, int64_t n) {
  const double eps = 9.094947017729282e-13;   // 2^-40
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double v = P[t];
    out[t] = (T)(fabs(v) < eps ? 0.0 : v);
  }
}

unsigned grid_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  return (unsigned)g;
}

struct C2 {
  double re, im;
};

void gate_matrix(const cutqc_gate& g, double2* m, int& nq) {
  const double r = 0.70710678118654752440;
  auto set2 = [&](C2 a, C2 b, C2 c, C2 d) {
    m[0] = make_double2(a.re, a.im);
    m[1] = make_double2(b.re, b.im);
    m[2] = make_double2(c.re, c.im);
    m[3] = make_double2(d.re, d.im);
    nq = 1;
  };
  const double t = g.param / 2;
  switch (g.op) {
    case CUTQC_GATE_H: set2({r, 0}, {r, 0}, {r, 0}, {-r, 0}); break;
    case CUTQC_GATE_X: set2({0, 0}, {1, 0}, {1, 0}, {0, 0}); break;
    case CUTQC_GATE_Y: set2({0, 0}, {0, -1}, {0, 1}, {0, 0}); break;
    case CUTQC_GATE_Z: set2({1, 0}, {0, 0}, {0, 0}, {-1, 0}); break;
    case CUTQC_GATE_S: set2({1, 0}, {0, 0}, {0, 0}, {0, 1}); break;
    case CUTQC_GATE_SDG: set2({1, 0}, {0, 0}, {0, 0}, {0, -1}); break;
    case CUTQC_GATE_T: set2({1, 0}, {0, 0}, {0, 0}, {r, r}); break;
    // sqrt of a Hermitian involution P: ((1+i) I + (1-i) P) / 2
    case CUTQC_GATE_SX: set2({0.5, 0.5}, {0.5, -0.5}, {0.5, -0.5}, {0.5, 0.5}); break;
    case CUTQC_GATE_SY: set2({0.5, 0.5}, {-0.5, -0.5}, {0.5, 0.5}, {0.5, 0.5}); break;
    case CUTQC_GATE_SW: {
      // W = (X + Y)/sqrt2 = [[0, (1-i)/sqrt2], [(1+i)/sqrt2, 0]]; (1-i)(1-i) = -2i, (1-i)(1+i) = 2
      set2({0.5, 0.5}, {0.0, -r}, {r, 0.0}, {0.5, 0.5});
      break;
    }
    case CUTQC_GATE_RX: set2({cos(t), 0}, {0, -sin(t)}, {0, -sin(t)}, {cos(t), 0}); break;
    case CUTQC_GATE_RY: set2({cos(t), 0}, {-sin(t), 0}, {sin(t), 0}, {cos(t), 0}); break;
    case CUTQC_GATE_RZ: set2({cos(t), -sin(t)}, {0, 0}, {0, 0}, {cos(t), sin(t)}); break;
    default: {
      nq = 2;
      for (int k = 0; k < 16; ++k) m[k] = make_double2(0, 0);
      for (int k = 0; k < 4; ++k) m[5 * k] = make_double2(1, 0);
      if (g.op == CUTQC_GATE_CZ) m[15] = make_double2(-1, 0);
      else if (g.op == CUTQC_GATE_CP) m[15] = make_double2(cos(g.param), sin(g.param));
      else {  // CX, control = q0 (more significant matrix index bit)
        m[10] = make_double2(0, 0);
        m[15] = make_double2(0, 0);
        m[11] = make_double2(1, 0);
        m[14] = make_double2(1, 0);
      }
    }
  }
}

// the per-device scratch block of the simulator (grow-only, at most 256 MiB)
struct SimScratch {
  void* p = nullptr;
  size_t bytes = 0;
};
std::map<int, SimScratch> g_sim_scratch;

char* sim_scratch(size_t bytes) {
  int dev = 0;
  CUTQC_CUDA(cudaGetDevice(&dev));
  SimScratch& sc = g_sim_scratch[dev];
  if (bytes > sc.bytes) {
    if (sc.p) CUTQC_CUDA(cudaFree(sc.p));
    sc.p = nullptr;
    sc.bytes = 0;
    CUTQC_CUDA(cudaMalloc(&sc.p, bytes));
    sc.bytes = bytes;
  }
  return static_cast<char*>(sc.p);
}

}  // namespace

void run_subcircuit_sim(const SimPlan& sp, int dtype, void* tensor, cudaStream_t s) {
  if (sp.k_out > kMaxMeasSim) fail(CUTQC_ERR_UNSUPPORTED, "simulator supports at most 8 measured cut qubits");
  if (sp.n_eff > 30) fail(CUTQC_ERR_UNSUPPORTED, "simulator supports at most 30 outputs");
  SimArgs a{};
  a.d = sp.d;
  a.k_in = sp.k_in;
  a.k_out = sp.k_out;
  a.n_eff = sp.n_eff;
  for (int j = 0; j < sp.k_in; ++j) a.init_bit[j] = sp.d - 1 - sp.init_q[j];
  for (int j = 0; j < sp.k_out; ++j) a.meas_bit[j] = sp.d - 1 - sp.meas_q[j];
  for (int j = 0; j < sp.n_eff; ++j) a.out_bit[j] = sp.d - 1 - sp.out_q[j];
  const int64_t dim = int64_t(1) << sp.d;
  const int nvar = 1 << (2 * sp.k_in);
  const int nmb = (int)std::lround(std::pow(3.0, sp.k_out));
  const int64_t inner = (int64_t(1) << (2 * sp.k_out)) * (int64_t(1) << sp.n_eff);
  const int64_t total = (int64_t)nvar * inner;
  // state chunk: psi and phi for nb variants within ~8 GiB
  const int64_t budget = int64_t(8) << 30;
  int nb = (int)std::max<int64_t>(1, std::min<int64_t>(nvar, budget / (dim * 32)));
  std::vector<std::pair<std::vector<double2>, int>> mats;
  for (const cutqc_gate& g : sp.gates) {
    std::vector<double2> m(16);
    int nq = 1;
    gate_matrix(g, m.data(), nq);
    mats.emplace_back(m, nq);
  }
  // runs of consecutive gates over at most L index bits, each run's tile
  // bits, its gates by tile position and the matrix table
  const int L = std::min(sp.d, kTileBits);
  std::vector<TileBits> runs;
  std::vector<std::pair<int, int>> run_gates;   // [first, count) into fg
  std::vector<FusedGate> fg;
  std::vector<float4> mt;   // matrix entries as double-float (re.hi, re.lo, im.hi, im.lo)
  {
    size_t gi = 0;
    while (gi < sp.gates.size()) {
      int64_t used = 0;
      size_t gj = gi;
      for (; gj < sp.gates.size(); ++gj) {
        int64_t m = int64_t(1) << (sp.d - 1 - sp.gates[gj].q0);
        if (mats[gj].second == 2) m |= int64_t(1) << (sp.d - 1 - sp.gates[gj].q1);
        if (__builtin_popcountll(used | m) > L) break;
        used |= m;
      }
      for (int b = 0; b < sp.d && __builtin_popcountll(used) < L; ++b) used |= int64_t(1) << b;
      TileBits t{};
      t.L = L;
      t.tmask = used;
      int pos[64];
      for (int b = 0, k = 0; b < sp.d; ++b)
        if ((used >> b) & 1) {
          pos[b] = k;
          t.tb[k++] = b;
        }
      runs.push_back(t);
      run_gates.emplace_back((int)fg.size(), (int)(gj - gi));
      for (size_t g = gi; g < gj; ++g) {
        FusedGate f{};
        f.nq = mats[g].second;
        f.diag = 1;
        for (int rr = 0; rr < 2 * f.nq; ++rr)
          for (int k = 0; k < 2 * f.nq; ++k) {
            const double2 e = mats[g].first[(size_t)(2 * f.nq) * rr + k];
            if (rr != k && (e.x != 0.0 || e.y != 0.0)) f.diag = 0;
          }
        f.p0 = pos[sp.d - 1 - sp.gates[g].q0];
        f.p1 = f.nq == 2 ? pos[sp.d - 1 - sp.gates[g].q1] : 0;
        f.mat = (int)mt.size();
        for (int e = 0; e < (f.nq == 2 ? 16 : 4); ++e) {
          const double2 z = mats[g].first[e];
          const float rh = (float)z.x, ih = (float)z.y;
          mt.push_back(make_float4(rh, (float)(z.x - (double)rh), ih, (float)(z.y - (double)ih)));
        }
        fg.push_back(f);
      }
      gi = gj;
    }
  }
  // one scratch block: state, rotated copy (more than 4 measured qubits),
  // attributed rows, gate and matrix tables.  Up to 256 MiB it is kept per
  // device between calls (calls are serialised and end with a stream
  // synchronisation, so the next call may reuse it); larger blocks are
  // allocated and freed per call.
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_phi = up((size_t)dim * nb * sizeof(double2));
  const size_t o_P = o_phi + (sp.k_out > kMaxRotSim ? up((size_t)dim * nb * sizeof(double2)) : 0);
  const size_t o_g = o_P + up((size_t)total * sizeof(double));
  const size_t o_m = o_g + up(fg.size() * sizeof(FusedGate));
  const size_t bytes = o_m + up(mt.size() * sizeof(float4));
  char* block = nullptr;
  const bool cached = bytes <= (size_t(256) << 20);
  if (cached) {
    block = sim_scratch(bytes);
  } else {
    CUTQC_CUDA(cudaStreamSynchronize(s));
    CUTQC_CUDA(cudaMalloc(&block, bytes));
  }
  double2* psi = reinterpret_cast<double2*>(block);
  double2* phi = reinterpret_cast<double2*>(block + o_phi);
  double* P = reinterpret_cast<double*>(block + o_P);
  FusedGate* dg = reinterpret_cast<FusedGate*>(block + o_g);
  float4* dm = reinterpret_cast<float4*>(block + o_m);
  try {
    if (!fg.empty()) {
      CUTQC_CUDA(cudaMemcpyAsync(dg, fg.data(), fg.size() * sizeof(FusedGate), cudaMemcpyHostToDevice, s));
      CUTQC_CUDA(cudaMemcpyAsync(dm, mt.data(), mt.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
    }
    const double2 hr = make_double2(0.70710678118654752440, 0.0);
    for (int s0 = 0; s0 < nvar; s0 += nb) {
      const int n = std::min(nb, nvar - s0);
      k_sim_init<<<grid_for(dim * n), 256, 0, s>>>(psi, a, s0, n);
      count_launch();
      check_launch("k_sim_init");
      for (size_t r = 0; r < runs.size(); ++r) {
        const unsigned blocks = (unsigned)(((int64_t)n) << (sp.d - L));
        k_gates_tile<<<blocks, 256, 0, s>>>(psi, sp.d, runs[r], dg + run_gates[r].first, run_gates[r].second, dm);
        count_launch();
        check_launch("k_gates_tile");
      }
      if (sp.k_out <= kMaxRotSim) {
        // the basis changes inside the attribution (no copy of the state),
        // every basis combination in one launch
        const dim3 grid(std::max(1u, grid_for((int64_t(1) << sp.n_eff) * n) / (unsigned)nmb), (unsigned)nmb);
        switch (sp.k_out) {
          case 0: k_attr_meas_rot<0><<<grid, 256, 0, s>>>(psi, a, s0, n, P); break;
          case 1: k_attr_meas_rot<1><<<grid, 256, 0, s>>>(psi, a, s0, n, P); break;
          case 2: k_attr_meas_rot<2><<<grid, 256, 0, s>>>(psi, a, s0, n, P); break;
          case 3: k_attr_meas_rot<3><<<grid, 256, 0, s>>>(psi, a, s0, n, P); break;
          default: k_attr_meas_rot<4><<<grid, 256, 0, s>>>(psi, a, s0, n, P); break;
        }
        count_launch();
        check_launch("k_attr_meas");
      }
      for (int mb = 0; mb < nmb && sp.k_out > kMaxRotSim; ++mb) {
        CUTQC_CUDA(cudaMemcpyAsync(phi, psi, (size_t)dim * n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        int t = mb;
        std::vector<int> bases(sp.k_out);
        for (int j = sp.k_out - 1; j >= 0; --j) {
          bases[j] = t % 3;
          t /= 3;
        }
        for (int j = 0; j < sp.k_out; ++j) {
          const int bit = sp.d - 1 - sp.meas_q[j];
          if (bases[j] == 1) {   // X: H
            k_gate1<<<grid_for(dim / 2 * n), 256, 0, s>>>(phi, sp.d, n, bit, hr, hr, hr, make_double2(-hr.x, 0));
            count_launch();
          } else if (bases[j] == 2) {   // Y: S^dagger then H, i.e. (1/sqrt2) [[1, -i], [1, i]]
            k_gate1<<<grid_for(dim / 2 * n), 256, 0, s>>>(phi, sp.d, n, bit, hr, make_double2(0, -hr.x), hr,
                                                          make_double2(0, hr.x));
            count_launch();
          }
        }
        k_attr_meas<<<grid_for((int64_t(1) << sp.n_eff) * n), 256, 0, s>>>(phi, a, s0, n, mb, P);
        count_launch();
        check_launch("k_attr_meas");
      }
    }
    for (int j = 0; j < sp.k_in; ++j) {
      const int64_t work = total / 4;
      k_attr_init<<<grid_for(work), 256, 0, s>>>(P, sp.k_in, j, inner);
      count_launch();
      check_launch("k_attr_init");
    }
    if (dtype == CUTQC_F64)
      k_sim_finish<double><<<grid_for(total), 256, 0, s>>>(P, static_cast<double*>(tensor), total);
    else
      k_sim_finish<float><<<grid_for(total), 256, 0, s>>>(P, static_cast<float*>(tensor), total);
    count_launch();
    check_launch("k_sim_finish");
    CUTQC_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    if (!cached) cudaFree(block);
    throw;
  }
  if (!cached) CUTQC_CUDA(cudaFree(block));
}

void release_sim_scratch() {
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_sim_scratch) {
    cudaSetDevice(kv.first);
    if (kv.second.p) cudaFree(kv.second.p);
  }
  g_sim_scratch.clear();
  cudaSetDevice(cur);
}

}  // namespace cutqc

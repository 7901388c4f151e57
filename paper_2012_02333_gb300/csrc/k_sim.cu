// GPU subcircuit simulator: input preparation for the reconstruction.
//
// For one subcircuit it simulates, in complex FP64, every physical variant
// (Fig. 3: each init slot prepared in |0>, |1>, |+>, |+i>; each measured cut
// qubit measured in the Z, X or Y basis), attributes the measured cut qubits'
// outcomes with the +-1 factors of Eq. 3 (basis I: both outcomes +1; X, Y, Z:
// outcome 0 -> +1, outcome 1 -> -1; I and Z share the Z-basis circuit), and
// combines the init variants into Pauli operators as in Eq. 2 (I = |0><0| +
// |1><1|, Z = |0><0| - |1><1|, X = 2|+><+| - I, Y = 2|+i><+i| - I).  The
// result is the tensor T[a][b][x] of the ABI.
//
// State layout: [variant][2^d] complex doubles, local qubit 0 = most
// significant bit of the index.  One kernel launch per gate over all
// variants of a chunk.  Attribution accumulates in FP64, entries below
// 2^-40 in magnitude are set to 0, then the tensor is cast to its dtype.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "internal.h"

namespace cutqc {

namespace {

constexpr int kMaxSlots = 12;
constexpr int kMaxMeasSim = 8;   // measured cut qubits per subcircuit in the simulator
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

struct Mat4 {
  double2 m[16];
};

// 4x4 gate on (q0, q1); matrix index = 2 * bit(q0) + bit(q1)
__global__ void k_gate2(double2* __restrict__ psi, int d, int nb, int b0, int b1, Mat4 U) {
  const int64_t quarter = int64_t(1) << (d - 2);
  const int64_t tot = quarter * nb;
  const int lo_b = b0 < b1 ? b0 : b1, hi_b = b0 < b1 ? b1 : b0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t >> (d - 2);
    int64_t i = t & (quarter - 1);
    // insert zero bits at lo_b then hi_b
    int64_t m = (int64_t(1) << lo_b) - 1;
    i = ((i & ~m) << 1) | (i & m);
    m = (int64_t(1) << hi_b) - 1;
    i = ((i & ~m) << 1) | (i & m);
    double2* p = psi + (v << d);
    int64_t idx[4];
    for (int k = 0; k < 4; ++k)
      idx[k] = i | ((int64_t)((k >> 1) & 1) << b0) | ((int64_t)(k & 1) << b1);
    double2 a[4];
    for (int k = 0; k < 4; ++k) a[k] = p[idx[k]];
    for (int r = 0; r < 4; ++r) {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < 4; ++k) acc = cadd(acc, cmul(U.m[4 * r + k], a[k]));
      p[idx[r]] = acc;
    }
  }
}

// Eq. 3 for one combination of measurement bases `mb` (base-3 digits Z=0,
// X=1, Y=2 per measurement slot, slot 0 most significant): for every variant
// s and output x, and every Pauli row b that this basis combination serves
// (slots measured in Z serve b = I and b = Z, X serves X, Y serves Y),
// P[s][b][x] = sum_m (prod_j sign(b_j, m_j)) p_s(x, m).
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
  double2 *psi = nullptr, *phi = nullptr;
  double* P = nullptr;
  CUTQC_CUDA(cudaStreamSynchronize(s));
  CUTQC_CUDA(cudaMalloc(&psi, (size_t)dim * nb * sizeof(double2)));
  CUTQC_CUDA(cudaMalloc(&phi, (size_t)dim * nb * sizeof(double2)));
  CUTQC_CUDA(cudaMalloc(&P, (size_t)total * sizeof(double)));
  try {
    std::vector<std::pair<std::vector<double2>, int>> mats;
    for (const cutqc_gate& g : sp.gates) {
      std::vector<double2> m(16);
      int nq = 1;
      gate_matrix(g, m.data(), nq);
      mats.emplace_back(m, nq);
    }
    const double2 hr = make_double2(0.70710678118654752440, 0.0);
    for (int s0 = 0; s0 < nvar; s0 += nb) {
      const int n = std::min(nb, nvar - s0);
      k_sim_init<<<grid_for(dim * n), 256, 0, s>>>(psi, a, s0, n);
      count_launch();
      check_launch("k_sim_init");
      for (size_t gi = 0; gi < sp.gates.size(); ++gi) {
        const cutqc_gate& g = sp.gates[gi];
        const double2* m = mats[gi].first.data();
        if (mats[gi].second == 1) {
          k_gate1<<<grid_for(dim / 2 * n), 256, 0, s>>>(psi, sp.d, n, sp.d - 1 - g.q0, m[0], m[1], m[2], m[3]);
        } else {
          Mat4 U;
          for (int k = 0; k < 16; ++k) U.m[k] = m[k];
          k_gate2<<<grid_for(dim / 4 * n), 256, 0, s>>>(psi, sp.d, n, sp.d - 1 - g.q0, sp.d - 1 - g.q1, U);
        }
        count_launch();
        check_launch("k_gate");
      }
      for (int mb = 0; mb < nmb; ++mb) {
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
    cudaFree(psi);
    cudaFree(phi);
    cudaFree(P);
    throw;
  }
  CUTQC_CUDA(cudaFree(psi));
  CUTQC_CUDA(cudaFree(phi));
  CUTQC_CUDA(cudaFree(P));
}

}  // namespace cutqc

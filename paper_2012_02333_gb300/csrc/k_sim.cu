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
// significant bit of the index.  One kernel launch per run of consecutive
// gates over at most 10 index bits (k_gates_tile), over all variants of a
// chunk.  Attribution accumulates in FP64, entries below
// 2^-40 in magnitude are set to 0, then the tensor is cast to its dtype.
#include <cuda_runtime.h>

#include <cmath>
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
// back.  The arithmetic is the per-gate kernels' (complex FP64), in the same
// order per amplitude, so the states are the same as gate by gate.
constexpr int kTileBits = 10;

struct FusedGate {
  int nq;        // 1 or 2
  int p0, p1;    // positions among the tile bits (p0: the matrix's more significant qubit)
  int mat;       // first entry of its matrix in the matrix table (4 or 16 entries)
};

struct TileBits {
  int L;
  int tb[kTileBits];   // index bit of tile position k, ascending
  int64_t tmask;       // the tile bits as a mask
};

__global__ __launch_bounds__(256) void k_gates_tile(double2* __restrict__ psi, int d, TileBits t,
                                                    const FusedGate* __restrict__ gates, int ng,
                                                    const double2* __restrict__ mats) {
  __shared__ double2 tile[1 << kTileBits];
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
  for (int j = tid; j < n; j += 256) tile[j] = p[at(j)];
  __syncthreads();
  for (int gi = 0; gi < ng; ++gi) {
    const FusedGate G = gates[gi];
    if (G.nq == 1) {
      const double2 u00 = mats[G.mat], u01 = mats[G.mat + 1], u10 = mats[G.mat + 2], u11 = mats[G.mat + 3];
      const int lo = (1 << G.p0) - 1;
      for (int q = tid; q < (n >> 1); q += 256) {
        const int i0 = ((q & ~lo) << 1) | (q & lo), i1 = i0 | (1 << G.p0);
        const double2 a0 = tile[i0], a1 = tile[i1];
        tile[i0] = cadd(cmul(u00, a0), cmul(u01, a1));
        tile[i1] = cadd(cmul(u10, a0), cmul(u11, a1));
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
        for (int k = 0; k < 4; ++k) idx[k] = i | (((k >> 1) & 1) << G.p0) | ((k & 1) << G.p1);
        double2 a[4];
        for (int k = 0; k < 4; ++k) a[k] = tile[idx[k]];
        for (int rr = 0; rr < 4; ++rr) {
          double2 acc = make_double2(0.0, 0.0);
          for (int k = 0; k < 4; ++k) acc = cadd(acc, cmul(mats[G.mat + 4 * rr + k], a[k]));
          tile[idx[rr]] = acc;
        }
      }
    }
    __syncthreads();
  }
  for (int j = tid; j < n; j += 256) p[at(j)] = tile[j];
}

// Eq. 3 for one combination of measurement bases `mb` (base-3 digits Z=0,
// X=1, Y=2 per measurement slot, slot 0 most significant): for every variant
// s and output x, and every Pauli row b that this basis combination serves
// (slots measured in Z serve b = I and b = Z, X serves X, Y serves Y),
// P[s][b][x] = sum_m (prod_j sign(b_j, m_j)) p_s(x, m).
// ROT: the state is the one before measurement and the kernel applies the
// basis changes itself (H for X, S^dagger then H for Y on each measured
// qubit) to the 2^k_out amplitudes of each output it holds, with the
// arithmetic of the gate kernels (so the result is the same as rotating a
// copy of the state first); for at most 4 measured qubits.
template <bool ROT>
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
    if constexpr (ROT) {
      constexpr int NM = 1 << kMaxRotSim;
      double2 amp[NM];
      for (int m = 0; m < nm; ++m) {
        int64_t y = ybase;
        for (int j = 0; j < a.k_out; ++j)
          if ((m >> (a.k_out - 1 - j)) & 1) y |= int64_t(1) << a.meas_bit[j];
        amp[m] = p[y];
      }
      const double r = 0.70710678118654752440;
      for (int j = 0; j < a.k_out; ++j) {
        if (basis[j] == 0) continue;
        // X: (1/sqrt2) [[1, 1], [1, -1]]; Y: (1/sqrt2) [[1, -i], [1, i]]
        const double2 u00 = make_double2(r, 0.0), u10 = make_double2(r, 0.0);
        const double2 u01 = basis[j] == 1 ? make_double2(r, 0.0) : make_double2(0.0, -r);
        const double2 u11 = basis[j] == 1 ? make_double2(-r, 0.0) : make_double2(0.0, r);
        const int bit = 1 << (a.k_out - 1 - j);
        for (int m = 0; m < nm; ++m) {
          if (m & bit) continue;
          const double2 a0 = amp[m], a1 = amp[m | bit];
          amp[m] = cadd(cmul(u00, a0), cmul(u01, a1));
          amp[m | bit] = cadd(cmul(u10, a0), cmul(u11, a1));
        }
      }
      for (int m = 0; m < nm; ++m) pr[m] = amp[m].x * amp[m].x + amp[m].y * amp[m].y;
    } else {
      for (int m = 0; m < nm; ++m) {
        int64_t y = ybase;
        for (int j = 0; j < a.k_out; ++j)
          if ((m >> (a.k_out - 1 - j)) & 1) y |= int64_t(1) << a.meas_bit[j];
        const double2 v = p[y];
        pr[m] = v.x * v.x + v.y * v.y;
      }
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
  if (sp.k_out > kMaxRotSim) CUTQC_CUDA(cudaMalloc(&phi, (size_t)dim * nb * sizeof(double2)));
  CUTQC_CUDA(cudaMalloc(&P, (size_t)total * sizeof(double)));
  try {
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
    std::vector<double2> mt;
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
          f.p0 = pos[sp.d - 1 - sp.gates[g].q0];
          f.p1 = f.nq == 2 ? pos[sp.d - 1 - sp.gates[g].q1] : 0;
          f.mat = (int)mt.size();
          mt.insert(mt.end(), mats[g].first.begin(), mats[g].first.begin() + (f.nq == 2 ? 16 : 4));
          fg.push_back(f);
        }
        gi = gj;
      }
    }
    FusedGate* dg = nullptr;
    double2* dm = nullptr;
    if (!fg.empty()) {
      CUTQC_CUDA(cudaMalloc(&dg, fg.size() * sizeof(FusedGate)));
      CUTQC_CUDA(cudaMalloc(&dm, mt.size() * sizeof(double2)));
      CUTQC_CUDA(cudaMemcpy(dg, fg.data(), fg.size() * sizeof(FusedGate), cudaMemcpyHostToDevice));
      CUTQC_CUDA(cudaMemcpy(dm, mt.data(), mt.size() * sizeof(double2), cudaMemcpyHostToDevice));
    }
    struct FreeTables {
      FusedGate* g;
      double2* m;
      ~FreeTables() {
        if (g) cudaFree(g);
        if (m) cudaFree(m);
      }
    } free_tables{dg, dm};
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
      for (int mb = 0; mb < nmb; ++mb) {
        if (sp.k_out <= kMaxRotSim) {
          // the basis changes inside the attribution: no copy of the state
          k_attr_meas<true><<<grid_for((int64_t(1) << sp.n_eff) * n), 256, 0, s>>>(psi, a, s0, n, mb, P);
          count_launch();
          check_launch("k_attr_meas");
          continue;
        }
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
        k_attr_meas<false><<<grid_for((int64_t(1) << sp.n_eff) * n), 256, 0, s>>>(phi, a, s0, n, mb, P);
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

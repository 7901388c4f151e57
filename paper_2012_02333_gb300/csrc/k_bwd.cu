// Adjoint of the reconstruction (not in the paper): dL/dT for an expectation
// value L = sum_x G(x) p(x) over the reconstructed distribution.
//
// With the final contraction P[m][n] = s * sum_e A[e][m] B[e][n] (s = 2^-K)
// and g = depA(m) + depB(n):
//   dL/dA[e][m] = s * sum_n G[g(m,n)] B[e][n],   dL/dB[e][n] = s * sum_m G[g(m,n)] A[e][m].
// Nothing per term is stored: the partials are recomputed from A and B.
//
// Explicit G (k_bwd_cc): a tiled CUDA-core contraction over the other side's
// output index, G gathered through the deposit tables.
//
// MaxCut G (k_bwd_rowsums, k_bwd_maxcut_grad, k_bwd_maxcut_loss): with the
// qubits split between the two sides, the cut count separates as
//   C(m, n) = C_A(m) + C_B(n) + sum_bridges [bit_i(m) != bit_j(n)],
// so dL/dA[e][m] = s * (C_A(m) S_B[e] + W_B[e] + sum_k Sel_B[k][1 - bit_ik(m)][e])
// with per-row sums S (plain), W (weighted by C), Sel (restricted to one bit
// value of a bridge endpoint).  G(x) is never materialised and the work is
// linear in the tensors' size.
#include <cuda_runtime.h>

#include "internal.h"

namespace cutqc {

namespace {

__device__ __forceinline__ uint64_t dep_tab(const uint64_t* __restrict__ tab, int nbytes, uint64_t v) {
  uint64_t g = 0;
  for (int b = 0; b < nbytes; ++b) g += __ldg(tab + b * 256 + ((v >> (8 * b)) & 255));
  return g;
}

__device__ __forceinline__ int cut_count(uint64_t v, const BwdEdges& ed) {
  int c = 0;
  for (int k = 0; k < ed.n; ++k) c += (int)(((v >> ed.p[k]) ^ (v >> ed.q[k])) & 1);
  return c;
}

// ---- MaxCut: per-row sums in FP64 (block per row) --------------------------
// out[row] = S, out[rows + row] = W, out[(2 + k) * rows + row] = Sel[k] (bit = 1)
template <typename T>
__global__ void k_bwd_rowsums(const T* __restrict__ X, int64_t cols, int64_t rows, BwdEdges internal,
                              BwdBits sel, double* __restrict__ out) {
  __shared__ double red[8][2 + 16];
  const int64_t row = blockIdx.x;
  const T* r = X + row * cols;
  double s = 0.0, w = 0.0, sb[16];
  for (int k = 0; k < sel.n; ++k) sb[k] = 0.0;
  for (int64_t m = threadIdx.x; m < cols; m += blockDim.x) {
    const double v = (double)r[m];
    s += v;
    w += v * cut_count((uint64_t)m, internal);
    for (int k = 0; k < sel.n; ++k)
      if ((m >> sel.p[k]) & 1) sb[k] += v;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    w += __shfl_xor_sync(0xffffffffu, w, o);
  }
  for (int k = 0; k < sel.n; ++k)
    for (int o = 16; o > 0; o >>= 1) sb[k] += __shfl_xor_sync(0xffffffffu, sb[k], o);
  if (lane == 0) {
    red[wid][0] = s;
    red[wid][1] = w;
    for (int k = 0; k < sel.n; ++k) red[wid][2 + k] = sb[k];
  }
  __syncthreads();
  if (threadIdx.x < 2 + sel.n) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i][threadIdx.x];
    out[(int64_t)threadIdx.x * rows + row] = t;
  }
}

// dX[rowX(e)][m] = s * (C_X(m) S_Y[rowY(e)] + W_Y[rowY(e)] + sum_k Sel_Y(k, 1 - bit_k(m))[rowY(e)])
template <typename T>
__global__ void k_bwd_maxcut_grad(const int32_t* __restrict__ rowX, const int32_t* __restrict__ rowY, int kmax,
                                  int64_t cols, BwdEdges internal, BwdBits bitX, const double* __restrict__ sumsY,
                                  int64_t rowsY, double scale, T* __restrict__ dX) {
  const int64_t tot = (int64_t)kmax * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(t / cols);
    const int64_t m = t % cols;
    const int64_t ry = rowY[e];
    const double S = sumsY[ry], W = sumsY[rowsY + ry];
    double g = cut_count((uint64_t)m, internal) * S + W;
    for (int k = 0; k < bitX.n; ++k) {
      const double s1 = sumsY[(2 + k) * rowsY + ry];
      g += ((m >> bitX.p[k]) & 1) ? (S - s1) : s1;
    }
    dX[(int64_t)rowX[e] * cols + m] = (T)(g * scale);
  }
}

// ---- MaxCut through a per-output key ------------------------------------
// key[m] = C(m) * 2^nsel + (bridge-endpoint bits of m, bit k = sel.p[k]): the
// only two things of m that the row sums and the gradient depend on.  Built
// once per side (2 bytes per output), it replaces the per-element edge loop.
__global__ void k_bwd_keys(int64_t cols, BwdEdges internal, BwdBits sel, uint16_t* __restrict__ keys) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < cols; m += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b = 0;
    for (int k = 0; k < sel.n; ++k) b |= (uint32_t)(((uint64_t)m >> sel.p[k]) & 1) << k;
    keys[m] = (uint16_t)(((uint32_t)cut_count((uint64_t)m, internal) << sel.n) | b);
  }
}

// compensated FP32 running sum (TwoSum; the error of each add is carried in c)
struct BF {
  float s, c;
};
__device__ __forceinline__ BF bf_add(BF a, float b) {
  const float t = a.s + b;
  const float bb = t - a.s;
  return {t, a.c + ((a.s - (t - bb)) + (b - bb))};
}

// FP32 row sums through the keys, one block of 512 threads per row: S, W and
// Sel in compensated FP32 (W adds v * C with the product's rounding error
// recovered exactly by an FMA), four 16-byte loads in flight per thread; FP64
// only for the reduction across threads.  The FP64 pipe is narrow on this
// part, so no FP64 instruction is spent per element.  NS >= the number of
// bridge bits (registers for exactly that many Sel sums).
template <int NS>
__global__ void __launch_bounds__(512) k_bwd_rowsums_keys(const float* __restrict__ X, int64_t cols, int64_t rows,
                                                          int nsel, const uint16_t* __restrict__ keys,
                                                          double* __restrict__ out) {
  constexpr int NV = 2 + NS;
  __shared__ double red[16][NV];
  const int64_t row = blockIdx.x;
  const float4* r = reinterpret_cast<const float4*>(X + row * cols);
  const ushort4* kk = reinterpret_cast<const ushort4*>(keys);
  BF S{0.0f, 0.0f}, W{0.0f, 0.0f}, sb[NS > 0 ? NS : 1];
#pragma unroll
  for (int k = 0; k < NS; ++k) sb[k] = BF{0.0f, 0.0f};
  const int64_t n4 = cols / 4;
  for (int64_t j0 = threadIdx.x; j0 < n4; j0 += 4 * (int64_t)blockDim.x) {
    float4 v4[4];
    ushort4 k4[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = j0 + u * (int64_t)blockDim.x;
      v4[u] = j < n4 ? __ldg(r + j) : make_float4(0.f, 0.f, 0.f, 0.f);
      k4[u] = j < n4 ? __ldg(kk + j) : make_ushort4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float v[4] = {v4[u].x, v4[u].y, v4[u].z, v4[u].w};
      const uint32_t key[4] = {k4[u].x, k4[u].y, k4[u].z, k4[u].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        S = bf_add(S, v[e]);
        const float c = (float)(key[e] >> nsel);
        const float p = v[e] * c;
        W = bf_add(W, p);
        W.c += fmaf(v[e], c, -p);   // the exact rounding error of the product
#pragma unroll
        for (int k = 0; k < NS; ++k)
          if (k < nsel) sb[k] = bf_add(sb[k], ((key[e] >> k) & 1) ? v[e] : 0.0f);
      }
    }
  }
  double t[NV];
  t[0] = (double)S.s + (double)S.c;
  t[1] = (double)W.s + (double)W.c;
#pragma unroll
  for (int k = 0; k < NS; ++k) t[2 + k] = (double)sb[k].s + (double)sb[k].c;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[i] += __shfl_xor_sync(0xffffffffu, t[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[wid][i] = t[i];
  __syncthreads();
  if (threadIdx.x < 2 + nsel) {
    double a = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i][threadIdx.x];
    out[(int64_t)threadIdx.x * rows + row] = a;
  }
}

// The gradient through the keys: for row e, dX[rowX(e)][m] depends on m only
// through key[m], so each block first evaluates the (C_max + 1) * 2^nsel
// values in FP64, in the order k_bwd_maxcut_grad uses, rounded once to T, and
// then writes table[key[m]] for its share of the row (4 outputs per step):
// the results equal k_bwd_maxcut_grad's bit for bit.  Grid: rows x chunks.
template <typename T>
__global__ void k_bwd_maxcut_grad_keys(const int32_t* __restrict__ rowX, const int32_t* __restrict__ rowY, int kmax,
                                       int64_t cols, int nchunk, int ntab, int nsel,
                                       const uint16_t* __restrict__ keys, const double* __restrict__ sumsY,
                                       int64_t rowsY, double scale, T* __restrict__ dX) {
  __shared__ T tab[4096];
  const int e = (int)(blockIdx.x / nchunk), ch = (int)(blockIdx.x % nchunk);
  if (e >= kmax) return;
  const int64_t ry = rowY[e];
  const double S = sumsY[ry], W = sumsY[rowsY + ry];
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) {
    const int c = i >> nsel;
    double g = c * S + W;
    for (int k = 0; k < nsel; ++k) {
      const double s1 = sumsY[(2 + k) * rowsY + ry];
      g += ((i >> k) & 1) ? (S - s1) : s1;
    }
    tab[i] = (T)(g * scale);
  }
  __syncthreads();
  const int64_t per = cols / 4 / nchunk;   // groups of 4 outputs in this block's chunk
  const int64_t j0 = (int64_t)ch * per;
  T* drow = dX + (int64_t)rowX[e] * cols;
  const ushort4* kk = reinterpret_cast<const ushort4*>(keys);
  for (int64_t j = j0 + threadIdx.x; j < j0 + per; j += blockDim.x) {
    const ushort4 k4 = __ldg(kk + j);
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float4*>(drow)[j] = make_float4(tab[k4.x], tab[k4.y], tab[k4.z], tab[k4.w]);
    } else {
      reinterpret_cast<double2*>(drow)[2 * j] = make_double2(tab[k4.x], tab[k4.y]);
      reinterpret_cast<double2*>(drow)[2 * j + 1] = make_double2(tab[k4.z], tab[k4.w]);
    }
  }
}

// L = s * sum_e [W_A S_B + S_A W_B + sum_k (Sel_A1 (S_B - Sel_B1) + (S_A - Sel_A1) Sel_B1)]
__global__ void k_bwd_maxcut_loss(const int32_t* __restrict__ rowA, const int32_t* __restrict__ rowB, int kmax,
                                  const double* __restrict__ sA, int64_t rowsA, const double* __restrict__ sB,
                                  int64_t rowsB, int nbridge, double scale, double* __restrict__ loss) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int e = threadIdx.x; e < kmax; e += blockDim.x) {
    const int64_t a = rowA[e], b = rowB[e];
    const double SA = sA[a], WA = sA[rowsA + a], SB = sB[b], WB = sB[rowsB + b];
    double v = WA * SB + SA * WB;
    for (int k = 0; k < nbridge; ++k) {
      const double a1 = sA[(2 + k) * rowsA + a], b1 = sB[(2 + k) * rowsB + b];
      v += a1 * (SB - b1) + (SA - a1) * b1;
    }
    acc += v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *loss = t * scale;
  }
}

// ---- explicit G: dX[rowX(e)][m] = s * sum_n G[depX(m) + depY(n)] Y[rowY(e)][n]
// tile 64 (e) x 64 (m), inner step 16 over n, 256 threads with 4 x 4 outputs
template <typename T>
__global__ void __launch_bounds__(256) k_bwd_cc(const T* __restrict__ Y, const T* __restrict__ G,
                                               const int32_t* __restrict__ rowX, const int32_t* __restrict__ rowY,
                                               int kmax, int64_t colsX, int64_t colsY, const uint64_t* __restrict__ depX,
                                               int nbX, const uint64_t* __restrict__ depY, int nbY, T scale,
                                               T* __restrict__ dX) {
  __shared__ T Ys[16][64 + 1];   // [n][e]
  __shared__ T Gs[16][64 + 1];   // [n][m]
  __shared__ uint64_t gm[64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t tilesM = (colsX + 63) / 64;
  const int e0 = (int)(blockIdx.x / tilesM) * 64;
  const int64_t m0 = (blockIdx.x % tilesM) * 64;
  if (tid < 64) gm[tid] = (m0 + tid < colsX) ? dep_tab(depX, nbX, (uint64_t)(m0 + tid)) : 0;
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int64_t n0 = 0; n0 < colsY; n0 += 16) {
    // load 64 e x 16 n of Y and 64 m x 16 n of G
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = tid + 256 * r;
      const int nn = idx & 15, ee = idx >> 4;
      const int e = e0 + ee;
      const int64_t n = n0 + nn;
      Ys[nn][ee] = (e < kmax && n < colsY) ? Y[(int64_t)rowY[e] * colsY + n] : T(0);
      const int mm = ee;
      Gs[nn][mm] = (m0 + mm < colsX && n < colsY) ? G[gm[mm] + dep_tab(depY, nbY, (uint64_t)n)] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = Ys[k][ty * 4 + i];
        b[i] = Gs[k][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = e0 + ty * 4 + i;
    if (e >= kmax) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t m = m0 + tx * 4 + j;
      if (m < colsX) dX[(int64_t)rowX[e] * colsX + m] = acc[i][j] * scale;
    }
  }
}

// L = sum over all entries of dX * X (the loss from one side's gradient), FP64
template <typename T>
__global__ void k_dot(const T* __restrict__ a, const T* __restrict__ b, int64_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(out, t);
  }
}

unsigned grid_for(int64_t work) {
  int64_t g = (work + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

size_t bwd_keys_bytes(int f, const BwdEdges& internal, const BwdBits& sel) {
  if (f < 3 || f > 24 || ((int64_t)(internal.n + 1) << sel.n) > 4096) return 0;
  return ((size_t(2) << f) + 255) / 256 * 256;
}

void launch_bwd_keys(int f, const BwdEdges& internal, const BwdBits& sel, uint16_t* keys, cudaStream_t s) {
  if (!bwd_keys_bytes(f, internal, sel)) fail(CUTQC_ERR_UNSUPPORTED, "no key table for this shape");
  const int64_t cols = int64_t(1) << f;
  k_bwd_keys<<<grid_for(cols), 256, 0, s>>>(cols, internal, sel, keys);
  count_launch();
  check_launch("k_bwd_keys");
}

void launch_bwd_rowsums(const void* X, int dtype, int64_t rows, int f, const BwdEdges& internal,
                        const BwdBits& sel, double* out, cudaStream_t s, const uint16_t* keys) {
  const int64_t cols = int64_t(1) << f;
  if (keys && dtype == CUTQC_F32 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    const float* Xf = static_cast<const float*>(X);
    if (sel.n <= 2)
      k_bwd_rowsums_keys<2><<<(unsigned)rows, 512, 0, s>>>(Xf, cols, rows, sel.n, keys, out);
    else if (sel.n <= 4)
      k_bwd_rowsums_keys<4><<<(unsigned)rows, 512, 0, s>>>(Xf, cols, rows, sel.n, keys, out);
    else
      k_bwd_rowsums_keys<16><<<(unsigned)rows, 512, 0, s>>>(Xf, cols, rows, sel.n, keys, out);
    count_launch();
    check_launch("k_bwd_rowsums_keys");
    return;
  }
  if (dtype == CUTQC_F64)
    k_bwd_rowsums<double><<<(unsigned)rows, 256, 0, s>>>(static_cast<const double*>(X), cols, rows, internal, sel, out);
  else
    k_bwd_rowsums<float><<<(unsigned)rows, 256, 0, s>>>(static_cast<const float*>(X), cols, rows, internal, sel, out);
  count_launch();
  check_launch("k_bwd_rowsums");
}

void launch_bwd_maxcut_grad(const int32_t* rowX, const int32_t* rowY, int kmax, int fX, const BwdEdges& internal,
                            const BwdBits& bitX, const double* sumsY, int64_t rowsY, double scale, void* dX, int dtype,
                            cudaStream_t s, const uint16_t* keys) {
  const int64_t cols = int64_t(1) << fX;
  if (keys && (reinterpret_cast<uintptr_t>(dX) & 15) == 0) {
    // chunks of at least 1024 outputs, enough blocks to fill the GPU
    int nchunk = 1;
    while ((int64_t)kmax * nchunk < 152 * 8 && cols / 4 / (nchunk * 2) >= 256) nchunk *= 2;
    const int ntab = (internal.n + 1) << bitX.n;
    const unsigned g = (unsigned)((int64_t)kmax * nchunk);
    if (dtype == CUTQC_F64)
      k_bwd_maxcut_grad_keys<double><<<g, 256, 0, s>>>(rowX, rowY, kmax, cols, nchunk, ntab, bitX.n, keys, sumsY,
                                                        rowsY, scale, static_cast<double*>(dX));
    else
      k_bwd_maxcut_grad_keys<float><<<g, 256, 0, s>>>(rowX, rowY, kmax, cols, nchunk, ntab, bitX.n, keys, sumsY,
                                                       rowsY, scale, static_cast<float*>(dX));
    count_launch();
    check_launch("k_bwd_maxcut_grad_keys");
    return;
  }
  const unsigned g = grid_for((int64_t)kmax * cols);
  if (dtype == CUTQC_F64)
    k_bwd_maxcut_grad<double><<<g, 256, 0, s>>>(rowX, rowY, kmax, cols, internal, bitX, sumsY, rowsY, scale,
                                                 static_cast<double*>(dX));
  else
    k_bwd_maxcut_grad<float><<<g, 256, 0, s>>>(rowX, rowY, kmax, cols, internal, bitX, sumsY, rowsY, scale,
                                                static_cast<float*>(dX));
  count_launch();
  check_launch("k_bwd_maxcut_grad");
}

void launch_bwd_maxcut_loss(const int32_t* rowA, const int32_t* rowB, int kmax, const double* sA, int64_t rowsA,
                            const double* sB, int64_t rowsB, int nbridge, double scale, double* loss, cudaStream_t s) {
  k_bwd_maxcut_loss<<<1, 1024, 0, s>>>(rowA, rowB, kmax, sA, rowsA, sB, rowsB, nbridge, scale, loss);
  count_launch();
  check_launch("k_bwd_maxcut_loss");
}

void launch_bwd_cc(const void* Y, const void* G, const int32_t* rowX, const int32_t* rowY, int kmax, int fX, int fY,
                   const uint64_t* depX, const uint64_t* depY, double scale, void* dX, int dtype, cudaStream_t s) {
  const int64_t colsX = int64_t(1) << fX, colsY = int64_t(1) << fY;
  const int64_t tiles = ((kmax + 63) / 64) * ((colsX + 63) / 64);
  const int nbX = (fX + 7) / 8, nbY = (fY + 7) / 8;
  if (dtype == CUTQC_F64)
    k_bwd_cc<double><<<(unsigned)tiles, 256, 0, s>>>(static_cast<const double*>(Y), static_cast<const double*>(G),
                                                     rowX, rowY, kmax, colsX, colsY, depX, nbX, depY, nbY, scale,
                                                     static_cast<double*>(dX));
  else
    k_bwd_cc<float><<<(unsigned)tiles, 256, 0, s>>>(static_cast<const float*>(Y), static_cast<const float*>(G), rowX,
                                                    rowY, kmax, colsX, colsY, depX, nbX, depY, nbY, (float)scale,
                                                    static_cast<float*>(dX));
  count_launch();
  check_launch("k_bwd_cc");
}

void launch_dot(const void* a, const void* b, int64_t n, int dtype, double* out, cudaStream_t s) {
  if (dtype == CUTQC_F64)
    k_dot<double><<<grid_for(n), 256, 0, s>>>(static_cast<const double*>(a), static_cast<const double*>(b), n, out);
  else
    k_dot<float><<<grid_for(n), 256, 0, s>>>(static_cast<const float*>(a), static_cast<const float*>(b), n, out);
  count_launch();
  check_launch("k_dot");
}

}  // namespace cutqc

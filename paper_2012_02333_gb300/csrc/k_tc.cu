// tcgen05 split-precision reconstruction (BF16 x3 / x6, FP32 accumulation in TMEM).
//
// The final contraction of the 4^K sum (Sec. 3.3), P[m][n] = 2^-K sum_e
// A[e][m] B[e][n], runs on the 5th-generation tensor cores.  Each FP32
// operand x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi), and
//   A.B ~= A_hi.B_hi + A_hi.B_lo + A_lo.B_hi
// (the lo.lo term is ~2^-16 relative).  The bf16 pieces are stored MN-major
// (one row of M or N values per kept term, the layout the tensors already
// have) and each pipeline stage holds every piece of one 32-wide k step, so
// one stage feeds all the products (hh, hm, mh; the x6 form splits into three
// pieces and adds hl, lh, mm for FP32-level accuracy).  The number of
// products is read on the device (chosen from an a-priori bound while the
// operands are prepared) so no host round trip is needed.
//
// Operand preparation finds the non-zero Kronecker terms (early termination,
// Sec. 4.2) and the split count, and writes the split pieces of the kept
// rows: k_pair_prep in one pass (one block per term, a look-back over the
// other terms' flags for its compacted row), k_stats_prep in two phases
// around a grid barrier (fewer terms than blocks, or TF32), k_prep when the
// statistics come from an earlier launch.
//
// k_tc_gemm: persistent, one CTA per SM, 192 threads:
//   warp 0     TMA producer: the split pieces of 32x128 A tiles and 32x256
//              B tiles (k x M / N, 128-byte swizzle, 64-element chunks) into
//              a 4-stage (x3) or 3-stage (x6) shared-memory ring;
//   warp 1     allocates 512 TMEM columns (two 128x256 FP32 accumulators)
//              and one thread issues tcgen05.mma (M=128, N=256, K=16);
//   warps 2-5  epilogue (one per TMEM lane quarter; EPI_WARPS = 8 splits the
//              columns between two warps per quarter): tcgen05.ld of their 32
//              TMEM lanes (lane = row),
//              scale by 2^-K, deposit (m, n) into the output index with the
//              additive per-bit tables held in registers, restage 16 x 32
//              blocks through shared memory so 16-byte streaming stores go
//              out in output-address order, compensated FP32 partial sums
//              (FP64 across threads); it drains one
//              accumulator while the MMA fills the other.
// Every wait on an mbarrier is bounded (2 s); on timeout the kernel raises an
// abort flag, records a status word, lets in-flight copies land and frees TMEM.
//
// TF32 x3 (the same kernels, instantiated with TF32 = true): the split of
// Ootomo and Yokota (2022) with TF32 pieces, x_hi = rna_tf32(x) and
// x_lo = rna_tf32(x - x_hi), both kept in FP32 containers with the low 13
// mantissa bits zero, and the products hi*hi + hi*lo + lo*hi with
// tcgen05.mma kind::tf32 (K = 8).  TF32 has FP32's exponent range, so no
// scaling of the lo piece is needed; the dropped lo*lo term and the rounding
// of the lo piece bound the error per product by about 3 * 2^-22 |a||b|.  A
// stage then holds 16 k of each piece, K-major (TF32 pieces are kept in the
// K-major layout, 64-byte rows of 16 k), the same stage sizes as BF16.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cfloat>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace cutqc {

namespace {

constexpr int BM = 128, BN = 256;
constexpr int BK = 64;                        // operand preparation works in 64-wide k blocks
constexpr int KS = 32;                        // one pipeline stage: 32 k = 64 bytes = one 64-byte swizzle row
constexpr int MN_CHUNK = 64;                  // MN-major bf16 stages: 64-element (128-byte) rows of one k
constexpr int MN_CHUNK_BYTES = MN_CHUNK * KS * 2;   // one chunk: 32 k rows of 128 bytes
constexpr int A_PIECE = BM * KS * 2;          // 8 KiB per split piece of A
constexpr int B_PIECE = BN * KS * 2;          // 16 KiB per split piece of B
constexpr int MAX_STAGES = 4;
constexpr int STAGE_AREA = 3 * 3 * (A_PIECE + B_PIECE);   // 216 KiB: 3 stages of 3 pieces or 4 of 2
constexpr int TMEM_COLS = 512;
constexpr int EPI_WARPS = 4;                  // one per TMEM lane quarter (8 measured slower)
constexpr int THREADS = 64 + 32 * EPI_WARPS;
// epilogue staging: per epilogue warp 16 rows x 32 columns of FP32, rows
// padded to 36 floats (conflict-free 16-byte writes)
constexpr int EPI_LD = 36;
constexpr int EPI_BUF = 16 * EPI_LD * 4;
constexpr size_t SMEM_BYTES = size_t(STAGE_AREA) + 1024 + 256 + size_t(EPI_WARPS) * EPI_BUF;
static_assert(SMEM_BYTES <= 232448, "shared memory per block");
constexpr long long WAIT_CYCLES = 4000000000ll;   // ~2 s at 2 GHz
// the one-pass preparation runs one block per Kronecker term, with both rows
// in registers: below this many terms the two-phase launch (statistics over
// rows, then tiles) keeps more SMs busy; rows longer than 4096 values, or
// more terms than resident blocks, go to the two-phase launch as well (a
// streamed one-pass form measured slower there)
constexpr int PAIR_PREP_MIN_TERMS = 128;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------ operand prep
// Each FP32 x is split into h = bf16(x), m = bf16(x - h), l = bf16(x - h - m).
// Segment s of the concatenated inner dimension pairs part PA[s] of A with
// part PB[s] of B (0 = h, 1 = m, 2 = l): hh, hm, mh | hl, lh, mm.  The first
// three segments are the x3 form, all six the x6 form.
__constant__ int kPartA[6] = {0, 0, 1, 0, 2, 1};
__constant__ int kPartB[6] = {0, 1, 0, 2, 0, 1};

struct PrepArgs {
  const float* T[2];          // A, B tensors
  int64_t cols[2];            // 2^fA, 2^fB
  int blocks0;                // column blocks of A (cols[0] / 64)
  int Kp, kmax;
  int fused;                  // compaction done here (kmax <= 4096) or read from crow / kcount / nseg
  const int32_t* rows;        // [2][kmax] row pairs (fused)
  const int32_t* crow;        // [2][kmax] compacted row pairs (not fused)
  const int32_t* nzA;
  const int32_t* nzB;
  const float* rmaxA;
  const float* rmaxB;
  double scale, split_tol;
  int nseg_fixed;
  int32_t* kcount;
  int32_t* nseg;
  double* bound;
  double* sum_zero;
  void* out[2];               // A', B': [piece][cols][Kp] (bf16, or FP32 containers of TF32 pieces)
};

// round to the nearest TF32 value (ties away from zero), kept in an FP32
// container with the low 13 mantissa bits zero
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// the three BF16 pieces of 4 FP32 values, each packed as 4 consecutive bf16
// (8 bytes): h = bf16(x), m = bf16(x - h), l = bf16(x - h - m); both
// differences are exact in FP32
__device__ __forceinline__ void split3_bf16x4(const float4 v, uint2 (&pc)[3]) {
  const float x[4] = {v.x, v.y, v.z, v.w};
  __nv_bfloat16 h[4], m[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = __float2bfloat16_rn(x[j]);
    const float r1 = x[j] - __bfloat162float(h[j]);
    m[j] = __float2bfloat16_rn(r1);
    l[j] = __float2bfloat16_rn(r1 - __bfloat162float(m[j]));
  }
  auto pack = [](const __nv_bfloat16 (&b)[4]) {
    uint2 u;
    u.x = (uint32_t)__bfloat16_as_ushort(b[0]) | ((uint32_t)__bfloat16_as_ushort(b[1]) << 16);
    u.y = (uint32_t)__bfloat16_as_ushort(b[2]) | ((uint32_t)__bfloat16_as_ushort(b[3]) << 16);
    return u;
  };
  pc[0] = pack(h);
  pc[1] = pack(m);
  pc[2] = pack(l);
}

// The pieces of T[row(k)][m] for the k-th kept term (0 for kcount <= k <
// Kp): h and m for the x3 form, h, m and l for x6.  BF16 pieces are
// MN-major, out[piece][k][m] with row pitch cols; TF32 pieces K-major,
// out[piece][m][k] with row pitch Kp.  One launch for
// both operands: blocks [0, blocks0) prepare A, the rest B.  When `fused`,
// every block finds its own compacted rows (a block-wide stable scan of the
// row pairs: early termination, Sec. 4.2) and the split count from the bound
// S = scale * sum_kept max|A| max|B|; block (0, 0) publishes the count, the
// split count and S for the contraction and zeroes the FP64 sum.
// One 64 (k) x 64 (m) tile of the operand preparation; (bx, by) = (column
// block over A then B, k block).  The row statistics it reads (fused mode)
// may have been written by the same kernel before a grid barrier, so they are
// read through L2 (__ldcg), never through a stale L1 line.
// pre_r0 / pre_r1: this thread's row pair t = threadIdx.x, read before the
// call (pre = true), for the first pass of the fused scan
template <bool TF32>
__device__ __forceinline__ void prep_tile(const PrepArgs& a, const int bx, const int by, const bool pre = false,
                                          const int pre_r0 = 0, const int pre_r1 = 0) {
  __syncthreads();   // the shared arrays may still be read by the previous tile
  __shared__ float s[64][65];
  __shared__ int32_t rowsel[64];
  __shared__ int warp_tot[8];
  __shared__ float warp_s[8];
  __shared__ int base_s, kc_s, nseg_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int which = bx < a.blocks0 ? 0 : 1;
  const int64_t m0 = (int64_t)(which == 0 ? bx : bx - a.blocks0) * 64;
  const int k0 = by * 64;
  const int64_t cols = a.cols[which];
  const float* T = a.T[which];
  if (a.fused) {
    if (tid == 0) base_s = 0;
    __syncthreads();
    float sacc = 0.0f;   // the bound in FP32 (a magnitude estimate; the FP64 pipe is narrow)
    const int32_t* ra = a.rows;
    const int32_t* rb = a.rows + a.kmax;
    for (int t0 = 0; t0 < a.kmax; t0 += 256) {
      const int t = t0 + tid;
      int keep = 0, r0 = 0, r1 = 0;
      float mxa = 0.0f, mxb = 0.0f;
      if (t < a.kmax) {
        r0 = (pre && t0 == 0) ? pre_r0 : ra[t];
        r1 = (pre && t0 == 0) ? pre_r1 : rb[t];
        // flags and maxima in one round trip (the maxima count only when kept)
        const int nza = __ldcg(a.nzA + r0), nzb = __ldcg(a.nzB + r1);
        mxa = __ldcg(a.rmaxA + r0);
        mxb = __ldcg(a.rmaxB + r1);
        keep = nza && nzb;
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) warp_tot[warp] = __popc(m);
      __syncthreads();
      int off = 0, tot = 0;
      for (int w = 0; w < 8; ++w) {
        if (w < warp) off += warp_tot[w];
        tot += warp_tot[w];
      }
      if (keep) {
        const int ci = base_s + off + __popc(m & ((1u << lane) - 1u));
        if (ci >= k0 && ci < k0 + 64) rowsel[ci - k0] = which == 0 ? r0 : r1;
        sacc = fmaf(mxa, mxb, sacc);
      }
      __syncthreads();
      if (tid == 0) base_s += tot;
      __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
    if (lane == 0) warp_s[warp] = sacc;
    __syncthreads();
    if (tid == 0) {
      float Sf = 0.0f;
      for (int w = 0; w < 8; ++w) Sf += warp_s[w];
      // FP32 accumulation error is far below 1e-4 relative: inflate so S stays an upper bound
      const double S = (double)Sf * a.scale * (1.0 + 1e-4);
      // BF16 x3 drops terms of at most ~3 * 2^-18 |a||b| per product
      const int ns = a.nseg_fixed ? a.nseg_fixed : (3.0 * 3.814697265625e-06 * S <= a.split_tol ? 3 : 6);
      kc_s = base_s;
      nseg_s = ns;
      if (bx == 0 && by == 0) {
        *a.kcount = base_s;
        *a.nseg = ns;
        *a.bound = S;
        if (a.sum_zero) *a.sum_zero = 0.0;
      }
    }
  } else {
    if (tid == 0) {
      kc_s = *a.kcount;
      nseg_s = *a.nseg;
    }
    __syncthreads();
    if (tid < 64 && k0 + tid < kc_s) rowsel[tid] = a.crow[which * a.kmax + k0 + tid];
  }
  __syncthreads();
  const int kc = kc_s, nseg = nseg_s;
  // the contraction reads k < 32 * ceil(kc / 32): tiles past that write nothing
  if (k0 >= (kc + 31) / 32 * 32) return;
  if constexpr (TF32) {
    {
      // all 16 loads first (read-only path), then the shared-memory stores: a
      // load interleaved with stores through a generic pointer would wait for
      // each of them in turn
      float ld[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int kk = i * 4 + tid / 64, mm = tid % 64, k = k0 + kk;
        ld[i] = (k < kc) ? __ldg(T + (int64_t)rowsel[kk] * cols + m0 + mm) : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) s[i * 4 + tid / 64][tid % 64] = ld[i];
    }
    __syncthreads();
    const int ml = tid / 4, kq = (tid % 4) * 16;
    __align__(16) float part[2][16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float v = s[kq + j][ml];
      const float h = tf32_rna(v);
      part[0][j] = h;
      part[1][j] = tf32_rna(v - h);   // v - h is exact in FP32
    }
    float* out = static_cast<float*>(a.out[which]);
#pragma unroll
    for (int pc = 0; pc < 2; ++pc) {
      const uint4* src = reinterpret_cast<const uint4*>(part[pc]);
      uint4* dst = reinterpret_cast<uint4*>(out + ((int64_t)pc * cols + m0 + ml) * a.Kp + k0 + kq);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = src[q];
    }
  } else {
    // BF16 pieces, MN-major (out[piece][k][m], rows of `cols`): no transpose;
    // thread (kr, mq) takes 4 consecutive m of k rows kr, kr + 16, ...
    const int mq = (tid & 15) * 4, kr = tid >> 4;
    float4 ld[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int kk = p * 16 + kr;
      ld[p] = (k0 + kk < kc) ? __ldg(reinterpret_cast<const float4*>(T + (int64_t)rowsel[kk] * cols + m0 + mq))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __nv_bfloat16* out = static_cast<__nv_bfloat16*>(a.out[which]);
    const int npieces = nseg == 3 ? 2 : 3;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      uint2 pc4[3];
      split3_bf16x4(ld[p], pc4);
      const int64_t row = k0 + p * 16 + kr;
#pragma unroll
      for (int pc = 0; pc < 3; ++pc)
        if (pc < npieces)
          *reinterpret_cast<uint2*>(out + ((int64_t)pc * a.Kp + row) * cols + m0 + mq) = pc4[pc];
    }
  }
}

template <bool TF32>
__global__ void __launch_bounds__(256) k_prep(const PrepArgs a) {
  CUTQC_PDL_WAIT();     // row statistics come from the previous kernel
  CUTQC_PDL_LAUNCH();   // the contraction may launch and set itself up
  prep_tile<TF32>(a, blockIdx.x, blockIdx.y);
}

// ---- row statistics + compaction + operand preparation in one launch -----
// Phase 1: one block per row of A then B (grid-stride): non-zero flag and
// max |x| (the early-termination test of Sec. 4.2 and the split bound).
// A grid barrier (cooperative launch, so every block is resident; the wait is
// bounded and a timeout sets the status word and ends the block).  Phase 2:
// the operand-preparation tiles (grid-stride), each block scanning the row
// flags itself (fused compaction).
struct StatsArgs {
  int64_t rows[2];
  int32_t* nz[2];
  float* rmax[2];
  unsigned* barrier;   // zeroed before the launch (its own per problem: batches run concurrently)
  int* status;
  int tilesX, tilesY;
};

__device__ __forceinline__ void stats_row(const float* __restrict__ row, int64_t cols, int32_t* flag, float* rmax) {
  __shared__ float red[8];
  __shared__ int nzs[8];
  float m = 0.0f;
  int nz = 0;
  const float4* rv = reinterpret_cast<const float4*>(row);
  const int64_t nv = cols / 4;
  for (int64_t i0 = threadIdx.x; i0 < nv; i0 += 4 * (int64_t)blockDim.x) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + (int64_t)u * blockDim.x;
      v[u] = i < nv ? __ldg(rv + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      nz |= (v[u].x != 0.f) | (v[u].y != 0.f) | (v[u].z != 0.f) | (v[u].w != 0.f);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w))));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    nz |= __shfl_xor_sync(0xffffffffu, nz, o);
  }
  __syncthreads();   // red / nzs may still be read for the previous row
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = m;
    nzs[threadIdx.x >> 5] = nz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      m = fmaxf(m, red[w]);
      nz |= nzs[w];
    }
    *flag = nz;
    *rmax = m;
  }
}

template <bool TF32>
__global__ void __launch_bounds__(256) k_stats_prep(const PrepArgs a, const StatsArgs sa) {
  CUTQC_PDL_LAUNCH();   // the contraction may launch and set itself up
  // the first 256 row pairs of the compaction are plan data: read them now
  int pre_r0 = 0, pre_r1 = 0;
  if ((int)threadIdx.x < a.kmax) {
    pre_r0 = __ldg(a.rows + threadIdx.x);
    pre_r1 = __ldg(a.rows + a.kmax + threadIdx.x);
  }
  const int64_t nrows = sa.rows[0] + sa.rows[1];
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    // selects, not a dynamic index into the parameter arrays (which would
    // copy them to local memory)
    const bool j0 = r < sa.rows[0];
    const int64_t rr = j0 ? r : r - sa.rows[0];
    const int64_t cols = j0 ? a.cols[0] : a.cols[1];
    stats_row((j0 ? a.T[0] : a.T[1]) + rr * cols, cols, (j0 ? sa.nz[0] : sa.nz[1]) + rr,
              (j0 ? sa.rmax[0] : sa.rmax[1]) + rr);
  }
  // grid barrier
  __shared__ int pass;
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: this block's statistics (written by this thread) are visible
    // to any block whose acquire load sees the count
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(sa.barrier) : "memory");
    const uint64_t t0 = gtimer();
    int ok = 1;
    while (ld_acquire(sa.barrier) < gridDim.x) {
      if (gtimer() - t0 > 2000000000ull) {   // 2 s
        ok = 0;
        atomicExch(sa.status, (int)DEV_TIMEOUT);
        break;
      }
      __nanosleep(20);
    }
    pass = ok;
  }
  __syncthreads();
  if (!pass) return;
  for (int t = blockIdx.x; t < sa.tilesX * sa.tilesY; t += gridDim.x)
    prep_tile<TF32>(a, t % sa.tilesX, t / sa.tilesX, true, pre_r0, pre_r1);
}

// ---- operand preparation reading each row once (BF16 pieces, MN-major) ---
// One block per Kronecker term t (a cooperative launch, so every block is
// resident; rows of at most 4096 values): phase 1 reads row rows[t] of A and
// row rows[kmax + t] of B into registers, finds whether both are non-zero
// (early termination, Sec. 4.2) and their max |.|, sets bit t of a kept-term
// mask and the product max|A| max|B| of a kept term, and splits the rows
// into their pieces while one bounded grid barrier completes (one counter,
// polled by one thread per block).  Phase 2: every block reads the mask and
// the products (a few hundred bytes, one round trip), so it knows the kept
// count before its term, the total, and the bound S = scale * sum_kept
// max|A| max|B| (summed in the same fixed order in every block, so all agree
// on the split count), and stores the pieces of a kept term to row
// `kept before t` of every piece matrix, or zero rows at
// kmax - 1 - (terms dropped before t) for a dropped term, written only where
// the contraction's last stage reads (rows below the kept count rounded up
// to a stage, zero rows past kmax included).
struct PairArgs {
  const float* T[2];
  int64_t cols[2];            // at most 4096 each
  int kmax, Kp;
  const int32_t* rows;        // [2][kmax] row pairs
  int32_t* nz[2];             // row flags and maxima (the row statistics of the plan)
  float* rmax[2];
  unsigned* barrier;          // zero before the launch
  unsigned* bits;             // [ceil(kmax / 32)], zero before the launch
  float* prod;                // [kmax]
  double scale, split_tol;
  int nseg_fixed;
  int32_t* kcount;
  int32_t* nseg;
  double* bound;
  double* sum_zero;
  int* status;
  __nv_bfloat16* out[2];      // [piece][Kp][cols]
};

__global__ void __launch_bounds__(256) k_pair_prep(const PairArgs a) {
  CUTQC_PDL_LAUNCH();   // the contraction may launch and set itself up
  __shared__ float red_m[2][8];
  __shared__ int red_z[2][8];
  __shared__ float red_s[8];
  __shared__ unsigned wsm[128];   // the kept-term mask (kmax <= 4096)
  __shared__ int pre_s[128];      // kept terms before each mask word
  __shared__ int pass, nseg_s, kend_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = blockIdx.x;
  if ((int)gridDim.x != a.kmax) {   // one term per block, or the barrier count is wrong
    if (t == 0 && tid == 0) atomicExch(a.status, (int)DEV_BAD_INDEX);
    return;
  }
  const int r0 = __ldg(a.rows + t), r1 = __ldg(a.rows + a.kmax + t);
  // thread j holds 8 consecutive values (2 float4) at j and j + 256 of each
  // row, and later their pieces, 16 bytes each
  const float4* row[2] = {reinterpret_cast<const float4*>(a.T[0] + (int64_t)r0 * a.cols[0]),
                          reinterpret_cast<const float4*>(a.T[1] + (int64_t)r1 * a.cols[1])};
  const int nv[2] = {(int)(a.cols[0] / 4), (int)(a.cols[1] / 4)};
  float4 v[2][2][2];
#pragma unroll
  for (int w = 0; w < 2; ++w)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = tid + 256 * u;
      const bool in = 2 * j < nv[w];
      v[w][u][0] = in ? __ldg(row[w] + 2 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
      v[w][u][1] = in ? __ldg(row[w] + 2 * j + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  float mx[2] = {0.0f, 0.0f};
  int nz[2] = {0, 0};
#pragma unroll
  for (int w = 0; w < 2; ++w)
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 x = v[w][u][h];
        nz[w] |= (x.x != 0.f) | (x.y != 0.f) | (x.z != 0.f) | (x.w != 0.f);
        mx[w] = fmaxf(mx[w], fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
      }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      mx[w] = fmaxf(mx[w], __shfl_xor_sync(0xffffffffu, mx[w], o));
      nz[w] |= __shfl_xor_sync(0xffffffffu, nz[w], o);
    }
  if (lane == 0)
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      red_m[w][warp] = mx[w];
      red_z[w][warp] = nz[w];
    }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
      for (int j = 1; j < 8; ++j) {
        mx[w] = fmaxf(mx[w], red_m[w][j]);
        nz[w] |= red_z[w][j];
      }
    const int keep = nz[0] && nz[1];
    a.prod[t] = keep ? mx[0] * mx[1] : 0.0f;
    if (keep) atomicOr(a.bits + (t >> 5), 1u << (t & 31));
    // arrive (release: the product and the mask bit are visible to whoever
    // sees the count), then split while the barrier completes
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.barrier) : "memory");
  }
  uint4 pcs[2][2][3];
#pragma unroll
  for (int w = 0; w < 2; ++w)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      uint2 lo[3], hi[3];
      split3_bf16x4(v[w][u][0], lo);
      split3_bf16x4(v[w][u][1], hi);
#pragma unroll
      for (int p = 0; p < 3; ++p) pcs[w][u][p] = make_uint4(lo[p].x, lo[p].y, hi[p].x, hi[p].y);
    }
  // grid barrier, bounded: a timeout sets the status word and ends the block
  if (tid == 0) {
    const uint64_t t0 = gtimer();
    int ok = 1;
    while (ld_acquire(a.barrier) < gridDim.x) {
      if (gtimer() - t0 > 2000000000ull) {   // 2 s
        ok = 0;
        atomicExch(a.status, (int)DEV_TIMEOUT);
        break;
      }
      __nanosleep(20);
    }
    pass = ok;
    a.nz[0][r0] = nz[0];   // the row statistics for later launches, off the path to the barrier
    a.rmax[0][r0] = mx[0];
    a.nz[1][r1] = nz[1];
    a.rmax[1][r1] = mx[1];
  }
  __syncthreads();
  if (!pass) return;
  // the mask and the products, through L2 (written by other blocks)
  const int nw = (a.kmax + 31) >> 5;
  float sacc = 0.0f;
  for (int j = tid; j < a.kmax; j += 256) sacc += __ldcg(a.prod + j);
  if (tid < nw) wsm[tid] = __ldcg(a.bits + tid);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
  if (lane == 0) red_s[warp] = sacc;
  __syncthreads();
  if (warp == 0) {
    // exclusive scan of the word counts, 4 words per lane
    int c[4], tot = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = lane * 4 + u;
      c[u] = i < nw ? __popc(wsm[i]) : 0;
      tot += c[u];
    }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int run = incl - tot;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = lane * 4 + u;
      if (i < nw) pre_s[i] = run;
      run += c[u];
    }
    const int kc = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) {
      float Sf = 0.0f;
      for (int j = 0; j < 8; ++j) Sf += red_s[j];
      // FP32 accumulation error is far below 1e-4 relative: inflate so S stays an upper bound
      const double S = (double)Sf * a.scale * (1.0 + 1e-4);
      // BF16 x3 drops terms of at most ~3 * 2^-18 |a||b| per product
      const int ns = a.nseg_fixed ? a.nseg_fixed : (3.0 * 3.814697265625e-06 * S <= a.split_tol ? 3 : 6);
      nseg_s = ns;
      kend_s = (kc + KS - 1) / KS * KS;
      if (t == 0) {
        *a.kcount = kc;
        *a.nseg = ns;
        *a.bound = S;
        if (a.sum_zero) *a.sum_zero = 0.0;
      }
    }
  }
  __syncthreads();
  const int npieces = nseg_s == 3 ? 2 : 3;
  const int kend = kend_s;   // the contraction reads rows 0 .. kend - 1
  const unsigned wbits = wsm[t >> 5];
  const int keep = (wbits >> (t & 31)) & 1;
  const int prefix = pre_s[t >> 5] + __popc(wbits & ((1u << (t & 31)) - 1u));
  const int64_t slot = keep ? prefix : a.kmax - 1 - (t - prefix);
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    __nv_bfloat16* o = a.out[w];
    const int64_t cols = a.cols[w];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = tid + 256 * u;
      if (2 * j < nv[w]) {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          if (p < npieces) {
            if (slot < kend)   // a kept row, or a zero row the last stage reads
              *reinterpret_cast<uint4*>(o + ((int64_t)p * a.Kp + slot) * cols + 8 * j) =
                  keep ? pcs[w][u][p] : make_uint4(0u, 0u, 0u, 0u);
            // zero rows past kmax that the last stage reads
            for (int64_t rr = (int64_t)a.kmax + t; rr < kend; rr += a.kmax)
              *reinterpret_cast<uint4*>(o + ((int64_t)p * a.Kp + rr) * cols + 8 * j) = make_uint4(0u, 0u, 0u, 0u);
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false on timeout (about 2 s of SM clock) or when another role
// has aborted; the clock and the abort flag are looked at every 1024 polls so
// the poll loop itself stays short
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 1023) == 0) {
      if (*abort_flag) return false;
      if (clock64() - t0 > WAIT_CYCLES) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// shared-memory matrix descriptor: MN-major, 128-byte swizzle.  The operand
// tile is 64-element (128-byte) chunks along M (or N), each chunk 32 k rows
// of 128 bytes (4096 bytes); the leading byte offset is the distance between
// chunks along M / N, the stride byte offset between groups of 8 k rows
__device__ __forceinline__ uint64_t mn128_desc(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)(MN_CHUNK_BYTES >> 4) << 16;   // leading byte offset: next 64-element chunk along M / N
  d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset: next 8 k rows
  d |= (uint64_t)1 << 46;                       // descriptor version
  d |= (uint64_t)2 << 61;                       // SWIZZLE_128B
  return d;
}
// shared-memory matrix descriptor: K-major, 64-byte swizzle (rows of 32 bf16),
// 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t sw64_desc(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused by swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)4 << 61;                  // SWIZZLE_64B
  return d;
}
// instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both MN-major
// (bits 15 and 16: A and B transposed)
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}
// instruction descriptor: kind::tf32, TF32 x TF32 -> FP32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// the same load without the wait, and a wait that names the destination
// registers, so their uses cannot be scheduled before it
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// 32-byte streaming store of 8 consecutive FP32 values (the address must be
// 32-byte aligned)
__device__ __forceinline__ void st_cs_v8(float* p, const float* v) {
  asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}

__device__ __forceinline__ uint64_t deposit(const uint64_t* __restrict__ tab, int nbytes, uint64_t v) {
  uint64_t g = 0;
  for (int b = 0; b < nbytes; ++b) g += __ldg(tab + b * 256 + ((v >> (8 * b)) & 255));
  return g;
}

// (value, index) order of the fused top-32: larger value first, then lower index
__device__ __forceinline__ bool tk_before(float v1, int64_t i1, float v2, int64_t i2) {
  return v1 > v2 || (v1 == v2 && i1 < i2);
}
// insert into the warp's sorted list (lane j holds the j-th best)
__device__ __forceinline__ void tk_insert(float& lv, int64_t& li, float v, int64_t idx, int lane) {
  const unsigned ahead = __ballot_sync(0xffffffffu, tk_before(lv, li, v, idx));
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

struct TcArgs {
  int Kp;
  int M, N;                   // rows of one piece of A' / B' (the piece offset of the TMA row coordinate)
  const int32_t* kcount;
  const int32_t* nseg;
  int tilesM, tilesN;
  const uint64_t* depA;
  const uint64_t* depB;
  int nbA, nbB;
  float* out;
  float scale;
  double* sum;
  int vecB;                   // consecutive columns that land on consecutive outputs: 1, 2, 4 or 8
  int staged;                 // restage the epilogue through shared memory (large outputs)
  int* status;
  float* topk_v;              // fused top-32 (dynamic-definition bins): one list of 32 per epilogue warp
  int64_t* topk_i;
};

// One work item of a CTA: rows tm*128 .. +127 and columns tn*256 + n0 ..
// + w - 1 of the output.  CTA b takes the full tiles b, b + G, b + 2G, ...
// (G CTAs) while whole rounds remain; when the last round has L < G tiles
// and 2L <= G, those tiles are cut into halves of 128 columns and CTA b < 2L
// takes half b % 2 of leftover tile b / 2, so no CTA owns a whole extra tile
// while others idle.  The producer, the MMA issuer and the epilogue walk the
// same list.
struct TcItem {
  int tm, tn, n0, w;
};
__device__ __forceinline__ bool tc_item(const TcArgs& a, int i, TcItem& it) {
  const int G = gridDim.x, b = blockIdx.x;
  const int ntiles = a.tilesM * a.tilesN;
  const int R = ntiles / G, L = ntiles - R * G;
  const int S = (L > 0 && 2 * L <= G) ? 2 : 1;
  int tile;
  it.n0 = 0;
  it.w = BN;
  if (i < R) {
    tile = b + i * G;
  } else if (i == R && b < L * S) {
    tile = R * G + b / S;
    if (S == 2) {
      it.w = BN / 2;
      it.n0 = (b & 1) * (BN / 2);
    }
  } else {
    return false;
  }
  it.tm = tile % a.tilesM;
  it.tn = tile / a.tilesM;
  return true;
}

// TK: also keep the fused top-32 (a separate instantiation, so the plain
// contraction carries none of its code).  tmBh: the B operand map with a
// 128-row box, for half-width items.
template <bool TK, bool TF32>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmBh, const TcArgs a) {
  // k per stage: 32 bf16 or 16 TF32 values, 64 bytes of every piece row
  constexpr int KSS = TF32 ? KS / 2 : KS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGE_AREA);   // 256 bytes of barriers
  uint64_t* empty = full + MAX_STAGES;
  uint64_t* tfull = empty + MAX_STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < MAX_STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  // everything above overlapped the operand preparation; what follows reads it
  CUTQC_PDL_WAIT();

  const int kc = *a.kcount;
  const int nseg = *a.nseg;
  const int npieces = (TF32 || nseg == 3) ? 2 : 3;          // h, m (x3) or h, m, l (x6); TF32: hi, lo
  const int stages = (TF32 || nseg == 3) ? 4 : 3;
  const uint32_t stage_bytes = (uint32_t)npieces * (A_PIECE + B_PIECE);
  const int nkb = (kc + KSS - 1) / KSS;                     // k steps of one stage

  if (nkb > 0 && warp == 0) {
    // ---- TMA producer (the warp waits, lane 0 issues): every split piece of
    // a 32-wide k step of A (128 rows) and B (the item's 256 or 128 rows)
    // into one stage (a half-width B piece fills the first half of its slot)
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    TcItem it;
    for (int i = 0; ok && tc_item(a, i, it); ++i) {
      const uint32_t item_bytes = (uint32_t)npieces * (uint32_t)(A_PIECE + it.w * 64);   // 64-byte piece rows
      const CUtensorMap* mapB = it.w == BN ? &tmB : &tmBh;
      for (int kb = 0; kb < nkb; ++kb) {
        ok = __all_sync(0xffffffffu, mbar_wait(&empty[stage], phase ^ 1, abort_flag));
        if (!ok) break;
        if (lane == 0) {
          uint8_t* st = smem + stage * stage_bytes;
          mbar_expect_tx(&full[stage], item_bytes);
          for (int pc = 0; pc < npieces; ++pc) {
            if constexpr (TF32) {
              tma_load_2d(st + pc * A_PIECE, &tmA, kb * KSS, pc * a.M + it.tm * BM, &full[stage]);
              tma_load_2d(st + npieces * A_PIECE + pc * B_PIECE, mapB, kb * KSS, pc * a.N + it.tn * BN + it.n0,
                          &full[stage]);
            } else {
              // k rows pc * Kp + kb * 32 .. + 31, 64-element chunks of M / N
              tma_load_3d(st + pc * A_PIECE, &tmA, 0, pc * a.Kp + kb * KSS, it.tm * (BM / MN_CHUNK), &full[stage]);
              tma_load_3d(st + npieces * A_PIECE + pc * B_PIECE, mapB, 0, pc * a.Kp + kb * KSS,
                          (it.tn * BN + it.n0) / MN_CHUNK, &full[stage]);
            }
          }
        }
        __syncwarp();
        if (++stage == stages) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  } else if (nkb > 0 && warp == 1) {
    // ---- MMA issuer (the warp waits, lane 0 issues): per stage the nseg
    // products hh, hm, mh (, hl, lh, mm), two K=16 MMAs each
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    TcItem it;
    for (int i = 0; ok && tc_item(a, i, it); ++i) {
      const uint32_t idesc = TF32 ? idesc_tf32(BM, it.w) : idesc_bf16_mn(BM, it.w);
      ok = __all_sync(0xffffffffu, mbar_wait(&tempty[acc], acc_phase ^ 1, abort_flag));
      if (!ok) break;
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + acc * BN;
      for (int kb = 0; kb < nkb; ++kb) {
        ok = __all_sync(0xffffffffu, mbar_wait(&full[stage], phase, abort_flag));
        if (!ok) break;
        tc_fence_after();
        if (lane == 0) {
          uint8_t* st = smem + stage * stage_bytes;
          for (int sg = 0; sg < nseg; ++sg) {
            // two MMAs per product and stage: K = 8 TF32 (K-major, 32 bytes
            // further along the row) or K = 16 bf16 (MN-major, 16 rows of 128
            // bytes further)
            if constexpr (TF32) {
              const uint64_t ad = sw64_desc(st + kPartA[sg] * A_PIECE);
              const uint64_t bd = sw64_desc(st + npieces * A_PIECE + kPartB[sg] * B_PIECE);
#pragma unroll
              for (int k = 0; k < 2; ++k) mma_tf32(d_tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | sg | k) != 0 ? 1u : 0u);
            } else {
              const uint64_t ad = mn128_desc(st + kPartA[sg] * A_PIECE);
              const uint64_t bd = mn128_desc(st + npieces * A_PIECE + kPartB[sg] * B_PIECE);
#pragma unroll
              for (int k = 0; k < 2; ++k)
                mma_bf16(d_tmem, ad + 128 * k, bd + 128 * k, idesc, (kb | sg | k) != 0 ? 1u : 0u);
            }
          }
          mma_commit(&empty[stage]);
        }
        __syncwarp();
        if (++stage == stages) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      if (lane == 0) mma_commit(&tfull[acc]);
      __syncwarp();
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  } else if (warp >= 2) {
    // ---- epilogue: warp w reads TMEM lanes 32 * (w % 4) .. +31 (lane = row),
    // columns 128 * hf .. +127 of the accumulator
    const int q = warp & 3;
    const int hf = (warp - 2) / 4;
    constexpr int CPW = BN / 32 / (EPI_WARPS / 4);   // 32-column chunks per warp
    static_assert(CPW % 4 == 0, "chunks go in pairs, also in half-width items");
    // this thread's share of the FP64 sum, accumulated in FP32 with TwoSum
    // (sum + compensation, about 48 bits; no FP64 instruction per chunk on
    // this part's narrow FP64 pipe)
    float lsum = 0.0f, lcomp = 0.0f;
    // the deposit is additive over disjoint index bits, so a row's output
    // address is dep(row base) + dep(lane) + dep(chunk column base) +
    // dep(column within the chunk); the per-thread parts live in registers
    const uint64_t dep_lane = deposit(a.depA, 1, (uint64_t)lane);
    uint64_t dlow[8], dcol[8], dtiny[4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      dlow[j] = deposit(a.depB, 1, (uint64_t)(4 * j));    // n bits 2-4
      dcol[j] = deposit(a.depB, 1, (uint64_t)(32 * j));   // n bits 5-7: chunk column base
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) dtiny[t] = deposit(a.depB, 1, (uint64_t)t);
    const bool vec = a.vecB >= 4;
    const bool staged = vec && a.staged;
    // 8 consecutive columns are 8 consecutive outputs (32 bytes, one sector);
    // with the next output bits on the rows, the 8 lanes of a row group then
    // write whole lines
    const bool vec8 = a.vecB >= 8;
    // fused top-32 of the written values, ranked by (value, output index)
    constexpr bool tk = TK;
    float tk_v = -FLT_MAX;
    int64_t tk_i = INT64_MAX;
    // Staged stores (outputs larger than L2, where the store stream is
    // DRAM-bound, and outputs in host memory; an output that stays in L2 goes
    // out directly from the registers, 16 bytes per row, which costs less
    // latency): a warp's 32-column chunk goes out in two passes of
    // 16 rows.  The 512 values of a pass are written to shared memory by row
    // and read back in output-address order: the 9 index bits (row bits 0-3,
    // column bits 0-4) are ranked by the output bit they deposit to, and lane
    // l of store step s takes ranks 128 s + 4 l .. + 3.  Column bits 0 and 1
    // deposit to output bits 0 and 1 (vec), so those 4 ranks are 4
    // consecutive columns and 4 consecutive outputs: one 16-byte store, and a
    // warp instruction writes 128 values in address order (whole lines where
    // the layout allows) instead of 16 bytes in each of 32 rows.
    float* ebuf = reinterpret_cast<float*>(smem + STAGE_AREA + 256) + (warp - 2) * (EPI_BUF / 4);
    int so[4];            // shared-memory offset (row * EPI_LD + column) of step s
    uint64_t rel[4];      // output offset of step s relative to the pass base
    {
      int pos[9], rk[9];
#pragma unroll
      for (int b = 0; b < 4; ++b) pos[b] = __ffsll((long long)deposit(a.depA, 1, 1ull << b)) - 1;
#pragma unroll
      for (int b = 0; b < 5; ++b) pos[4 + b] = __ffsll((long long)deposit(a.depB, 1, 1ull << b)) - 1;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        rk[i] = 0;
#pragma unroll
        for (int j = 0; j < 9; ++j) rk[i] += pos[j] < pos[i] ? 1 : 0;
      }
#pragma unroll
      for (int st = 0; st < 4; ++st) {
        const int r = 128 * st + 4 * lane;
        int mm = 0, nn = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) mm |= ((r >> rk[b]) & 1) << b;
#pragma unroll
        for (int b = 0; b < 5; ++b) nn |= ((r >> rk[4 + b]) & 1) << b;
        so[st] = mm * EPI_LD + nn;
        rel[st] = deposit(a.depA, 1, (uint64_t)mm) + deposit(a.depB, 1, (uint64_t)nn);
      }
    }
    const uint64_t dpass1 = deposit(a.depA, 1, 16ull);   // row bit 4: second pass
    int acc = 0;
    uint32_t acc_phase = 0;
    // this thread's row of item it: tm*128 + 32q + lane; columns tn*256 + n0 +
    // 32c + j.  The item's output base comes from the deposit tables in
    // global memory (dependent round trips to L2), so the next item's is
    // loaded while this one drains.
    auto item_base = [&](const TcItem& t) {
      return deposit(a.depA, a.nbA, (uint64_t)t.tm * BM + 32 * q) + deposit(a.depB, a.nbB, (uint64_t)t.tn * BN + t.n0);
    };
    TcItem it, itn;
    bool have = tc_item(a, 0, it);
    uint64_t gnext = have ? item_base(it) : 0;
    for (int i = 0; have; ++i, it = itn) {
      const uint64_t gbase = gnext;
      have = tc_item(a, i + 1, itn);
      if (have) gnext = item_base(itn);
      if (nkb > 0) {
        const bool ok = mbar_wait(&tfull[acc], acc_phase, abort_flag);
        if (!__all_sync(0xffffffffu, ok)) break;
        tc_fence_after();
      }
      // the TMEM load of the next 32-column chunk is in flight while this one
      // is processed (two register buffers)
      auto taddr = [&](int c) {
        return tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + 32 * c);
      };
      auto process = [&](const int c, uint32_t (&r)[32]) {
        // sum of this 32-column row piece: pairwise in FP32 (error <= 5 * 2^-24 *
        // sum |v|), then one compensated FP32 add into the thread's share
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) * a.scale;
        float t16[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) t16[j] = v[2 * j] + v[2 * j + 1];
#pragma unroll
        for (int w = 8; w > 0; w >>= 1)
#pragma unroll
          for (int j = 0; j < w; ++j) t16[j] += t16[j + w];
        {
          const float t = lsum + t16[0];
          const float bb = t - lsum;
          lcomp += (lsum - (t - bb)) + (t16[0] - bb);
          lsum = t;
        }
        uint64_t dc = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) dc = (k == c) ? dcol[k] : dc;
        if constexpr (TK) {
          // the warp's current 32nd best; a chunk with no value at or above it
          // (the usual case once the list has filled) costs one vote
          float thr_v = __shfl_sync(0xffffffffu, tk_v, 31);
          bool cand = false;
#pragma unroll
          for (int j = 0; j < 32; ++j) cand |= v[j] >= thr_v;
          if (__any_sync(0xffffffffu, cand)) {
            const uint64_t rowg = gbase + dep_lane + dc;
            int64_t thr_i = __shfl_sync(0xffffffffu, tk_i, 31);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int64_t idx = (int64_t)(rowg + dlow[j >> 2] + dtiny[j & 3]);
              unsigned m = __ballot_sync(0xffffffffu, tk_before(v[j], idx, thr_v, thr_i));
              if (m) {
                while (m) {
                  const int src = __ffs(m) - 1;
                  m &= m - 1;
                  tk_insert(tk_v, tk_i, __shfl_sync(0xffffffffu, v[j], src), __shfl_sync(0xffffffffu, idx, src),
                            lane);
                }
                thr_v = __shfl_sync(0xffffffffu, tk_v, 31);
                thr_i = __shfl_sync(0xffffffffu, tk_i, 31);
              }
            }
          }
        }
        if (staged) {
          float* cbase = a.out + gbase + dc;
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            if ((lane >> 4) == p) {
              float4* dst = reinterpret_cast<float4*>(ebuf + (lane & 15) * EPI_LD);
#pragma unroll
              for (int j = 0; j < 8; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
            __syncwarp();
            float* pbase = cbase + (p ? dpass1 : 0);
#pragma unroll
            for (int st = 0; st < 4; ++st)
              __stcs(reinterpret_cast<float4*>(pbase + rel[st]), *reinterpret_cast<const float4*>(ebuf + so[st]));
            __syncwarp();
          }
        } else if (vec8) {
          float* orow = a.out + gbase + dep_lane + dc;
#pragma unroll
          for (int j = 0; j < 4; ++j) st_cs_v8(orow + dlow[2 * j], v + 8 * j);
        } else if (vec) {
          float* orow = a.out + gbase + dep_lane + dc;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            __stcs(reinterpret_cast<float4*>(orow + dlow[j]), make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
        } else {
          float* orow = a.out + gbase + dep_lane + dc;
#pragma unroll
          for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int t = 0; t < 4; ++t) orow[dlow[j] + dtiny[t]] = v[4 * j + t];
        }
      };
      uint32_t ra[32], rb[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) ra[j] = rb[j] = 0u;
      // chunks of this warp in the item: CPW, or half as many for a half-width item
      const int cpw = it.w == BN ? CPW : CPW / 2;
      const int c0 = hf * cpw;
      if (nkb > 0) tmem_ld32_issue(taddr(c0), ra);
#pragma unroll 1
      for (int c = c0; c < c0 + cpw; c += 2) {
        if (nkb > 0) {
          tmem_wait32(ra);
          tmem_ld32_issue(taddr(c + 1), rb);
        }
        process(c, ra);
        if (nkb > 0) {
          tmem_wait32(rb);
          if (c + 2 < c0 + cpw) tmem_ld32_issue(taddr(c + 2), ra);
        }
        process(c + 1, rb);
      }
      if (nkb > 0) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
    }
    if (a.sum) {
#pragma unroll
      double local = (double)lsum + (double)lcomp;
      for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
      if (lane == 0) atomicAdd(a.sum, local);
    }
    if constexpr (TK) {
      const int64_t list = (int64_t)blockIdx.x * EPI_WARPS + (warp - 2);
      a.topk_v[list * 32 + lane] = tk_v;
      a.topk_i[list * 32 + lane] = tk_i;
    }
  }
  __syncwarp();
  if (*abort_flag) {
    // let copies and MMAs already in flight land before TMEM and smem go away
    if (threadIdx.x == 0) {
      atomicExch(a.status, (int)DEV_TIMEOUT);
      const uint64_t t0 = gtimer();
      while (gtimer() - t0 < 2000000ull) __nanosleep(1000);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------ wait self-test
__global__ void k_wait_selftest(int* status, long long limit_ns) {
  __shared__ unsigned flag;
  flag = 0u;
  __syncwarp();
  const uint64_t t0 = gtimer();
  while (*reinterpret_cast<volatile unsigned*>(&flag) == 0u) {
    if ((long long)(gtimer() - t0) > limit_ns) {
      atomicExch(status, (int)DEV_TIMEOUT);
      return;
    }
    __nanosleep(1000);
  }
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (!fn) fail(CUTQC_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  return fn;
}

// rows of 64 bytes per box: 32 bf16 or 16 FP32 (TF32) elements
CUtensorMap make_map(const void* base, uint64_t rows, uint64_t inner, uint32_t box_rows, bool tf32) {
  CUtensorMap m;
  const uint64_t es = tf32 ? 4 : 2;
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {inner * es};
  const cuuint32_t box[2] = {(cuuint32_t)(64 / es), box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                           const_cast<void*>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(CUTQC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

// BF16 pieces, MN-major: [rows = pieces * Kp][cols] viewed as (64 elements
// of a chunk, k row, chunk of 64 along cols), box 64 x 32 k rows x `chunks`:
// in shared memory the chunks lie 4096 bytes apart, 128-byte rows within each
CUtensorMap make_map_mn(const void* base, uint64_t rows, uint64_t cols, uint32_t chunks) {
  CUtensorMap m;
  const cuuint64_t dims[3] = {MN_CHUNK, rows, cols / MN_CHUNK};
  const cuuint64_t strides[2] = {cols * 2, MN_CHUNK * 2};
  const cuuint32_t box[3] = {MN_CHUNK, (cuuint32_t)KS, chunks};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(CUTQC_ERR_CUDA, "cuTensorMapEncodeTiled failed (MN-major operand map)");
  return m;
}

int kpad(const Contraction& c) { return (c.kmax + BK - 1) / BK * BK; }

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

void launch_wait_selftest(int* status, int limit_us, cudaStream_t s) {
  k_wait_selftest<<<1, 1, 0, s>>>(status, (long long)limit_us * 1000);
  count_launch();
  check_launch("k_wait_selftest");
}

bool tc_supported(const Contraction& c) {
  return c.dtype == CUTQC_F32 && c.batch == 1 && c.fA >= 7 && c.fB >= 8 && c.kmax >= 1;
}

size_t tc_workspace_bytes(const Contraction& c) {
  const size_t Kp = kpad(c);
  const size_t M = size_t(1) << c.fA, N = size_t(1) << c.fB;
  // per (row, k): 3 bf16 pieces (6 bytes) or 2 TF32 pieces in FP32 containers (8 bytes)
  return align256(M * Kp * 8) + align256(N * Kp * 8) + 256;
}

void launch_tc_bf16x3(const Contraction& c, void* ws, size_t ws_bytes, cudaStream_t s, const TcFusedStats* fused) {
  if (!tc_supported(c)) fail(CUTQC_ERR_UNSUPPORTED, "shape not supported by the tensor-core path");
  if (ws_bytes < tc_workspace_bytes(c)) fail(CUTQC_ERR_OOM, "tensor-core workspace too small");
  const int Kp = kpad(c);
  const int64_t M = int64_t(1) << c.fA, N = int64_t(1) << c.fB;
  const bool tf32 = c.tf32;
  char* w = static_cast<char*>(ws);
  void* Ab = w;
  void* Bb = w + align256((size_t)M * Kp * 8);
  int* status = c.status;
  if (!status) fail(CUTQC_ERR_ARG, "tensor-core path needs the device status word");
  if (!c.nseg || !c.bound) fail(CUTQC_ERR_ARG, "tensor-core path needs the split count");
  PrepArgs pa{};
  pa.T[0] = static_cast<const float*>(c.A);
  pa.T[1] = static_cast<const float*>(c.B);
  pa.cols[0] = M;
  pa.cols[1] = N;
  pa.blocks0 = (int)(M / 64);
  pa.Kp = Kp;
  pa.kmax = c.kmax;
  pa.fused = !c.compacted && c.kmax <= 4096;
  pa.rows = c.rows;
  pa.crow = c.crow;
  pa.nzA = c.nzA;
  pa.nzB = c.nzB;
  pa.rmaxA = c.rmaxA;
  pa.rmaxB = c.rmaxB;
  pa.scale = c.scale;
  pa.split_tol = c.split_tol;
  pa.nseg_fixed = tf32 ? 3 : c.nseg_fixed;
  pa.kcount = c.kcount;
  pa.nseg = c.nseg;
  pa.bound = c.bound;
  pa.sum_zero = c.sum;
  pa.out[0] = Ab;
  pa.out[1] = Bb;
  static int pair_blocks = -1;   // resident blocks of the one-pass preparation on the device
  if (pair_blocks < 0) {
    int dev = 0, sms = 0, per_sm = 0;
    CUTQC_CUDA(cudaGetDevice(&dev));
    CUTQC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUTQC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_prep, 256, 0));
    pair_blocks = per_sm * sms;
  }
  if (fused && !tf32 && c.kmax >= PAIR_PREP_MIN_TERMS && c.kmax <= pair_blocks && M <= 4096 && N <= 4096) {
    if (c.kmax > 4096) fail(CUTQC_ERR_UNSUPPORTED, "fused row statistics need kmax <= 4096");
    if (!fused->look) fail(CUTQC_ERR_ARG, "the preparation needs its barrier and mask words");
    PairArgs pr{};
    pr.T[0] = pa.T[0];
    pr.T[1] = pa.T[1];
    pr.cols[0] = M;
    pr.cols[1] = N;
    pr.kmax = c.kmax;
    pr.Kp = Kp;
    pr.rows = c.rows;
    pr.nz[0] = fused->nzA;
    pr.nz[1] = fused->nzB;
    pr.rmax[0] = fused->rmaxA;
    pr.rmax[1] = fused->rmaxB;
    const int nw = (c.kmax + 31) / 32;
    pr.barrier = fused->look;
    pr.bits = fused->look + 1;
    pr.prod = reinterpret_cast<float*>(fused->look + 1 + nw);
    pr.scale = c.scale;
    pr.split_tol = c.split_tol;
    pr.nseg_fixed = pa.nseg_fixed;
    pr.kcount = c.kcount;
    pr.nseg = c.nseg;
    pr.bound = c.bound;
    pr.sum_zero = c.sum;
    pr.status = status;
    pr.out[0] = static_cast<__nv_bfloat16*>(Ab);
    pr.out[1] = static_cast<__nv_bfloat16*>(Bb);
    const unsigned grid = (unsigned)c.kmax;   // one block per term
    CUTQC_CUDA(cudaMemsetAsync(fused->look, 0, sizeof(unsigned) * (size_t)(1 + nw), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every block resident: the grid barrier cannot starve
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUTQC_CUDA(cudaLaunchKernelEx(&cfg, k_pair_prep, pr));
    count_launch();
    check_launch("k_pair_prep");
  } else if (fused) {
    if (c.kmax > 4096) fail(CUTQC_ERR_UNSUPPORTED, "fused row statistics need kmax <= 4096");
    pa.fused = 1;
    pa.nzA = fused->nzA;
    pa.nzB = fused->nzB;
    pa.rmaxA = fused->rmaxA;
    pa.rmaxB = fused->rmaxB;
    StatsArgs sa{};
    sa.rows[0] = c.rowsA;
    sa.rows[1] = c.rowsB;
    sa.nz[0] = fused->nzA;
    sa.nz[1] = fused->nzB;
    sa.rmax[0] = fused->rmaxA;
    sa.rmax[1] = fused->rmaxB;
    sa.barrier = fused->barrier;
    sa.status = status;
    sa.tilesX = (int)((M + N) / 64);
    sa.tilesY = Kp / 64;
    static int coop_blocks[2] = {0, 0};   // resident blocks per SM (bf16, TF32 instantiation)
    static int coop_sms = 0;
    if (!coop_blocks[tf32]) {
      int dev = 0;
      CUTQC_CUDA(cudaGetDevice(&dev));
      CUTQC_CUDA(cudaDeviceGetAttribute(&coop_sms, cudaDevAttrMultiProcessorCount, dev));
      CUTQC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &coop_blocks[tf32], tf32 ? k_stats_prep<true> : k_stats_prep<false>, 256, 0));
      if (coop_blocks[tf32] < 1) fail(CUTQC_ERR_CUDA, "operand preparation cannot be resident");
    }
    const int64_t want = std::max<int64_t>(sa.rows[0] + sa.rows[1], (int64_t)sa.tilesX * sa.tilesY);
    const unsigned grid = (unsigned)std::min<int64_t>(want, (int64_t)coop_blocks[tf32] * coop_sms);
    CUTQC_CUDA(cudaMemsetAsync(fused->barrier, 0, sizeof(unsigned), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every block resident: the grid barrier cannot starve
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (tf32)
      CUTQC_CUDA(cudaLaunchKernelEx(&cfg, k_stats_prep<true>, pa, sa));
    else
      CUTQC_CUDA(cudaLaunchKernelEx(&cfg, k_stats_prep<false>, pa, sa));
    count_launch();
    check_launch("k_stats_prep");
  } else {
    if (!pa.fused && !c.compacted) {
      Contraction cc = c;
      cc.sum_zero = c.sum;
      launch_compact(cc, s);
    }
    const dim3 pg((unsigned)((M + N) / 64), (unsigned)(Kp / 64));
    if (tf32)
      CUTQC_CUDA(launch_pdl(k_prep<true>, pg, dim3(256), 0, s, pa));
    else
      CUTQC_CUDA(launch_pdl(k_prep<false>, pg, dim3(256), 0, s, pa));
    count_launch();
    check_launch("k_prep");
  }

  // TF32: the pieces of each operand stacked along rows, [piece * rows +
  // row][k]; BF16: [piece * Kp + k][row] (MN-major)
  const CUtensorMap tmA = tf32 ? make_map(Ab, (uint64_t)M * 2, (uint64_t)Kp, BM, true)
                               : make_map_mn(Ab, (uint64_t)Kp * 3, (uint64_t)M, BM / MN_CHUNK);
  const CUtensorMap tmB = tf32 ? make_map(Bb, (uint64_t)N * 2, (uint64_t)Kp, BN, true)
                               : make_map_mn(Bb, (uint64_t)Kp * 3, (uint64_t)N, BN / MN_CHUNK);
  const CUtensorMap tmBh = tf32 ? make_map(Bb, (uint64_t)N * 2, (uint64_t)Kp, BN / 2, true)
                                : make_map_mn(Bb, (uint64_t)Kp * 3, (uint64_t)N, BN / 2 / MN_CHUNK);
  TcArgs a;
  a.Kp = Kp;
  a.M = (int)M;
  a.N = (int)N;
  a.kcount = c.kcount;
  a.nseg = c.nseg;
  a.tilesM = (int)(M / BM);
  a.tilesN = (int)(N / BN);
  a.depA = c.depA;
  a.depB = c.depB;
  a.nbA = (c.fA + 7) / 8;
  a.nbB = (c.fB + 7) / 8;
  a.out = static_cast<float*>(c.out);
  a.scale = (float)c.scale;
  a.sum = c.sum;
  // 32-byte stores need a 32-byte aligned output (16 bytes is the minimum the
  // entry points accept)
  a.vecB = (c.vecB >= 8 && reinterpret_cast<uintptr_t>(c.out) % 32 != 0) ? 4 : c.vecB;
  // restage through shared memory for outputs beyond L2 (128 MiB of FP32) and
  // for outputs in host memory, where whole-line stores matter most
  a.staged = (c.out_host || M * N >= (int64_t(1) << 25)) ? 1 : 0;
  a.topk_v = c.topk_v;
  a.topk_i = c.topk_i;
  a.status = status;
  static int sms = 0;
  static bool attr = false;
  if (!attr) {
    CUTQC_CUDA(cudaFuncSetAttribute(k_tc_gemm<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SMEM_BYTES));
    CUTQC_CUDA(cudaFuncSetAttribute(k_tc_gemm<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SMEM_BYTES));
    CUTQC_CUDA(cudaFuncSetAttribute(k_tc_gemm<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SMEM_BYTES));
    CUTQC_CUDA(cudaFuncSetAttribute(k_tc_gemm<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SMEM_BYTES));
    int dev = 0;
    CUTQC_CUDA(cudaGetDevice(&dev));
    CUTQC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    attr = true;
  }
  const int tiles = a.tilesM * a.tilesN;
  const int grid = tiles < sms ? tiles : sms;
  cudaEvent_t ev = nullptr;
  if (c.profile) prof_begin(s, &ev);
  auto* kern = a.topk_v ? (tf32 ? k_tc_gemm<true, true> : k_tc_gemm<true, false>)
                        : (tf32 ? k_tc_gemm<false, true> : k_tc_gemm<false, false>);
  CUTQC_CUDA(launch_pdl(kern, dim3(grid), dim3(THREADS), SMEM_BYTES, s, tmA, tmB, tmBh, a));
  count_launch();
  check_launch("k_tc_gemm");
  if (c.topk_nlists) *c.topk_nlists = c.topk_v ? grid * EPI_WARPS : 0;
  if (c.profile) prof_end(s, ev);
}

}  // namespace cutqc

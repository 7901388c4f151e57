// tcgen05 split-precision reconstruction (BF16 x3 / x6, FP32 accumulation in TMEM).
//
// The final contraction of the 4^K sum (Sec. 3.3), P[m][n] = 2^-K sum_e
// A[e][m] B[e][n], runs on the 5th-generation tensor cores.  Each FP32
// operand x is split into x_hi = bf16(x) and x_lo = bf16(x - x_hi), and
//   A.B ~= A_hi.B_hi + A_hi.B_lo + A_lo.B_hi
// (the lo.lo term is ~2^-16 relative).  The three products are one GEMM over a
// concatenated inner dimension: A' = [A_hi | A_hi | A_lo] and
// B' = [B_hi | B_lo | B_hi], both stored K-major in bf16.  The x6 form splits
// into three pieces and appends hl, lh and mm segments (FP32-level accuracy);
// the number of segments is read on the device (chosen by the compaction
// kernel from an a-priori bound) so no host round trip is needed.
//
// k_prep_split (operand preparation): gathers the compacted rows (terms whose
// factor rows are all zero were dropped: early termination, Sec. 4.2),
// transposes them to K-major through shared memory and writes the splits.
//
// k_tc_gemm: persistent, one CTA per SM, 192 threads:
//   warp 0     TMA producer: 128x64 A tiles and 256x64 B tiles (128-byte
//              swizzle) into a 4-stage shared-memory ring;
//   warp 1     allocates 512 TMEM columns (two 128x256 FP32 accumulators)
//              and one thread issues tcgen05.mma (M=128, N=256, K=16);
//   warps 2-5  epilogue: tcgen05.ld of their 32 TMEM lanes, scale by 2^-K,
//              deposit (m, n) into the output index, 16-byte stores, FP64
//              partial sums; it drains one accumulator while the MMA fills
//              the other.
// Every wait on an mbarrier is bounded (2 s); on timeout the kernel raises an
// abort flag, records a status word, lets in-flight copies land and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace cutqc {

namespace {

constexpr int BM = 128, BN = 256, BK = 64;   // BK bf16 = 128 bytes = one swizzle row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;          // 16 KiB
constexpr int B_BYTES = BN * BK * 2;          // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 512;
constexpr int THREADS = 192;
constexpr int EPI_PITCH = 33;                 // padded row pitch of the epilogue staging buffer
constexpr int EPI_WARP_BYTES = 32 * EPI_PITCH * 4;
constexpr size_t SMEM_BYTES = size_t(STAGES) * STAGE_BYTES + 4 * EPI_WARP_BYTES + 1024 + 256;

// Epilogue staging.  An epilogue warp holds a 32 x 32 chunk (lane = low 5 bits
// of m, register = low 5 bits of n).  Those 10 index bits land on 10 output
// bit positions; ordering them by position gives each chunk element a "slot"
// whose order is the output address order.  The warp writes the chunk to
// shared memory row by row ([lane][col], pitch 33: conflict-free), then reads
// it back slot by slot and stores to global memory in address order: runs of
// 2^contig consecutive floats become coalesced 16-byte stores.  All maps are
// additive over disjoint bits, so each is a sum of a low and a high table.
struct EpiTab {
  int32_t slo[32], shi[32];      // staging offset (floats) of slot bits 0-4 / 5-9
  uint64_t glo[32], ghi[32];     // output offset of slot bits 0-4 / 5-9
  int32_t contig;                // slots 0..2^contig-1 are consecutive in memory
  int32_t pad[3];
};
constexpr uint64_t WAIT_NS = 2000000000ull;

// ------------------------------------------------------------ operand prep
// Each FP32 x is split into h = bf16(x), m = bf16(x - h), l = bf16(x - h - m).
// Segment s of the concatenated inner dimension pairs part PA[s] of A with
// part PB[s] of B (0 = h, 1 = m, 2 = l): hh, hm, mh | hl, lh, mm.  The first
// three segments are the x3 form, all six the x6 form.
__constant__ int kPartA[6] = {0, 0, 1, 0, 2, 1};
__constant__ int kPartB[6] = {0, 1, 0, 2, 0, 1};

// out[m][seg * Kp + k] = part(T[rowsel[k]][m]) for k < kcount (0 for
// kcount <= k < Kp), for the first *nseg segments; row pitch 6 * Kp.
__global__ void __launch_bounds__(256) k_prep_split(const float* __restrict__ T, int64_t cols,
                                                    const int32_t* __restrict__ rowsel,
                                                    const int32_t* __restrict__ kcount,
                                                    const int32_t* __restrict__ nseg_ptr, int Kp, int which,
                                                    __nv_bfloat16* __restrict__ out) {
  __shared__ float s[64][65];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.x * 64;
  const int k0 = blockIdx.y * 64;
  const int kc = *kcount;
  const int nseg = *nseg_ptr;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int kk = i * 4 + tid / 64, mm = tid % 64, k = k0 + kk;
    s[kk][mm] = (k < kc) ? T[(int64_t)rowsel[k] * cols + m0 + mm] : 0.0f;
  }
  __syncthreads();
  const int ml = tid / 4, kq = (tid % 4) * 16;
  __align__(16) __nv_bfloat16 part[3][16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float v = s[kq + j][ml];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(mid);
    part[0][j] = h;
    part[1][j] = mid;
    part[2][j] = __float2bfloat16_rn(r2);
  }
  const int64_t row = (m0 + ml) * (int64_t)(6 * Kp);
  for (int seg = 0; seg < nseg; ++seg) {
    const int pi = which == 0 ? kPartA[seg] : kPartB[seg];
    const uint4* src = reinterpret_cast<const uint4*>(part[pi]);
    uint4* dst = reinterpret_cast<uint4*>(out + row + (int64_t)seg * Kp + k0 + kq);
    dst[0] = src[0];
    dst[1] = src[1];
  }
}

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
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
// bounded wait: false on timeout or when another role has aborted
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > WAIT_NS) {
      *abort_flag = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused by swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // SWIZZLE_128B
  return d;
}
// instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
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

__device__ __forceinline__ uint64_t deposit(const uint64_t* __restrict__ tab, int nbytes, uint64_t v) {
  uint64_t g = 0;
  for (int b = 0; b < nbytes; ++b) g += __ldg(tab + b * 256 + ((v >> (8 * b)) & 255));
  return g;
}

struct TcArgs {
  int Kp;
  const int32_t* kcount;
  const int32_t* nseg;
  int tilesM, tilesN;
  const uint64_t* depA;
  const uint64_t* depB;
  int nbA, nbB;
  float* out;
  float scale;
  double* sum;
  int vecB;
  const void* epi;
  int* status;
};

__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);   // 256 bytes of barriers
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
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

  const int kc = *a.kcount;
  const int nkb = (kc + BK - 1) / BK;
  const int total_kb = *a.nseg * nkb;
  const int ntiles = a.tilesM * a.tilesN;

  if (nkb > 0 && warp == 0 && lane == 0) {
    // ---- TMA producer
    int stage = 0;
    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
      const int tm = tile % a.tilesM, tn = tile / a.tilesM;
      for (int kb = 0; kb < total_kb; ++kb) {
        const int seg = kb / nkb, kk = kb % nkb;
        const int x = seg * a.Kp + kk * BK;
        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) break;
        mbar_expect_tx(&full[stage], STAGE_BYTES);
        tma_load_2d(sA + stage * A_BYTES, &tmA, x, tm * BM, &full[stage]);
        tma_load_2d(sB + stage * B_BYTES, &tmB, x, tn * BN, &full[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  } else if (nkb > 0 && warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16(BM, BN);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      if (!mbar_wait(&tempty[acc], acc_phase ^ 1, abort_flag)) break;
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + acc * BN;
      for (int kb = 0; kb < total_kb; ++kb) {
        if (!mbar_wait(&full[stage], phase, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = sw128_desc(sA + stage * A_BYTES);
        const uint64_t bd = sw128_desc(sB + stage * B_BYTES);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          mma_bf16(d_tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
        mma_commit(&empty[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      mma_commit(&tfull[acc]);
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  } else if (warp >= 2) {
    // ---- epilogue: warp w reads TMEM lanes 32 * (w % 4) .. +31
    const int q = warp & 3;
    float* stage_buf = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256) + (warp - 2) * (32 * EPI_PITCH);
    const EpiTab* et = static_cast<const EpiTab*>(a.epi);
    double local = 0.0;
    // per-thread constants of the read-back: slots 4*lane + t (t < 4) of each
    // 128-slot pass it (< 8): staging offset slo[(4l+t)&31] + shi[4it + l/8]
    int32_t rs_lo[4];
    uint64_t rg_lo[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      rs_lo[t] = et->slo[(4 * lane + t) & 31];
      rg_lo[t] = et->glo[(4 * lane + t) & 31];
    }
    int32_t rs_hi[8];
    uint64_t rg_hi[8], dcol[8];
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      rs_hi[it] = et->shi[4 * it + (lane >> 3)];
      rg_hi[it] = et->ghi[4 * it + (lane >> 3)];
      dcol[it] = deposit(a.depB, 1, (uint64_t)(32 * it));   // chunk column base, n bits 5-7
    }
    const bool vec = et->contig >= 2;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int tm = tile % a.tilesM, tn = tile / a.tilesM;
      // chunk base: rows tm*128 + 32q (m bits >= 5), columns tn*256 (n bits >= 8)
      const uint64_t gT = deposit(a.depA, a.nbA, (uint64_t)tm * BM + 32 * q) +
                          deposit(a.depB, a.nbB, (uint64_t)tn * BN);
      if (nkb > 0) {
        const bool ok = mbar_wait(&tfull[acc], acc_phase, abort_flag);
        if (!__all_sync(0xffffffffu, ok)) break;
        tc_fence_after();
      }
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t r[32];
        if (nkb > 0) {
          tmem_ld32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + 32 * c), r);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = 0u;
        }
        // sum of this 32-column row piece: pairwise in FP32 (error <= 5 * 2^-24 *
        // sum |v|), then one FP64 add (the FP64 pipe is narrow on this part)
        float t16[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          t16[j] = __uint_as_float(r[2 * j]) * a.scale + __uint_as_float(r[2 * j + 1]) * a.scale;
#pragma unroll
        for (int w = 8; w > 0; w >>= 1)
#pragma unroll
          for (int j = 0; j < w; ++j) t16[j] += t16[j + w];
        local += (double)t16[0];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 32; ++j) stage_buf[lane * EPI_PITCH + j] = __uint_as_float(r[j]) * a.scale;
        __syncwarp();
        uint64_t dc = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) dc = (k == c) ? dcol[k] : dc;
        float* obase = a.out + gT + dc;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int32_t sh = rs_hi[it];
          const uint64_t gh = rg_hi[it];
          const float v0 = stage_buf[rs_lo[0] + sh], v1 = stage_buf[rs_lo[1] + sh];
          const float v2 = stage_buf[rs_lo[2] + sh], v3 = stage_buf[rs_lo[3] + sh];
          if (vec) {
            __stcs(reinterpret_cast<float4*>(obase + gh + rg_lo[0]), make_float4(v0, v1, v2, v3));
          } else {
            obase[gh + rg_lo[0]] = v0;
            obase[gh + rg_lo[1]] = v1;
            obase[gh + rg_lo[2]] = v2;
            obase[gh + rg_lo[3]] = v3;
          }
        }
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
      for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
      if (lane == 0) atomicAdd(a.sum, local);
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

CUtensorMap make_map(const void* base, uint64_t rows, uint64_t inner, uint32_t box_rows) {
  CUtensorMap m;
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(CUTQC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

int kpad(const Contraction& c) { return (c.kmax + BK - 1) / BK * BK; }

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

bool tc_supported(const Contraction& c) {
  return c.dtype == CUTQC_F32 && c.batch == 1 && c.fA >= 7 && c.fB >= 8 && c.kmax >= 1 && c.epi_tab;
}

std::vector<uint8_t> tc_epilogue_table(const std::vector<uint64_t>& va, const std::vector<uint64_t>& vb) {
  std::vector<uint8_t> bytes;
  if (va.size() < 5 || vb.size() < 5) return bytes;
  // the 10 chunk index bits: lane bits (m bits 0-4) and column bits (n bits 0-4)
  struct Bit {
    uint64_t value;
    int32_t stage;
  };
  std::vector<Bit> bits;
  for (int b = 0; b < 5; ++b) bits.push_back({va[b], (int32_t)(EPI_PITCH << b)});
  for (int b = 0; b < 5; ++b) bits.push_back({vb[b], (int32_t)(1 << b)});
  std::sort(bits.begin(), bits.end(), [](const Bit& x, const Bit& y) { return x.value < y.value; });
  EpiTab t{};
  for (int i = 0; i < 32; ++i) {
    for (int k = 0; k < 5; ++k) {
      if ((i >> k) & 1) {
        t.slo[i] += bits[k].stage;
        t.shi[i] += bits[5 + k].stage;
        t.glo[i] += bits[k].value;
        t.ghi[i] += bits[5 + k].value;
      }
    }
  }
  int j = 0;
  while (j < 10 && bits[j].value == (uint64_t(1) << j)) ++j;
  t.contig = j;
  bytes.resize(sizeof(EpiTab));
  std::memcpy(bytes.data(), &t, sizeof(EpiTab));
  return bytes;
}

size_t tc_workspace_bytes(const Contraction& c) {
  const size_t Kp = kpad(c);
  const size_t M = size_t(1) << c.fA, N = size_t(1) << c.fB;
  return align256(M * 6 * Kp * 2) + align256(N * 6 * Kp * 2) + 256;
}

void launch_tc_bf16x3(const Contraction& c, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (!tc_supported(c)) fail(CUTQC_ERR_UNSUPPORTED, "shape not supported by the tensor-core path");
  if (ws_bytes < tc_workspace_bytes(c)) fail(CUTQC_ERR_OOM, "tensor-core workspace too small");
  const int Kp = kpad(c);
  const int64_t M = int64_t(1) << c.fA, N = int64_t(1) << c.fB;
  char* w = static_cast<char*>(ws);
  auto* Ab = reinterpret_cast<__nv_bfloat16*>(w);
  auto* Bb = reinterpret_cast<__nv_bfloat16*>(w + align256((size_t)M * 6 * Kp * 2));
  int* status = reinterpret_cast<int*>(w + align256((size_t)M * 6 * Kp * 2) + align256((size_t)N * 6 * Kp * 2));
  if (!c.nseg) fail(CUTQC_ERR_ARG, "tensor-core path needs the split count");
  k_prep_split<<<dim3((unsigned)(M / 64), (unsigned)(Kp / 64)), 256, 0, s>>>(
      static_cast<const float*>(c.A), M, c.crow, c.kcount, c.nseg, Kp, 0, Ab);
  count_launch();
  check_launch("k_prep_split(A)");
  k_prep_split<<<dim3((unsigned)(N / 64), (unsigned)(Kp / 64)), 256, 0, s>>>(
      static_cast<const float*>(c.B), N, c.crow + c.kmax, c.kcount, c.nseg, Kp, 1, Bb);
  count_launch();
  check_launch("k_prep_split(B)");

  const CUtensorMap tmA = make_map(Ab, (uint64_t)M, (uint64_t)6 * Kp, BM);
  const CUtensorMap tmB = make_map(Bb, (uint64_t)N, (uint64_t)6 * Kp, BN);
  TcArgs a;
  a.Kp = Kp;
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
  a.vecB = c.vecB;
  a.epi = c.epi_tab;
  a.status = status;
  static int sms = 0;
  static bool attr = false;
  if (!attr) {
    CUTQC_CUDA(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
    int dev = 0;
    CUTQC_CUDA(cudaGetDevice(&dev));
    CUTQC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    attr = true;
  }
  const int tiles = a.tilesM * a.tilesN;
  const int grid = tiles < sms ? tiles : sms;
  k_tc_gemm<<<grid, THREADS, SMEM_BYTES, s>>>(tmA, tmB, a);
  count_launch();
  check_launch("k_tc_gemm");
}

}  // namespace cutqc

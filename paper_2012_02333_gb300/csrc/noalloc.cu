// Full-definition reconstruction that allocates no device memory.
//
// cutqc_reconstruct_fd allocates a workspace and a plan cache with cudaMalloc
// the first time it sees a problem shape.  Some callers cannot allow that:
// processes whose device memory is entirely reserved up front by another
// allocator, or latency-sensitive callers that forbid device allocation after
// start-up because cudaMalloc / cudaFree can synchronise the device and stall
// work on other streams.  cutqc_reconstruct_fd_noalloc serves them: it runs
// the same CUDA-core contraction (row checks, stable compaction of the
// non-zero Kronecker terms, the FP32 / FP64 contraction with the fused FP64
// sum) for a circuit cut into two subcircuits, with all of its scratch in one
// fixed array in device global memory declared in this file.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it until the process exits.  Host code cannot use its name as
// a device address, so the first call on each device looks the address up
// with cudaGetSymbolAddress (with that device current) and caches it.  Every
// call shares the array and leaves its contents behind; each kernel writes the
// scratch it reads before reading it, and the FP64 sum is cleared by the call,
// so nothing has to start at zero.  Calls whose work overlaps on the GPU (for
// example on two streams) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace cutqc {

namespace {

constexpr size_t kScratchBytes = size_t(4) << 20;   // 4 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_sym_mu;
std::map<int, unsigned char*> g_sym_addr;   // device -> device address of g_noalloc_scratch

unsigned char* scratch_address() {
  int dev = 0;
  CUTQC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_sym_mu);
  auto it = g_sym_addr.find(dev);
  if (it != g_sym_addr.end()) return it->second;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    fail(CUTQC_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e));
  g_sym_addr[dev] = static_cast<unsigned char*>(p);
  return static_cast<unsigned char*>(p);
}

size_t up(size_t x) { return (x + 255) / 256 * 256; }

struct Call {
  const cutqc_problem* p;
  void* out;
  double* sum_p;
  cudaStream_t s;
};

void run(void* ctx) {
  const Call& call = *static_cast<const Call*>(ctx);
  if (!call.p) fail(CUTQC_ERR_ARG, "problem is NULL");
  if (!call.out) fail(CUTQC_ERR_ARG, "out is NULL");
  // 16-byte vector stores (the tensors are checked by the planner)
  if (reinterpret_cast<uintptr_t>(call.out) % 16) fail(CUTQC_ERR_ARG, "out must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(call.sum_p) % 8) fail(CUTQC_ERR_ARG, "sum_p must be 8-byte aligned");
  PairPlanHost h;
  plan_pair_host(call.p, h);
  // scratch layout: rows | compacted rows | count | row flags A, B | row max A, B | deposit tables A, B
  size_t off = 0;
  const size_t o_rows = off;
  off = up(off + h.rows.size() * 4);
  const size_t o_crow = off;
  off = up(off + h.rows.size() * 4);
  const size_t o_kc = off;
  off = up(off + 4);
  const size_t o_nzA = off;
  off = up(off + (size_t)h.rowsA * 4);
  const size_t o_nzB = off;
  off = up(off + (size_t)h.rowsB * 4);
  const size_t o_mxA = off;
  off = up(off + (size_t)h.rowsA * 4);
  const size_t o_mxB = off;
  off = up(off + (size_t)h.rowsB * 4);
  const size_t o_dA = off;
  off = up(off + h.depA.size() * 8);
  const size_t o_dB = off;
  off = up(off + h.depB.size() * 8);
  if (off > kScratchBytes)
    fail(CUTQC_ERR_UNSUPPORTED, "problem needs " + std::to_string(off) + " bytes of scratch; this entry point has " +
                                    std::to_string(kScratchBytes) + " (about K <= 8 cuts)");
  unsigned char* base = scratch_address();
  // the plan's tables go into the array by plain copies on the call's stream
  CUTQC_CUDA(cudaMemcpyAsync(base + o_rows, h.rows.data(), h.rows.size() * 4, cudaMemcpyHostToDevice, call.s));
  CUTQC_CUDA(cudaMemcpyAsync(base + o_dA, h.depA.data(), h.depA.size() * 8, cudaMemcpyHostToDevice, call.s));
  CUTQC_CUDA(cudaMemcpyAsync(base + o_dB, h.depB.data(), h.depB.size() * 8, cudaMemcpyHostToDevice, call.s));
  const cutqc_subcircuit& sa = call.p->sub[h.sub_a];
  const cutqc_subcircuit& sb = call.p->sub[h.sub_b];
  launch_row_stats(sa.tensor, call.p->dtype, h.rowsA, h.fA, reinterpret_cast<int32_t*>(base + o_nzA),
                   reinterpret_cast<float*>(base + o_mxA), call.s);
  launch_row_stats(sb.tensor, call.p->dtype, h.rowsB, h.fB, reinterpret_cast<int32_t*>(base + o_nzB),
                   reinterpret_cast<float*>(base + o_mxB), call.s);
  Contraction c;
  c.A = sa.tensor;
  c.B = sb.tensor;
  c.fA = h.fA;
  c.fB = h.fB;
  c.batch = 1;
  c.kmax = h.kmax;
  c.rows = reinterpret_cast<const int32_t*>(base + o_rows);
  c.crow = reinterpret_cast<int32_t*>(base + o_crow);
  c.kcount = reinterpret_cast<int32_t*>(base + o_kc);
  c.depA = reinterpret_cast<const uint64_t*>(base + o_dA);
  c.depB = reinterpret_cast<const uint64_t*>(base + o_dB);
  c.out = call.out;
  c.scale = std::ldexp(1.0, -h.K);
  c.sum = call.sum_p;
  c.vecB = h.vecB;
  c.dtype = call.p->dtype;
  c.nzA = reinterpret_cast<const int32_t*>(base + o_nzA);
  c.nzB = reinterpret_cast<const int32_t*>(base + o_nzB);
  if (call.sum_p) CUTQC_CUDA(cudaMemsetAsync(call.sum_p, 0, sizeof(double), call.s));
  launch_compact(c, call.s);
  launch_cc_gemm(c, call.s);
}

}  // namespace

}  // namespace cutqc

extern "C" int cutqc_reconstruct_fd_noalloc(const cutqc_problem* problem, void* out, double* sum_p, void* stream) {
  cutqc::Call call{problem, out, sum_p, static_cast<cudaStream_t>(stream)};
  return cutqc::run_guarded(&cutqc::run, &call);
}

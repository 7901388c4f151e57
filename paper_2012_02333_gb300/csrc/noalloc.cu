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
// scratch it reads before reading it, and the compaction clears the FP64 sum
// before the contraction adds to it, so nothing has to start at zero.  Calls
// whose work overlaps on the GPU (for example on two streams) race on the
// array.
//
// The plan's tables (the row pair of every Kronecker term and the bit-deposit
// tables of both sides) are written into the array by a small kernel from its
// launch parameters, so a call reads no host buffer after it returns and
// makes no host-to-device copy.
#include <cuda_runtime.h>

#include <algorithm>
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

// The plan tables of a two-subcircuit contraction, as launch parameters.
// Every cut joins the two subcircuits, so the inner index k runs over all
// 4^K assignments, cut 0 in the most significant base-4 digit.
struct TableArgs {
  int K, kmax;
  int32_t mulA[12], mulB[12];   // weight of cut j's digit in the row index of A / B
  int fA, fB, nbA, nbB;         // output bits per side; 256-entry tables per side
  uint64_t va[40], vb[40];      // output bit value of index bit i (least significant first)
  int32_t* rows;                // [2][kmax]: row of A, row of B
  uint64_t* depA;               // [nbA][256]
  uint64_t* depB;               // [nbB][256]
};

__global__ void k_noalloc_tables(const TableArgs a) {
  const int64_t total = (int64_t)a.kmax + (int64_t)(a.nbA + a.nbB) * 256;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < a.kmax) {
      const int k = (int)i;
      int32_t ra = 0, rb = 0;
      for (int j = 0; j < a.K; ++j) {
        const int d = (k >> (2 * (a.K - 1 - j))) & 3;
        ra += d * a.mulA[j];
        rb += d * a.mulB[j];
      }
      a.rows[k] = ra;
      a.rows[a.kmax + k] = rb;
      continue;
    }
    int64_t t = i - a.kmax;
    const bool sideA = t < (int64_t)a.nbA * 256;
    if (!sideA) t -= (int64_t)a.nbA * 256;
    const int b = (int)(t >> 8), v = (int)(t & 255);
    const int f = sideA ? a.fA : a.fB;
    uint64_t g = 0;
    for (int j = 0; j < 8; ++j) {
      const int ib = 8 * b + j;
      if (((v >> j) & 1) && ib < f) g += sideA ? a.va[ib] : a.vb[ib];
    }
    (sideA ? a.depA : a.depB)[t] = g;
  }
}

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
  // out: device memory of the current device, or mapped pinned host memory
  // (written through its device alias); anything else is refused here,
  // before anything runs
  bool out_host = false;
  void* out = resolve_device_out(call.out, &out_host);
  if (call.sum_p && !is_device_memory_here(call.sum_p))
    fail(CUTQC_ERR_ARG, "sum_p must be device memory of the current device");
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
  const cutqc_subcircuit& sa = call.p->sub[h.sub_a];
  const cutqc_subcircuit& sb = call.p->sub[h.sub_b];
  // the tables as launch parameters, checked against the host plan
  TableArgs ta{};
  ta.K = h.K;
  ta.kmax = h.kmax;
  ta.fA = h.fA;
  ta.fB = h.fB;
  ta.nbA = (int)(h.depA.size() / 256);
  ta.nbB = (int)(h.depB.size() / 256);
  if (h.K > 12 || h.fA > 40 || h.fB > 40 || h.kmax != (1 << (2 * h.K)))
    fail(CUTQC_ERR_UNSUPPORTED, "shape outside the allocation-free plan");
  auto weights = [&](const cutqc_subcircuit& sc, int32_t* mul) {
    const int len = sc.k_in + sc.k_out;
    for (int pos = 0; pos < len; ++pos) {
      const int cut = pos < sc.k_in ? sc.in_cut[pos] : sc.out_cut[pos - sc.k_in];
      mul[cut] = int32_t(1) << (2 * (len - 1 - pos));
    }
  };
  weights(sa, ta.mulA);
  weights(sb, ta.mulB);
  const int n = call.p->n_qubits;
  for (int i = 0; i < h.fA; ++i) ta.va[i] = uint64_t(1) << (n - 1 - sa.out_qubit[h.fA - 1 - i]);
  for (int i = 0; i < h.fB; ++i) ta.vb[i] = uint64_t(1) << (n - 1 - sb.out_qubit[h.fB - 1 - i]);
  for (int k = 0; k < h.kmax; ++k) {
    int32_t ra = 0, rb = 0;
    for (int j = 0; j < h.K; ++j) {
      const int d = (k >> (2 * (h.K - 1 - j))) & 3;
      ra += d * ta.mulA[j];
      rb += d * ta.mulB[j];
    }
    if (ra != h.rows[k] || rb != h.rows[h.kmax + k]) fail(CUTQC_ERR_SHAPE, "internal: row table disagrees with the plan");
  }
  for (int side = 0; side < 2; ++side) {
    const std::vector<uint64_t>& want = side ? h.depB : h.depA;
    const uint64_t* v = side ? ta.vb : ta.va;
    const int f = side ? h.fB : h.fA;
    for (size_t t = 0; t < want.size(); ++t) {
      uint64_t g = 0;
      for (int j = 0; j < 8; ++j)
        if (((t & 255) >> j) & 1 && 8 * (int)(t >> 8) + j < f) g += v[8 * (t >> 8) + j];
      if (g != want[t]) fail(CUTQC_ERR_SHAPE, "internal: deposit table disagrees with the plan");
    }
  }
  unsigned char* base = scratch_address();
  ta.rows = reinterpret_cast<int32_t*>(base + o_rows);
  ta.depA = reinterpret_cast<uint64_t*>(base + o_dA);
  ta.depB = reinterpret_cast<uint64_t*>(base + o_dB);
  {
    const int64_t total = (int64_t)ta.kmax + (int64_t)(ta.nbA + ta.nbB) * 256;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 1024);
    k_noalloc_tables<<<blocks, 256, 0, call.s>>>(ta);
    count_launch();
    check_launch("k_noalloc_tables");
  }
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
  c.out = out;
  c.out_host = out_host;
  c.scale = std::ldexp(1.0, -h.K);
  c.sum = call.sum_p;
  c.sum_zero = call.sum_p;   // the compaction clears it before the contraction adds to it
  c.vecB = h.vecB;
  c.dtype = call.p->dtype;
  c.nzA = reinterpret_cast<const int32_t*>(base + o_nzA);
  c.nzB = reinterpret_cast<const int32_t*>(base + o_nzB);
  // the CUDA-core kernels have no bounded waits and no device-side checks,
  // so they write no device status word (c.status stays null)
  launch_compact(c, call.s);
  launch_cc_gemm(c, call.s);
}

}  // namespace

}  // namespace cutqc

extern "C" int cutqc_reconstruct_fd_noalloc(const cutqc_problem* problem, void* out, double* sum_p, void* stream) {
  cutqc::Call call{problem, out, sum_p, static_cast<cudaStream_t>(stream)};
  return cutqc::run_guarded(&cutqc::run, &call);
}

// Internal declarations shared by the library's translation units.
// Nothing here crosses the C ABI (include/cutqc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cutqc.h"

namespace cutqc {

// ---------------------------------------------------------------- errors
// Thrown inside the library only; every entry point converts it to a status.
struct Error {
  int status;
  std::string msg;
};
[[noreturn]] void fail(int status, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define CUTQC_CUDA(call) ::cutqc::check_cuda((call), #call)

void count_launch(int n = 1);

// Programmatic dependent launch: the kernel may start while the previous
// kernel on the stream finishes; it must execute grid_dep_wait() before it
// reads anything that kernel wrote.  grid_dep_launch() lets the next
// programmatically launched kernel start early.
#define CUTQC_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")
#define CUTQC_PDL_LAUNCH() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")
template <typename Kernel, typename... Args>
inline cudaError_t launch_pdl(Kernel k, dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// cutqc_profile: bracket one launch of a main-contraction kernel with events
// recorded on its stream (no-ops while profiling is off)
void prof_begin(cudaStream_t s, cudaEvent_t* ev);
void prof_end(cudaStream_t s, cudaEvent_t ev);

// Runs `f` under the library lock, converting errors to a status and the
// thread's last-error message (the body of every C entry point).
int run_guarded(void (*f)(void*), void* ctx);

// Host-only plan of a two-subcircuit full-definition contraction (no device
// allocation): the final step's row pairs, deposit tables and shape.
struct PairPlanHost {
  int fA = 0, fB = 0, kmax = 0, vecB = 1, sub_a = 0, sub_b = 1, K = 0;
  int rowsA = 0, rowsB = 0;
  std::vector<int32_t> rows;        // [2][kmax]
  std::vector<uint64_t> depA, depB; // [ceil(f/8)][256]
};
void plan_pair_host(const cutqc_problem* p, PairPlanHost& out);
// The device address a kernel writes a full-definition output through: `p`
// itself for device or managed memory of the current device, the device
// alias for pinned host memory mapped for the device (*host = true); any
// other pointer is rejected with CUTQC_ERR_ARG.
void* resolve_device_out(void* p, bool* host);
// true for device memory of the current device and for managed memory
bool is_device_memory_here(const void* p);
void check_launch(const char* what);

// Device status word values (written by kernels, read at sync points).
enum DeviceStatus : int { DEV_OK = 0, DEV_BAD_INDEX = 1, DEV_TIMEOUT = 2 };

// ------------------------------------------------------ the contraction
// One batched contraction (the 4^K sum between two groups of subcircuits):
//   out[batch][g] = scale * sum_k A[rowA(batch,k)][m] * B[rowB(batch,k)][n]
// with g = depA(m) + depB(n) (bit deposit into the output index) and
// m in [0, 2^fA), n in [0, 2^fB).
struct Contraction {
  const void* A = nullptr;      // device, [rowsA][2^fA] row-major
  const void* B = nullptr;      // device, [rowsB][2^fB]
  int fA = 0, fB = 0;
  int batch = 1;                // independent outputs (group builds)
  int kmax = 1;                 // inner extent before compaction
  const int32_t* rows = nullptr;   // device [batch][2][kmax]: rowA, rowB
  int32_t* crow = nullptr;         // device [batch][2][kmax]: compacted rows
  int32_t* kcount = nullptr;       // device [batch]: compacted inner extent
  const uint64_t* depA = nullptr;  // device [ceil(fA/8)][256]
  const uint64_t* depB = nullptr;  // device [ceil(fB/8)][256]
  uint64_t out_batch_stride = 0;   // elements between batch outputs
  void* out = nullptr;
  double scale = 1.0;
  double* sum = nullptr;           // device double or null
  int vecB = 1;                    // consecutive n -> consecutive g run length (1, 2, 4, 8)
  int dtype = CUTQC_F32;
  const int32_t* nzA = nullptr;    // device row non-zero flags of A (or null)
  const int32_t* nzB = nullptr;
  const float* rmaxA = nullptr;    // device row max |.| of A (or null)
  const float* rmaxB = nullptr;
  int rowsA = 0, rowsB = 0;
  // split-precision control (tensor-core path): the compaction also computes
  // the a-priori magnitude S = scale * sum_kept max|A_row| max|B_row| into
  // *bound, and writes the number of split products to *nseg: `nseg_fixed`
  // if non-zero, else 3 when split_err3 * S <= split_tol, otherwise 6.
  double* bound = nullptr;
  int32_t* nseg = nullptr;
  bool profile = false;            // bracket the contraction kernel for cutqc_profile
  double* sum_zero = nullptr;      // device double the compaction zeroes before the contraction adds to it
  bool compacted = false;          // crow / kcount / nseg / bound already written (row statistics did it)
  int nseg_fixed = 0;
  double split_tol = 2.5e-7;
  bool tf32 = false;               // tensor-core path: TF32 x3 pieces instead of bf16
  int* status = nullptr;           // device status word (DeviceStatus) of this device
  bool out_host = false;           // `out` is pinned host memory (written over the host link)
  // tensor-core path only: keep a top-32 of the written values per epilogue
  // warp (lists of 32 at topk_v / topk_i) and report the number of lists
  float* topk_v = nullptr;
  int64_t* topk_i = nullptr;
  int* topk_nlists = nullptr;
};

// k_cc.cu
// Stable compaction of a contraction's row pairs (early termination) and the
// split-count choice, done by the last block of a row-statistics launch.
struct CompactJob {
  int active = 0;
  const int32_t* rows = nullptr;       // [2][kmax]
  int kmax = 0;
  const int32_t* nzA = nullptr;
  const int32_t* nzB = nullptr;
  const float* rmaxA = nullptr;
  const float* rmaxB = nullptr;
  int32_t* crow = nullptr;             // [2][kmax]
  int32_t* kcount = nullptr;
  double scale = 1.0;
  double* bound = nullptr;
  int32_t* nseg = nullptr;
  int nseg_fixed = 0;
  double split_tol = 2.5e-7;
  double* sum_zero = nullptr;
  unsigned* counter = nullptr;         // zero before the launch
};
struct RowStatsJobs {   // up to two tensors whose rows get non-zero flags and max |.|
  int n;
  const void* t[2];
  int64_t rows[2], cols[2];
  int32_t* flags[2];
  float* rmax[2];
  int chunks[2];          // blocks per row (set by the launcher; long rows of few-row tensors are split)
  int warp[2];            // 1: rows of at most 2048 values, reduced by warps (set by the launcher)
  int64_t blocks0;        // blocks of tensor 0 (set by the launcher)
  CompactJob cj;
};
void launch_row_stats(const RowStatsJobs& jobs, int dtype, cudaStream_t s);
void launch_row_stats(const void* T, int dtype, int rows, int f, int32_t* flags, float* rmax, cudaStream_t s);
void launch_compact(const Contraction& c, cudaStream_t s);
void launch_cc_gemm(const Contraction& c, cudaStream_t s);
void launch_fill_zero(void* p, size_t bytes, cudaStream_t s);
// Low-rank final contraction (at most 16 kept terms, the N side owning the
// two lowest output bits): one problem, or a device list of problems and work
// items built by lowrank_batch_tables (all of one dtype) in one launch.
bool lowrank_eligible(const Contraction& c);
int64_t lowrank_items(const Contraction& c);
void launch_lowrank(const Contraction& c, cudaStream_t s);
size_t lowrank_batch_bytes(const std::vector<Contraction>& cs);
void lowrank_batch_tables(const std::vector<Contraction>& cs, std::vector<char>& host, int64_t* n_items);
void launch_lowrank_batch(const void* dev_tables, const std::vector<Contraction>& cs, int64_t n_items,
                          cudaStream_t s);

// k_attr.cu: tensor T[a][b][x] of one subcircuit from its variant distributions
// P[s][mb][y] (Eq. 2, Eq. 3); arguments already validated
void launch_attribute(const void* P, int dtype, int d, int k_in, const int* meas_q, int k_out, const int* out_q,
                      int n_eff, void* tensor, cudaStream_t s);

// k_metrics.cu: Eq. 16 chi^2 and total variation; inverse-transform sampling.
// Scratch is the caller's (sizes below); the distance scratch must start
// zeroed and is left zeroed.
size_t distance_scratch_bytes();
void launch_distance(const void* a, const void* b, int64_t n, int dtype, double* chi2, double* tv, void* scratch,
                     cudaStream_t s);
size_t sample_scratch_bytes(int64_t n);
void launch_sample(const void* p, int64_t n, int dtype, const double* u, int64_t m, int64_t* out, void* scratch,
                   cudaStream_t s);

// k_tc.cu
// One block, one thread: waits on a device flag that nothing sets, bounded by
// `limit_us`, then records DEV_TIMEOUT in *status (the bounded-wait path of
// every kernel that waits, exercised without any other work).
void launch_wait_selftest(int* status, int limit_us, cudaStream_t s);
bool tc_supported(const Contraction& c);
// With `fused`, the row statistics of both operands (non-zero flags and row
// max |.| into the given arrays), the compaction and the operand preparation
// run as one cooperative launch with a grid barrier (kmax <= 4096): for BF16
// pieces and at least 128 terms one block per term reads its two rows once
// (`look`: 8 * kmax bytes for the barrier counter, a kept-term mask and the
// bound products; the launch zeroes the counter and the mask first), else the
// statistics run over rows and the preparation over tiles (`barrier`, a
// device counter the launch zeroes first); without `fused` the statistics
// come from an earlier launch.
struct TcFusedStats {
  int32_t* nzA;
  int32_t* nzB;
  float* rmaxA;
  float* rmaxB;
  unsigned* barrier;
  unsigned* look;
};
void launch_tc_bf16x3(const Contraction& c, void* ws, size_t ws_bytes, cudaStream_t s,
                      const TcFusedStats* fused = nullptr);
size_t tc_workspace_bytes(const Contraction& c);


// k_dd.cu
struct DdEvalSub {
  int64_t rows, cols;
  const void* m;               // merged tensor [rows][2^a] in the problem's dtype
  const float* mc;             // FP32 tensors: compensation term of each merged value
  int a, mg, nbA, nbM;
  uint64_t zoom;
  const uint64_t* depAct;
  const uint64_t* depMrg;
  int act_rank[36];
  int cuts[12];
  int ncuts;
};
struct DdEvalArgs {
  int n_sub, n_cuts, n_active, n_cand;
  int f64;                     // merged tensors are FP64
  int64_t max_rows;
  double scale;
  const int64_t* cand_idx;
  const void* tens[16];
  DdEvalSub sub[16];
};
// log2 of the chunks each output's run is split into by the contiguous-run merge (0 = none)
int dd_merge_chunks(int64_t rows, int a, int mg);
// the deposit tables of up to 32 index bits each (bit i = the output value of
// index bit i, least significant first), built on the device: no host copy
void launch_deposit_tables(const uint64_t* act, int na, const uint64_t* mrg, int nm, uint64_t* tab_act,
                           uint64_t* tab_mrg, cudaStream_t s);
// blk: the active index bits below the highest merged bit, when every bit
// below it is merged or active, none is zoomed and at most two are active
// (dd_merge_block; 0 = not that layout): the block form then sums each
// contiguous block of 2^(mg + popcount(blk)) values into its outputs
void launch_dd_merge(const void* T, int dtype, int64_t rows, int f, int a, int mg, const uint64_t* depAct,
                     const uint64_t* depMrg, uint64_t zoom, bool run, bool dense_bits, void* M, float* MC,
                     void* part, cudaStream_t s, uint64_t blk = 0);
uint64_t dd_merge_block(uint64_t merged_mask, int mg, uint64_t active_mask, uint64_t zoom);
size_t topk_workspace_bytes(int64_t n);
void launch_topk(const void* bins, int dtype, int64_t n, void* ws, float* out_v, int64_t* out_i, cudaStream_t s);
// merge nlists lists of 32 (value, index) candidates, laid out like launch_topk's workspace
void launch_topk_lists(void* ws, int64_t nlists, float* out_v, int64_t* out_i, cudaStream_t s);
// chunks of the Kronecker terms per candidate in the FP64 re-evaluation (<= 64)
int dd_eval_chunks(int n_cuts);
void launch_dd_rerank(const DdEvalArgs& a, int dtype, double* m64, double* part, double* val, cudaStream_t s);

// k_bwd.cu
struct BwdEdges {   // edges as pairs of index bits (least significant = 0)
  int n;
  int p[96], q[96];
};
struct BwdBits {
  int n;
  int p[16];
};
// The MaxCut adjoint through a per-output key (cut count and bridge bits of
// each output index, 2 bytes per output): bwd_keys_bytes is the workspace the
// keys of one side need, 0 when the shape does not take them (f outside
// 3..24, or more than 4096 (count, bits) combinations); launch_bwd_keys builds
// them.  With keys the row sums of FP32 tensors run in compensated FP32 and
// the gradient is a table lookup per output (the same values as without).
size_t bwd_keys_bytes(int f, const BwdEdges& internal, const BwdBits& sel);
void launch_bwd_keys(int f, const BwdEdges& internal, const BwdBits& sel, uint16_t* keys, cudaStream_t s);
void launch_bwd_rowsums(const void* X, int dtype, int64_t rows, int f, const BwdEdges& internal, const BwdBits& sel,
                        double* out, cudaStream_t s, const uint16_t* keys = nullptr);
void launch_bwd_maxcut_grad(const int32_t* rowX, const int32_t* rowY, int kmax, int fX, const BwdEdges& internal,
                            const BwdBits& bitX, const double* sumsY, int64_t rowsY, double scale, void* dX, int dtype,
                            cudaStream_t s, const uint16_t* keys = nullptr);
void launch_bwd_maxcut_loss(const int32_t* rowA, const int32_t* rowB, int kmax, const double* sA, int64_t rowsA,
                            const double* sB, int64_t rowsB, int nbridge, double scale, double* loss, cudaStream_t s);
void launch_bwd_cc(const void* Y, const void* G, const int32_t* rowX, const int32_t* rowY, int kmax, int fX, int fY,
                   const uint64_t* depX, const uint64_t* depY, double scale, void* dX, int dtype, cudaStream_t s);
void launch_dot(const void* a, const void* b, int64_t n, int dtype, double* out, cudaStream_t s);

// k_sim.cu
struct SimPlan {
  int d, k_in, k_out, n_eff;
  std::vector<int32_t> init_q, meas_q, out_q;
  std::vector<cutqc_gate> gates;
};
void run_subcircuit_sim(const SimPlan& p, int dtype, void* tensor, cudaStream_t s);
void release_sim_scratch();   // frees the simulator's cached scratch on every device

}  // namespace cutqc

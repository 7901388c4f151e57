// The C ABI (include/cutqc.h): validation, the contraction planner, the
// per-device workspace and plan cache, and the host side of every call.
//
// Planner.  A cut circuit with S subcircuits is reduced to one contraction
// between two groups (Sec. 3.3: the 4^K Kronecker products).  While more than
// two nodes remain, the pair of connected nodes whose merged tensor is
// smallest is merged first (the greedy "smallest subcircuits first" order of
// Sec. 4.2, which keeps the carried-over vectors small); a merge is itself a
// batched contraction over the cuts internal to the pair, batched over the
// pair's remaining open cuts, with the output bits concatenated.  The last
// contraction deposits its (m, n) pairs into the uncut circuit's output index.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <charconv>
#include <cmath>
#include <functional>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace cutqc {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;
static thread_local int g_last_algo = CUTQC_CC;
static thread_local const int32_t* g_last_nseg = nullptr;     // device
static thread_local const double* g_last_bound = nullptr;     // device
static thread_local cudaStream_t g_last_stream = nullptr;
static std::atomic<int64_t> g_launches{0};
static std::recursive_mutex g_mu;
static uint64_t g_call = 0;   // outermost API calls so far (under the library lock)
static int g_depth = 0;       // nesting of guarded calls

void fail(int status, const std::string& msg) { throw Error{status, msg}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    const int st = (e == cudaErrorMemoryAllocation) ? CUTQC_ERR_OOM : CUTQC_ERR_CUDA;
    fail(st, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

void count_launch(int n) { g_launches += n; }

void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) fail(CUTQC_ERR_CUDA, std::string("launch of ") + what + ": " + cudaGetErrorString(e));
}

template <class F>
static int guarded(F&& f) {
  std::lock_guard<std::recursive_mutex> lk(g_mu);
  if (g_depth == 0) ++g_call;
  struct Depth {
    Depth() { ++g_depth; }
    ~Depth() { --g_depth; }
  } depth;
  try {
    f();
    return CUTQC_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return CUTQC_ERR_OOM;
  } catch (...) {
    g_last_error = "unexpected internal error";
    return CUTQC_ERR_CUDA;
  }
}

int run_guarded(void (*f)(void*), void* ctx) {
  return guarded([&] { f(ctx); });
}

// ------------------------------------------------------------- validation
static constexpr int kMaxCuts = 12;
static constexpr int kMaxSub = 16;
static constexpr int kMaxFD = 34;
static constexpr int kMaxQubits = 4096;

static size_t dtype_size(int dt) { return dt == CUTQC_F64 ? 8 : 4; }

// Device arrays are read and written with 16-byte (and wider) vector
// accesses, device scalars with their natural width: a pointer that breaks
// this would fault on the GPU, so it is rejected here instead.
static void need_aligned(const void* p, size_t bytes, const char* what) {
  if (p && reinterpret_cast<uintptr_t>(p) % bytes != 0)
    fail(CUTQC_ERR_ARG, std::string(what) + " must be " + std::to_string(bytes) + "-byte aligned");
}

static void validate(const cutqc_problem* p, bool need_tensors) {
  if (!p) fail(CUTQC_ERR_ARG, "problem is NULL");
  if (p->dtype != CUTQC_F32 && p->dtype != CUTQC_F64) fail(CUTQC_ERR_ARG, "dtype must be CUTQC_F32 or CUTQC_F64");
  if (p->n_sub < 1 || !p->sub) fail(CUTQC_ERR_ARG, "need n_sub >= 1 subcircuits");
  if (p->n_sub > kMaxSub) fail(CUTQC_ERR_UNSUPPORTED, "n_sub > 16");
  if (p->n_qubits < 1) fail(CUTQC_ERR_SHAPE, "n_qubits must be >= 1");
  if (p->n_qubits > kMaxQubits) fail(CUTQC_ERR_UNSUPPORTED, "n_qubits > 4096");
  if (p->n_cuts < 0) fail(CUTQC_ERR_SHAPE, "n_cuts must be >= 0");
  if (p->n_cuts > kMaxCuts) fail(CUTQC_ERR_UNSUPPORTED, "n_cuts > 12");
  std::vector<int> in_seen(p->n_cuts, -1), out_seen(p->n_cuts, -1), q_seen(p->n_qubits, 0);
  int total_eff = 0;
  for (int c = 0; c < p->n_sub; ++c) {
    const cutqc_subcircuit& s = p->sub[c];
    if (s.k_in < 0 || s.k_out < 0 || s.n_eff < 0) fail(CUTQC_ERR_SHAPE, "negative slot or output count");
    if (s.k_in + s.k_out > kMaxCuts) fail(CUTQC_ERR_UNSUPPORTED, "subcircuit has more than 12 cut slots");
    if (s.n_eff > 40) fail(CUTQC_ERR_UNSUPPORTED, "subcircuit has more than 40 output qubits");
    if ((s.k_in && !s.in_cut) || (s.k_out && !s.out_cut) || (s.n_eff && !s.out_qubit))
      fail(CUTQC_ERR_ARG, "NULL slot or output array");
    if (need_tensors && !s.tensor) fail(CUTQC_ERR_ARG, "NULL tensor pointer");
    if (need_tensors) need_aligned(s.tensor, 16, "a subcircuit tensor");
    for (int j = 0; j < s.k_in; ++j) {
      const int k = s.in_cut[j];
      if (k < 0 || k >= p->n_cuts) fail(CUTQC_ERR_SHAPE, "init slot names a cut id out of range");
      if (in_seen[k] >= 0) fail(CUTQC_ERR_SHAPE, "cut id appears in two init slots");
      in_seen[k] = c;
    }
    for (int j = 0; j < s.k_out; ++j) {
      const int k = s.out_cut[j];
      if (k < 0 || k >= p->n_cuts) fail(CUTQC_ERR_SHAPE, "measurement slot names a cut id out of range");
      if (out_seen[k] >= 0) fail(CUTQC_ERR_SHAPE, "cut id appears in two measurement slots");
      out_seen[k] = c;
    }
    for (int i = 0; i < s.n_eff; ++i) {
      const int q = s.out_qubit[i];
      if (q < 0 || q >= p->n_qubits) fail(CUTQC_ERR_SHAPE, "output qubit out of range");
      if (q_seen[q]) fail(CUTQC_ERR_SHAPE, "output qubit appears twice");
      q_seen[q] = 1;
    }
    total_eff += s.n_eff;
  }
  for (int k = 0; k < p->n_cuts; ++k) {
    if (in_seen[k] < 0 || out_seen[k] < 0) fail(CUTQC_ERR_SHAPE, "cut id without both an init and a measurement slot");
    if (in_seen[k] == out_seen[k]) fail(CUTQC_ERR_SHAPE, "cut joins a subcircuit to itself");
  }
  if (total_eff != p->n_qubits) fail(CUTQC_ERR_SHAPE, "output qubits do not cover n_qubits");
}

// ------------------------------------------------------------------ plans
struct Node {
  std::vector<int> cuts;    // open cut ids, row digit order (first = most significant)
  std::vector<int> bits;    // output position of each x bit (x bit 0 = most significant)
  int orig = -1;            // original subcircuit, or -1 for a merge result
  int f() const { return (int)bits.size(); }
  int64_t rows() const { return int64_t(1) << (2 * cuts.size()); }
};

struct Step {
  int a = -1, b = -1, result = -1;    // node indices (result -1: final output)
  int batch = 1, kmax = 1;
  std::vector<int32_t> rows;          // [batch][2][kmax]
  std::vector<uint64_t> depA, depB;   // [ceil(f/8)][256]
  uint64_t out_stride = 0;
  int vecB = 1;
  size_t off_rows = 0, off_depA = 0, off_depB = 0;   // in the plan's device block
  size_t ws_crow = 0, ws_kcount = 0;                 // in the workspace
  size_t ws_bound = 0, ws_nseg = 0, ws_counter = 0, ws_look = 0;
};

struct DdSubPlan {
  int64_t rows = 1;
  int f = 0, a = 0, mg = 0;
  uint64_t zoom = 0;                   // x index bits fixed by zoomed qubits
  std::vector<uint64_t> depAct, depMrg;
  size_t off_act = 0, off_mrg = 0;     // in the plan's DD table block
  std::vector<int> act_rank;           // bin rank of each active output (x-bit order)
  std::vector<int> cuts;
  size_t ws_merged = 0;                // offset of the merged tensor in the front region
  size_t ws_mc = 0;                    // ... and of its compensation terms (FP32 tensors)
  size_t ws_part = 0;                  // partial sums of split runs (contiguous-run merge)
  bool run = false;                    // merged qubits are the lowest output bits
  bool dense = false;                  // ... and the active qubits the bits directly above them
  uint64_t blk = 0;                    // active bits below the highest merged one (block form of the merge)
};

struct Plan {
  int n_out = 0, K = 0, dtype = CUTQC_F32;
  uint64_t used_call = 0;              // the last API call that used the plan (it is not evicted during it)
  int tuned = -1;                      // measured final form under CUTQC_AUTO (batched calls): -1 not yet,
                                       // CUTQC_CC, or CUTQC_AUTO (tensor core, device-chosen split)
  std::vector<DdSubPlan> dd;           // dynamic definition only
  size_t dd_front = 0;
  void* ddtab = nullptr;
  std::vector<Node> nodes;
  std::vector<Step> steps;
  std::vector<size_t> ws_node;    // workspace offset of each merge-result tensor
  std::vector<size_t> ws_nz;      // workspace offset of each node's row flags
  std::vector<size_t> ws_rmax;    // workspace offset of each node's row max |.|
  size_t ws_bytes = 0;
  void* dtab = nullptr;
  size_t dtab_bytes = 0;
  ~Plan() {
    if (dtab) cudaFree(dtab);
    if (ddtab) cudaFree(ddtab);
  }
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  uint64_t gen = 0;
};

constexpr int kBranches = 8;      // parallel branches of a captured batch

struct DeviceState {
  void* ws = nullptr;
  size_t ws_bytes = 0;
  uint64_t ws_gen = 0;            // bumped whenever the workspace moves
  void* one = nullptr;            // a device constant 1.0 (f64) / 1.0f (f32)
  std::unordered_map<std::string, std::unique_ptr<Plan>> plans;
  std::vector<std::string> order;
  std::unordered_map<std::string, GraphEntry> graphs;   // captured batched calls
  cudaStream_t branch[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {}, mid[kBranches] = {};
  int* status = nullptr;          // device status word written by kernels with bounded waits
  void* aux = nullptr;            // distance / sampling scratch (zeroed when (re)allocated)
  size_t aux_bytes = 0;
  // device work lists of batched low-rank contractions, per batch (they point
  // into the workspace, so they go whenever the captured graphs go)
  std::unordered_map<std::string, void*> lr_tables;
  uint64_t plan_gen = 0;          // bumped whenever a plan is evicted
  // repeated batched calls: the raw arguments -> the captured graph's key
  struct BatchFast {
    std::string gk;
    uint64_t ws_gen = 0, plan_gen = 0;
  };
  std::unordered_map<std::string, BatchFast> batch_fast;
};
static std::map<int, DeviceState> g_dev;

// main-kernel timing (cutqc_profile)
static bool g_profile = false;
static bool g_capturing = false;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_events;

void prof_begin(cudaStream_t s, cudaEvent_t* a) {
  *a = nullptr;
  if (!g_profile || g_capturing) return;
  CUTQC_CUDA(cudaEventCreate(a));
  CUTQC_CUDA(cudaEventRecord(*a, s));
}
void prof_end(cudaStream_t s, cudaEvent_t a) {
  if (!a) return;
  cudaEvent_t b;
  CUTQC_CUDA(cudaEventCreate(&b));
  CUTQC_CUDA(cudaEventRecord(b, s));
  g_prof_events.emplace_back(a, b);
}

static DeviceState& device_state() {
  int dev = 0;
  CUTQC_CUDA(cudaGetDevice(&dev));
  return g_dev[dev];
}

// The device status word (DeviceStatus) of this device, allocated and zeroed
// on first use (outside any stream capture: every entry point that launches a
// waiting kernel asks for it before launching).
static int* status_word(DeviceState& ds) {
  if (!ds.status) {
    CUTQC_CUDA(cudaMalloc(&ds.status, 256));
    CUTQC_CUDA(cudaMemset(ds.status, 0, sizeof(int)));
  }
  return ds.status;
}

// After the caller has synchronised: report and clear a recorded device status.
static void check_status(DeviceState& ds) {
  if (!ds.status) return;
  int v = 0;
  CUTQC_CUDA(cudaMemcpy(&v, ds.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v == DEV_OK) return;
  CUTQC_CUDA(cudaMemset(ds.status, 0, sizeof(int)));
  if (v == DEV_TIMEOUT)
    fail(CUTQC_ERR_TIMEOUT, "a bounded device wait ran out; outputs of the calls since the last check are invalid");
  fail(CUTQC_ERR_DEVICE, "a device-side check failed; outputs of the calls since the last check are invalid");
}

// Scratch of cutqc_distance (a fixed region that must stay zeroed between
// calls: its kernel resets it) followed by that of cutqc_sample.
static size_t aux_distance_bytes() { return (distance_scratch_bytes() + 255) / 256 * 256; }
static char* aux_buffer(DeviceState& ds, size_t sample_bytes) {
  const size_t need = aux_distance_bytes() + (sample_bytes + 255) / 256 * 256;
  if (need > ds.aux_bytes) {
    if (ds.aux) CUTQC_CUDA(cudaFree(ds.aux));
    ds.aux = nullptr;
    ds.aux_bytes = 0;
    CUTQC_CUDA(cudaMalloc(&ds.aux, need));
    CUTQC_CUDA(cudaMemset(ds.aux, 0, need));
    ds.aux_bytes = need;
  }
  return static_cast<char*>(ds.aux);
}

static void drop_graphs(DeviceState& ds) {
  for (auto& kv : ds.graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  ds.graphs.clear();
  ds.batch_fast.clear();
  for (auto& kv : ds.lr_tables)
    if (kv.second) cudaFree(kv.second);
  ds.lr_tables.clear();
}

static void* workspace(DeviceState& ds, size_t bytes) {
  if (bytes > ds.ws_bytes) {
    drop_graphs(ds);   // captured launches point into the old workspace
    ++ds.ws_gen;
    if (ds.ws) CUTQC_CUDA(cudaFree(ds.ws));
    ds.ws = nullptr;
    ds.ws_bytes = 0;
    const size_t want = std::max(bytes, size_t(1) << 20);
    CUTQC_CUDA(cudaMalloc(&ds.ws, want));
    ds.ws_bytes = want;
  }
  return ds.ws;
}

static size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// deposit tables for one side: entry [byte][v] = sum over set bits j of v of
// the output bit value of index bit (8*byte + j) (index bit 0 = least
// significant = the node's last x bit)
static std::vector<uint64_t> deposit_table(const std::vector<uint64_t>& bitval) {
  const int f = (int)bitval.size();
  const int nb = (f + 7) / 8;
  std::vector<uint64_t> t(std::max(nb, 1) * 256, 0);
  for (int b = 0; b < nb; ++b)
    for (int v = 0; v < 256; ++v) {
      uint64_t g = 0;
      for (int j = 0; j < 8; ++j)
        if ((v >> j) & 1) {
          const int ib = 8 * b + j;
          if (ib < f) g += bitval[ib];
        }
      t[b * 256 + v] = g;
    }
  return t;
}

static int64_t row_index(const Node& nd, const std::vector<int>& digit) {
  int64_t r = 0;
  for (int c : nd.cuts) r = 4 * r + digit[c];
  return r;
}

// Build the contraction of nodes a and b.  result >= 0: a merge whose output
// node has open cuts `open` and bits a.bits ++ b.bits; result < 0: the final
// contraction into n_out output bits.
static Step make_step(Plan& P, int ia, int ib, int result, const std::vector<int>& open, int ncuts_total) {
  const Node& A = P.nodes[ia];
  const Node& B = P.nodes[ib];
  std::vector<int> inner;
  for (int c : A.cuts)
    if (std::find(B.cuts.begin(), B.cuts.end(), c) != B.cuts.end()) inner.push_back(c);
  std::sort(inner.begin(), inner.end());
  Step st;
  st.a = ia;
  st.b = ib;
  st.result = result;
  st.batch = 1 << (2 * open.size());
  st.kmax = 1 << (2 * inner.size());
  st.rows.resize((size_t)st.batch * 2 * st.kmax);
  std::vector<int> digit(std::max(ncuts_total, 1), 0);
  for (int bt = 0; bt < st.batch; ++bt) {
    for (size_t j = 0; j < open.size(); ++j) digit[open[j]] = (bt >> (2 * (open.size() - 1 - j))) & 3;
    for (int k = 0; k < st.kmax; ++k) {
      for (size_t j = 0; j < inner.size(); ++j) digit[inner[j]] = (k >> (2 * (inner.size() - 1 - j))) & 3;
      st.rows[(size_t)bt * 2 * st.kmax + k] = (int32_t)row_index(A, digit);
      st.rows[(size_t)bt * 2 * st.kmax + st.kmax + k] = (int32_t)row_index(B, digit);
    }
  }
  const int fA = A.f(), fB = B.f();
  std::vector<uint64_t> va(fA), vb(fB);
  if (result >= 0) {
    // concatenation: x = (xA, xB), xB in the low bits
    for (int i = 0; i < fA; ++i) va[i] = uint64_t(1) << (fB + i);
    for (int i = 0; i < fB; ++i) vb[i] = uint64_t(1) << i;
    st.out_stride = uint64_t(1) << (fA + fB);
    st.vecB = 4;
  } else {
    // index bit i (from the least significant) of m is x bit f-1-i
    for (int i = 0; i < fA; ++i) va[i] = uint64_t(1) << (P.n_out - 1 - A.bits[fA - 1 - i]);
    for (int i = 0; i < fB; ++i) vb[i] = uint64_t(1) << (P.n_out - 1 - B.bits[fB - 1 - i]);
    st.out_stride = 0;
    int run = 0;
    while (run < fB && run < 3 && vb[run] == (uint64_t(1) << run)) ++run;
    st.vecB = 1 << run;
  }
  st.depA = deposit_table(va);
  st.depB = deposit_table(vb);
  return st;
}

// Plan a problem whose nodes are given (original subcircuits, or merged DD
// tensors) with output positions already in the nodes' bits.
// One greedy merge among the live nodes: the connected pair whose merged
// tensor is smallest (ties: lowest indices; an unconnected pair only when no
// pair shares a cut), appended as a batched group-build step.
static void merge_best_pair(Plan& P, std::vector<int>& live, int ncuts) {
  auto shared = [&](int i, int j) {
    int s = 0;
    for (int c : P.nodes[i].cuts)
      if (std::find(P.nodes[j].cuts.begin(), P.nodes[j].cuts.end(), c) != P.nodes[j].cuts.end()) ++s;
    return s;
  };
  {
    // the connected pair with the smallest merged tensor (ties: lowest indices)
    double best = -1;
    int bi = -1, bj = -1;
    bool best_conn = false;
    for (size_t x = 0; x < live.size(); ++x)
      for (size_t y = x + 1; y < live.size(); ++y) {
        const int i = live[x], j = live[y];
        const int sh = shared(i, j);
        const int open = (int)(P.nodes[i].cuts.size() + P.nodes[j].cuts.size()) - 2 * sh;
        const double size = std::ldexp(1.0, 2 * open + P.nodes[i].f() + P.nodes[j].f());
        const bool conn = sh > 0;
        if (bi < 0 || (conn && !best_conn) || (conn == best_conn && size < best)) {
          best = size;
          bi = i;
          bj = j;
          best_conn = conn;
        }
      }
    Node m;
    for (int c : P.nodes[bi].cuts)
      if (std::find(P.nodes[bj].cuts.begin(), P.nodes[bj].cuts.end(), c) == P.nodes[bj].cuts.end()) m.cuts.push_back(c);
    for (int c : P.nodes[bj].cuts)
      if (std::find(P.nodes[bi].cuts.begin(), P.nodes[bi].cuts.end(), c) == P.nodes[bi].cuts.end()) m.cuts.push_back(c);
    std::sort(m.cuts.begin(), m.cuts.end());
    m.bits = P.nodes[bi].bits;
    m.bits.insert(m.bits.end(), P.nodes[bj].bits.begin(), P.nodes[bj].bits.end());
    if (m.rows() * (int64_t(1) << m.f()) > (int64_t(1) << 36))
      fail(CUTQC_ERR_UNSUPPORTED, "an intermediate group tensor would exceed 2^36 entries");
    P.nodes.push_back(m);
    const int r = (int)P.nodes.size() - 1;
    P.steps.push_back(make_step(P, bi, bj, r, m.cuts, ncuts));
    live.erase(std::find(live.begin(), live.end(), bi));
    live.erase(std::find(live.begin(), live.end(), bj));
    live.push_back(r);
  }
}

static void plan_contractions(Plan& P, int ncuts) {
  std::vector<int> live;
  for (size_t i = 0; i < P.nodes.size(); ++i) live.push_back((int)i);
  while (live.size() > 2) merge_best_pair(P, live, ncuts);
  if (live.size() == 1) {
    // no partner: contract with a constant 1 node (f = 0, no cuts)
    Node one;
    one.orig = -2;
    P.nodes.push_back(one);
    live.push_back((int)P.nodes.size() - 1);
  }
  int a = live[0], b = live[1];
  // the N side (vector stores) is the node holding the lowest output bit
  auto holds_last = [&](int i) {
    for (int pos : P.nodes[i].bits)
      if (pos == P.n_out - 1) return true;
    return false;
  };
  if (holds_last(a) && !holds_last(b)) std::swap(a, b);
  P.steps.push_back(make_step(P, a, b, -1, {}, ncuts));
}

static void finalize_plan(Plan& P) {
  // device tables
  size_t off = 0;
  for (Step& st : P.steps) {
    st.off_rows = off;
    off = align_up(off + st.rows.size() * 4);
    st.off_depA = off;
    off = align_up(off + st.depA.size() * 8);
    st.off_depB = off;
    off = align_up(off + st.depB.size() * 8);
  }
  P.dtab_bytes = std::max<size_t>(off, 256);
  CUTQC_CUDA(cudaMalloc(&P.dtab, P.dtab_bytes));
  std::vector<char> host(P.dtab_bytes, 0);
  for (Step& st : P.steps) {
    std::memcpy(host.data() + st.off_rows, st.rows.data(), st.rows.size() * 4);
    std::memcpy(host.data() + st.off_depA, st.depA.data(), st.depA.size() * 8);
    std::memcpy(host.data() + st.off_depB, st.depB.data(), st.depB.size() * 8);
  }
  CUTQC_CUDA(cudaMemcpy(P.dtab, host.data(), P.dtab_bytes, cudaMemcpyHostToDevice));
  // workspace layout: merge results, row flags, compacted rows, counts
  size_t w = 0;
  const size_t es = dtype_size(P.dtype);
  P.ws_node.assign(P.nodes.size(), 0);
  P.ws_nz.assign(P.nodes.size(), 0);
  for (size_t i = 0; i < P.nodes.size(); ++i) {
    if (P.nodes[i].orig == -1) {
      P.ws_node[i] = w;
      w = align_up(w + (size_t)P.nodes[i].rows() * ((size_t)1 << P.nodes[i].f()) * es);
    }
  }
  P.ws_rmax.assign(P.nodes.size(), 0);
  for (size_t i = 0; i < P.nodes.size(); ++i) {
    P.ws_nz[i] = w;
    w = align_up(w + (size_t)P.nodes[i].rows() * 4);
    P.ws_rmax[i] = w;
    w = align_up(w + (size_t)P.nodes[i].rows() * 4);
  }
  for (Step& st : P.steps) {
    st.ws_crow = w;
    w = align_up(w + st.rows.size() * 4);
    st.ws_kcount = w;
    w = align_up(w + (size_t)st.batch * 4);
    st.ws_bound = w;
    w = align_up(w + 8);
    st.ws_nseg = w;
    w = align_up(w + 4);
    st.ws_counter = w;
    w = align_up(w + 4);
    st.ws_look = w;   // barrier, kept-term mask and bound products of the operand preparation
    w = align_up(w + (st.batch == 1 && st.kmax <= 4096 ? (size_t)st.kmax * 8 : 0));
  }
  P.ws_bytes = w;
}

static void put_int(std::string& o, long long v) {
  char buf[24];
  const auto r = std::to_chars(buf, buf + sizeof buf, v);
  o.append(buf, r.ptr);
}

static std::string fd_key(const cutqc_problem* p, int mode, const int8_t* role, int algo) {
  std::string o;
  o.reserve(64 + 48 * (size_t)p->n_sub);
  put_int(o, mode);
  o += ':';
  put_int(o, algo);
  o += ':';
  put_int(o, p->n_qubits);
  o += ',';
  put_int(o, p->n_cuts);
  o += ',';
  put_int(o, p->n_sub);
  o += ',';
  put_int(o, p->dtype);
  o += '|';
  for (int c = 0; c < p->n_sub; ++c) {
    const cutqc_subcircuit& s = p->sub[c];
    put_int(o, s.k_in);
    o += ',';
    put_int(o, s.k_out);
    o += ',';
    put_int(o, s.n_eff);
    o += ':';
    for (int j = 0; j < s.k_in; ++j) {
      put_int(o, s.in_cut[j]);
      o += ',';
    }
    o += ';';
    for (int j = 0; j < s.k_out; ++j) {
      put_int(o, s.out_cut[j]);
      o += ',';
    }
    o += ';';
    for (int j = 0; j < s.n_eff; ++j) {
      put_int(o, s.out_qubit[j]);
      o += ',';
    }
    o += '|';
  }
  if (role)
    for (int q = 0; q < p->n_qubits; ++q) put_int(o, role[q]);
  return o;
}

// Plans are cached per device (at most 64 beyond those the current call
// uses).  Evicting one drops the captured graphs, whose launches read its
// device tables, and bumps the plan generation checked by the batch fast path.

static Plan& get_plan(DeviceState& ds, const std::string& key, const std::function<void(Plan&)>& build) {
  auto it = ds.plans.find(key);
  if (it != ds.plans.end()) {
    it->second->used_call = g_call;
    return *it->second;
  }
  if (ds.plans.size() >= 64) {
    for (size_t k = 0; k < ds.order.size(); ++k) {
      auto victim = ds.plans.find(ds.order[k]);
      if (victim->second->used_call == g_call) continue;   // referenced by this call
      drop_graphs(ds);
      ++ds.plan_gen;
      ds.plans.erase(victim);
      ds.order.erase(ds.order.begin() + (std::ptrdiff_t)k);
      break;
    }
  }
  auto P = std::make_unique<Plan>();
  build(*P);
  P->used_call = g_call;
  Plan& ref = *P;
  ds.plans.emplace(key, std::move(P));
  ds.order.push_back(key);
  return ref;
}

static void build_fd_plan(Plan& P, const cutqc_problem* p) {
  P.n_out = p->n_qubits;
  P.K = p->n_cuts;
  P.dtype = p->dtype;
  for (int c = 0; c < p->n_sub; ++c) {
    const cutqc_subcircuit& s = p->sub[c];
    Node nd;
    nd.orig = c;
    for (int j = 0; j < s.k_in; ++j) nd.cuts.push_back(s.in_cut[j]);
    for (int j = 0; j < s.k_out; ++j) nd.cuts.push_back(s.out_cut[j]);
    for (int i = 0; i < s.n_eff; ++i) nd.bits.push_back(s.out_qubit[i]);
    P.nodes.push_back(nd);
  }
  plan_contractions(P, p->n_cuts);
  finalize_plan(P);
}

// Adjoint plan for subcircuit c of a circuit cut into more than two
// subcircuits: every other subcircuit merged into one group node R by the
// same greedy group builds as the forward plan (recomputed, never stored
// between calls), then the pair (c, R) as the last step, whose row pairs and
// deposit tables the adjoint contraction of G against R uses.  Every cut of c
// joins it to R, so each row of c and of R appears in exactly one term.
static void build_bwd_plan(Plan& P, const cutqc_problem* p, int csub) {
  P.n_out = p->n_qubits;
  P.K = p->n_cuts;
  P.dtype = p->dtype;
  for (int c = 0; c < p->n_sub; ++c) {
    const cutqc_subcircuit& s = p->sub[c];
    Node nd;
    nd.orig = c;
    for (int j = 0; j < s.k_in; ++j) nd.cuts.push_back(s.in_cut[j]);
    for (int j = 0; j < s.k_out; ++j) nd.cuts.push_back(s.out_cut[j]);
    for (int i = 0; i < s.n_eff; ++i) nd.bits.push_back(s.out_qubit[i]);
    P.nodes.push_back(nd);
  }
  std::vector<int> live;
  for (int c = 0; c < p->n_sub; ++c)
    if (c != csub) live.push_back(c);
  while (live.size() > 1) merge_best_pair(P, live, p->n_cuts);
  P.steps.push_back(make_step(P, csub, live[0], -1, {}, p->n_cuts));
  finalize_plan(P);
}

// Run a plan.  `tensor(i)` gives the device pointer of original node i.
void plan_pair_host(const cutqc_problem* p, PairPlanHost& out) {
  validate(p, true);
  if (p->n_sub != 2) fail(CUTQC_ERR_UNSUPPORTED, "this entry point takes exactly two subcircuits");
  if (p->n_qubits > kMaxFD) fail(CUTQC_ERR_UNSUPPORTED, "full definition needs n_qubits <= 34");
  Plan P;
  P.n_out = p->n_qubits;
  P.K = p->n_cuts;
  P.dtype = p->dtype;
  for (int c = 0; c < 2; ++c) {
    const cutqc_subcircuit& s = p->sub[c];
    Node nd;
    nd.orig = c;
    for (int j = 0; j < s.k_in; ++j) nd.cuts.push_back(s.in_cut[j]);
    for (int j = 0; j < s.k_out; ++j) nd.cuts.push_back(s.out_cut[j]);
    for (int i = 0; i < s.n_eff; ++i) nd.bits.push_back(s.out_qubit[i]);
    P.nodes.push_back(nd);
  }
  plan_contractions(P, p->n_cuts);
  const Step& st = P.steps.back();
  out.fA = P.nodes[st.a].f();
  out.fB = P.nodes[st.b].f();
  out.kmax = st.kmax;
  out.vecB = st.vecB;
  out.sub_a = P.nodes[st.a].orig;
  out.sub_b = P.nodes[st.b].orig;
  out.K = p->n_cuts;
  out.rowsA = (int)P.nodes[st.a].rows();
  out.rowsB = (int)P.nodes[st.b].rows();
  out.rows = st.rows;
  out.depA = st.depA;
  out.depB = st.depB;
}

// Dynamic-definition plan: one node per subcircuit holding its merged tensor
// (rows x 2^#active outputs of the subcircuit), output positions = the bin
// ranks of the active qubits (lowest-numbered active qubit = most significant).
static void build_dd_plan(Plan& P, const cutqc_problem* p, const int8_t* role) {
  std::vector<int> rank(p->n_qubits, -1);
  int na = 0;
  for (int q = 0; q < p->n_qubits; ++q)
    if (role[q] == 0) rank[q] = na++;
  P.n_out = na;
  P.K = p->n_cuts;
  P.dtype = p->dtype;
  const size_t es = dtype_size(p->dtype);
  size_t front = 0;
  for (int c = 0; c < p->n_sub; ++c) {
    const cutqc_subcircuit& s = p->sub[c];
    DdSubPlan d;
    d.f = s.n_eff;
    d.rows = int64_t(1) << (2 * (s.k_in + s.k_out));
    std::vector<uint64_t> act_val, mrg_val;
    Node nd;
    nd.orig = c;
    for (int j = 0; j < s.k_in; ++j) nd.cuts.push_back(s.in_cut[j]);
    for (int j = 0; j < s.k_out; ++j) nd.cuts.push_back(s.out_cut[j]);
    for (int j = 0; j < s.n_eff; ++j) {
      const int q = s.out_qubit[j];
      const uint64_t xbit = uint64_t(1) << (s.n_eff - 1 - j);
      if (role[q] == 0) {
        act_val.push_back(xbit);
        d.act_rank.push_back(rank[q]);
        nd.bits.push_back(rank[q]);
      } else if (role[q] == 1) {
        mrg_val.push_back(xbit);
      } else if (role[q] == 3) {
        d.zoom |= xbit;
      }
    }
    d.a = (int)act_val.size();
    d.mg = (int)mrg_val.size();
    // index bit i (least significant first) of xa / xm is the (count-1-i)-th listed output
    std::reverse(act_val.begin(), act_val.end());
    std::reverse(mrg_val.begin(), mrg_val.end());
    d.depAct = deposit_table(act_val);
    d.depMrg = deposit_table(mrg_val);
    d.cuts = nd.cuts;
    // merged outputs exactly on the lowest x index bits 0 .. mg-1?
    {
      uint64_t mm = 0;
      for (uint64_t v : mrg_val) mm |= v;
      d.run = d.mg > 0 && mm == ((uint64_t(1) << d.mg) - 1);
      uint64_t am = 0;
      for (uint64_t v : act_val) am |= v;
      d.dense = d.run && am == (((uint64_t(1) << d.a) - 1) << d.mg);
      d.blk = d.run ? 0 : dd_merge_block(mm, d.mg, am, d.zoom);
    }
    d.ws_merged = front;
    front = align_up(front + (size_t)d.rows * ((size_t)1 << d.a) * es);
    d.ws_mc = front;
    if (p->dtype == CUTQC_F32) front = align_up(front + (size_t)d.rows * ((size_t)1 << d.a) * 4);
    d.ws_part = front;
    if (d.run) front = align_up(front + ((size_t)d.rows << (d.a + dd_merge_chunks(d.rows, d.a, d.mg))) * 8);
    P.dd.push_back(d);
    P.nodes.push_back(nd);
  }
  P.dd_front = front;
  plan_contractions(P, p->n_cuts);
  finalize_plan(P);
  size_t off = 0;
  for (DdSubPlan& d : P.dd) {
    d.off_act = off;
    off = align_up(off + d.depAct.size() * 8);
    d.off_mrg = off;
    off = align_up(off + d.depMrg.size() * 8);
  }
  CUTQC_CUDA(cudaMalloc(&P.ddtab, std::max<size_t>(off, 256)));
  std::vector<char> host(std::max<size_t>(off, 256), 0);
  for (DdSubPlan& d : P.dd) {
    std::memcpy(host.data() + d.off_act, d.depAct.data(), d.depAct.size() * 8);
    std::memcpy(host.data() + d.off_mrg, d.depMrg.data(), d.depMrg.size() * 8);
  }
  CUTQC_CUDA(cudaMemcpy(P.ddtab, host.data(), host.size(), cudaMemcpyHostToDevice));
}

// Run a plan.  The workspace holds [front | the plan's own buffers | back];
// `pre(front_ptr)` is called once the workspace exists and returns the device
// tensors of the plan's original nodes.  Returns a pointer to the back region.
// Output of a full-definition call: device (or managed) memory of the current
// device, or pinned host memory mapped into the device's address space; the
// kernels then write the probabilities straight into host memory over the
// host link, and the device alias of the buffer is what they are given.
// Unregistered host memory and other devices' memory are rejected here,
// before anything is launched.
static void* resolve_out(void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    fail(CUTQC_ERR_ARG, "out is not a pointer CUDA knows");
  }
  int dev = 0;
  CUTQC_CUDA(cudaGetDevice(&dev));
  switch (at.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      if (at.type == cudaMemoryTypeDevice && at.device != dev) fail(CUTQC_ERR_ARG, "out is on another device");
      return p;
    case cudaMemoryTypeHost:
      if (!at.devicePointer) fail(CUTQC_ERR_ARG, "out is pinned host memory not mapped for the device");
      return at.devicePointer;
    default:
      fail(CUTQC_ERR_ARG, "out must be device memory or pinned (page-locked, mapped) host memory");
  }
}

static bool is_host_memory(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

void* resolve_device_out(void* p, bool* host) {
  *host = is_host_memory(p);
  return resolve_out(p);
}

bool is_device_memory_here(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = 0;
  CUTQC_CUDA(cudaGetDevice(&dev));
  return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

static char* run_plan(DeviceState& ds, Plan& P, size_t front, size_t back,
                      const std::function<std::vector<const void*>(char*)>& pre, void* out, double* sum, int algo,
                      cudaStream_t s, char* ws_given = nullptr, size_t* bytes_only = nullptr,
                      size_t topk_back_off = SIZE_MAX, int* topk_nlists = nullptr, bool groups_only = false,
                      char** base_out = nullptr, std::vector<Contraction>* defer_lowrank = nullptr) {
  // topk_back_off: where in the back region a tensor-core final contraction
  // may leave its fused top-32 lists (*topk_nlists of them; 0 when it did not).
  // groups_only: run the group builds but not the last step (the adjoint
  // reads the group tensors at *base_out + P.ws_node[...])
  if (topk_nlists) *topk_nlists = 0;
  size_t tc_ws = 0;
  std::vector<Contraction> cs(P.steps.size());
  char* base = nullptr;
  // the constant-one node
  if (!ds.one) {
    CUTQC_CUDA(cudaMalloc(&ds.one, 16));
    const double one64 = 1.0;
    const float one32 = 1.0f;
    CUTQC_CUDA(cudaMemcpy(ds.one, &one64, 8, cudaMemcpyHostToDevice));
    CUTQC_CUDA(cudaMemcpy(static_cast<char*>(ds.one) + 8, &one32, 4, cudaMemcpyHostToDevice));
  }
  const void* one = P.dtype == CUTQC_F64 ? ds.one : static_cast<char*>(ds.one) + 8;
  for (size_t i = 0; i < P.steps.size(); ++i) {
    Contraction& c = cs[i];
    const Step& st = P.steps[i];
    c.fA = P.nodes[st.a].f();
    c.fB = P.nodes[st.b].f();
    c.batch = st.batch;
    c.kmax = st.kmax;
    c.out_batch_stride = st.out_stride;
    c.vecB = st.vecB;
    c.dtype = P.dtype;
    c.scale = (i + 1 == P.steps.size()) ? std::ldexp(1.0, -P.K) : 1.0;
    c.rowsA = (int)P.nodes[st.a].rows();
    c.rowsB = (int)P.nodes[st.b].rows();
  }
  // decide the algorithm of the final step: under CUTQC_AUTO a contraction
  // of at most 16 kept terms takes the streaming CUDA-core form (its output
  // stream is all the work; measured faster than the tensor-core form) unless
  // the caller wants the top bins, which the tensor-core epilogue keeps while
  // writing them (a separate scan of 2^30 bins costs more); the rest of FP32
  // the tensor-core form where the shape allows it
  const bool want_topk = topk_nlists && topk_back_off != SIZE_MAX;
  int final_algo = algo;
  if (final_algo == CUTQC_AUTO)
    final_algo = (P.dtype == CUTQC_F32 && (!lowrank_eligible(cs.back()) || want_topk)) ? CUTQC_TC_BF16X3 : CUTQC_CC;
  if (algo == CUTQC_AUTO && final_algo == CUTQC_CC) algo = CUTQC_CC;
  const bool tc_algo = final_algo == CUTQC_TC_BF16X3 || final_algo == CUTQC_TC_BF16X6 || final_algo == CUTQC_TC_TF32X3;
  if (tc_algo && P.dtype != CUTQC_F32) fail(CUTQC_ERR_ARG, "the tensor-core forms need FP32 tensors");
  size_t need = P.ws_bytes;
  const bool use_tc_final = tc_algo && tc_supported(cs.back());
  if (use_tc_final) {
    tc_ws = tc_workspace_bytes(cs.back());
    need = align_up(need) + tc_ws;
  }
  front = align_up(front);
  need = align_up(need);
  if (bytes_only) {
    *bytes_only = front + need + align_up(back);
    return nullptr;
  }
  char* ws = ws_given ? ws_given : static_cast<char*>(workspace(ds, front + need + back));
  base = ws + front;
  if (base_out) *base_out = base;
  const std::vector<const void*> orig_tensor = pre(ws);
  auto node_ptr = [&](int i) -> const void* {
    const Node& nd = P.nodes[i];
    if (nd.orig >= 0) return orig_tensor[nd.orig];
    if (nd.orig == -2) return one;
    return base + P.ws_node[i];
  };
  auto dtab = static_cast<char*>(P.dtab);
  // row flags and max |.| of each step's operands, both in one launch
  std::vector<int> flagged(P.nodes.size(), 0);
  auto ensure_flags = [&](int ia, int ib, const CompactJob* cj = nullptr) {
    RowStatsJobs j{};
    if (cj) j.cj = *cj;
    for (int i : {ia, ib}) {
      if (flagged[i]) continue;
      flagged[i] = 1;
      const Node& nd = P.nodes[i];
      j.t[j.n] = node_ptr(i);
      j.rows[j.n] = nd.rows();
      j.cols[j.n] = int64_t(1) << nd.f();
      j.flags[j.n] = reinterpret_cast<int32_t*>(base + P.ws_nz[i]);
      j.rmax[j.n] = reinterpret_cast<float*>(base + P.ws_rmax[i]);
      ++j.n;
    }
    if (j.n) launch_row_stats(j, P.dtype, s);
    else if (cj) fail(CUTQC_ERR_CUDA, "compaction job without a row-statistics launch");
  };
  for (size_t i = 0; i < P.steps.size(); ++i) {
    const Step& st = P.steps[i];
    Contraction& c = cs[i];
    const bool last_step = (i + 1 == P.steps.size());
    if (last_step && groups_only) break;
    if (last_step && !use_tc_final && defer_lowrank && lowrank_eligible(c) && !flagged[st.a] && !flagged[st.b] &&
        !is_host_memory(out)) {
      // a low-rank CUDA-core final contraction: its row statistics, its
      // compaction and the contraction run in the caller's one launch over
      // every such problem of a batch
      flagged[st.a] = flagged[st.b] = 1;
      c.A = node_ptr(st.a);
      c.B = node_ptr(st.b);
      c.rows = reinterpret_cast<const int32_t*>(dtab + st.off_rows);
      c.depA = reinterpret_cast<const uint64_t*>(dtab + st.off_depA);
      c.depB = reinterpret_cast<const uint64_t*>(dtab + st.off_depB);
      c.crow = reinterpret_cast<int32_t*>(base + st.ws_crow);
      c.kcount = reinterpret_cast<int32_t*>(base + st.ws_kcount);
      c.nzA = reinterpret_cast<const int32_t*>(base + P.ws_nz[st.a]);
      c.nzB = reinterpret_cast<const int32_t*>(base + P.ws_nz[st.b]);
      c.rmaxA = reinterpret_cast<const float*>(base + P.ws_rmax[st.a]);
      c.rmaxB = reinterpret_cast<const float*>(base + P.ws_rmax[st.b]);
      c.status = status_word(ds);
      c.out = out;
      c.sum = sum;
      defer_lowrank->push_back(c);
      g_last_algo = CUTQC_CC;
      break;
    }
    const bool both_new = !flagged[st.a] || !flagged[st.b];
    TcFusedStats fstats{};
    bool fused_stats = false;
    if (last_step && use_tc_final && !flagged[st.a] && !flagged[st.b] && st.kmax <= 4096) {
      // the row statistics of both operands run inside the operand preparation
      flagged[st.a] = flagged[st.b] = 1;
      fstats.nzA = reinterpret_cast<int32_t*>(base + P.ws_nz[st.a]);
      fstats.nzB = reinterpret_cast<int32_t*>(base + P.ws_nz[st.b]);
      fstats.rmaxA = reinterpret_cast<float*>(base + P.ws_rmax[st.a]);
      fstats.rmaxB = reinterpret_cast<float*>(base + P.ws_rmax[st.b]);
      fstats.barrier = reinterpret_cast<unsigned*>(base + st.ws_counter);
      fstats.look = reinterpret_cast<unsigned*>(base + st.ws_look);
      fused_stats = true;
    } else if (last_step && use_tc_final && both_new && st.kmax <= 4096) {
      // the last row-statistics block compacts the terms and picks the split
      CompactJob cj;
      cj.active = 1;
      cj.rows = reinterpret_cast<const int32_t*>(dtab + st.off_rows);
      cj.kmax = st.kmax;
      cj.nzA = reinterpret_cast<const int32_t*>(base + P.ws_nz[st.a]);
      cj.nzB = reinterpret_cast<const int32_t*>(base + P.ws_nz[st.b]);
      cj.rmaxA = reinterpret_cast<const float*>(base + P.ws_rmax[st.a]);
      cj.rmaxB = reinterpret_cast<const float*>(base + P.ws_rmax[st.b]);
      cj.crow = reinterpret_cast<int32_t*>(base + st.ws_crow);
      cj.kcount = reinterpret_cast<int32_t*>(base + st.ws_kcount);
      cj.scale = c.scale;
      cj.bound = reinterpret_cast<double*>(base + st.ws_bound);
      cj.nseg = reinterpret_cast<int32_t*>(base + st.ws_nseg);
      cj.nseg_fixed = (algo == CUTQC_TC_BF16X3 || algo == CUTQC_TC_TF32X3) ? 3 : (algo == CUTQC_TC_BF16X6 ? 6 : 0);
      cj.sum_zero = sum;
      cj.counter = reinterpret_cast<unsigned*>(base + st.ws_counter);
      CUTQC_CUDA(cudaMemsetAsync(cj.counter, 0, sizeof(unsigned), s));
      ensure_flags(st.a, st.b, &cj);
      c.compacted = true;
    } else {
      ensure_flags(st.a, st.b);
    }
    c.A = node_ptr(st.a);
    c.B = node_ptr(st.b);
    c.rows = reinterpret_cast<const int32_t*>(dtab + st.off_rows);
    c.depA = reinterpret_cast<const uint64_t*>(dtab + st.off_depA);
    c.depB = reinterpret_cast<const uint64_t*>(dtab + st.off_depB);
    c.crow = reinterpret_cast<int32_t*>(base + st.ws_crow);
    c.kcount = reinterpret_cast<int32_t*>(base + st.ws_kcount);
    c.nzA = reinterpret_cast<const int32_t*>(base + P.ws_nz[st.a]);
    c.nzB = reinterpret_cast<const int32_t*>(base + P.ws_nz[st.b]);
    const bool final_step = last_step;
    if (final_step && use_tc_final) {
      c.rmaxA = reinterpret_cast<const float*>(base + P.ws_rmax[st.a]);
      c.rmaxB = reinterpret_cast<const float*>(base + P.ws_rmax[st.b]);
      c.bound = reinterpret_cast<double*>(base + st.ws_bound);
      c.nseg = reinterpret_cast<int32_t*>(base + st.ws_nseg);
      c.nseg_fixed = (algo == CUTQC_TC_BF16X3 || algo == CUTQC_TC_TF32X3) ? 3 : (algo == CUTQC_TC_BF16X6 ? 6 : 0);
      c.tf32 = algo == CUTQC_TC_TF32X3;
      g_last_nseg = c.nseg;
      g_last_bound = c.bound;
      g_last_stream = s;
    }
    c.status = status_word(ds);
    if (final_step && use_tc_final && topk_nlists && topk_back_off != SIZE_MAX) {
      char* tk = base + need + topk_back_off;
      c.topk_v = reinterpret_cast<float*>(tk);
      c.topk_i = reinterpret_cast<int64_t*>(tk + (size_t)152 * 8 * 4 * 32 * 4);
      c.topk_nlists = topk_nlists;
    }
    c.out = final_step ? out : static_cast<void*>(base + P.ws_node[st.result]);
    c.out_host = final_step && is_host_memory(out);
    c.sum = final_step ? sum : nullptr;
    c.profile = final_step;
    if (!(final_step && use_tc_final)) {
      c.sum_zero = c.sum;
      launch_compact(c, s);   // the tensor-core path compacts inside its operand preparation
    }
    if (final_step && use_tc_final)
      launch_tc_bf16x3(c, base + align_up(P.ws_bytes), tc_ws, s, fused_stats ? &fstats : nullptr);
    else if (final_step && lowrank_eligible(c))
      launch_lowrank(c, s);
    else
      launch_cc_gemm(c, s);
    if (final_step) g_last_algo = use_tc_final ? (algo == CUTQC_AUTO ? CUTQC_TC_BF16X3 : algo) : CUTQC_CC;
  }
  return base + need;
}

// Autotuning cache: the measured final form (CUTQC_CC or CUTQC_AUTO, the
// tensor-core path) per problem structure, kept for the process and, when
// the environment variable CUTQC_AUTOTUNE_CACHE names a file, read from it on
// first use and appended to after each new measurement (one "form key" line
// per structure, keys prefixed by the device's name and SM count).
static std::unordered_map<std::string, int> g_tuned;
static bool g_tuned_loaded = false;

static std::string device_tag() {
  int dev = 0;
  CUTQC_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp pr{};
  CUTQC_CUDA(cudaGetDeviceProperties(&pr, dev));
  std::string name(pr.name);
  for (char& ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  return name + "/" + std::to_string(pr.multiProcessorCount);
}

static int autotune_lookup(const std::string& key) {
  if (!g_tuned_loaded) {
    g_tuned_loaded = true;
    if (const char* path = std::getenv("CUTQC_AUTOTUNE_CACHE")) {
      if (FILE* f = std::fopen(path, "r")) {
        char buf[8192];
        while (std::fgets(buf, sizeof buf, f)) {
          std::string line(buf);
          while (!line.empty() && (line.back() == '\n' || line.back() == '\r')) line.pop_back();
          const size_t sp = line.find(' ');
          if (sp == std::string::npos) continue;
          const int form = std::atoi(line.substr(0, sp).c_str());
          if (form == CUTQC_CC || form == CUTQC_AUTO) g_tuned[line.substr(sp + 1)] = form;
        }
        std::fclose(f);
      }
    }
  }
  auto it = g_tuned.find(device_tag() + "|" + key);
  return it == g_tuned.end() ? -1 : it->second;
}

static void autotune_store(const std::string& key, int form) {
  const std::string full = device_tag() + "|" + key;
  g_tuned[full] = form;
  if (const char* path = std::getenv("CUTQC_AUTOTUNE_CACHE")) {
    if (FILE* f = std::fopen(path, "a")) {
      std::fprintf(f, "%d %s\n", form, full.c_str());
      std::fclose(f);
    }
  }
}

// Batched full definition.  Every problem gets its own region of the
// workspace, so problems are independent and run on parallel stream branches.
// The first call with a given set of shapes and pointers runs eagerly (and,
// under CUTQC_AUTO with FP32 tensors, times the CUDA-core and tensor-core
// forms of each problem's final contraction once and keeps the faster); the
// call is then captured into a CUDA graph that later identical calls replay
// with a single launch.
// The raw arguments of a batched call (every field and array the plans,
// work lists and graph depend on, and every pointer): identical calls map to
// the same captured graph without rebuilding plan keys and sizes.
static std::string batch_signature(const cutqc_problem* problems, int n, void* const* out, int algo,
                                   const double* sum_p) {
  std::string sig;
  auto put = [&](const void* p, size_t bytes) { sig.append(static_cast<const char*>(p), bytes); };
  put(&algo, sizeof algo);
  put(&n, sizeof n);
  put(&sum_p, sizeof sum_p);
  for (int i = 0; i < n; ++i) {
    const cutqc_problem& p = problems[i];
    put(&p.n_qubits, sizeof p.n_qubits);
    put(&p.n_cuts, sizeof p.n_cuts);
    put(&p.n_sub, sizeof p.n_sub);
    put(&p.dtype, sizeof p.dtype);
    for (int c = 0; c < p.n_sub; ++c) {
      const cutqc_subcircuit& sc = p.sub[c];
      put(&sc.k_in, sizeof sc.k_in);
      put(&sc.k_out, sizeof sc.k_out);
      put(&sc.n_eff, sizeof sc.n_eff);
      put(sc.in_cut, sizeof(int32_t) * (size_t)sc.k_in);
      put(sc.out_cut, sizeof(int32_t) * (size_t)sc.k_out);
      put(sc.out_qubit, sizeof(int32_t) * (size_t)sc.n_eff);
      put(&sc.tensor, sizeof sc.tensor);
    }
    put(&out[i], sizeof out[i]);
  }
  return sig;
}

static void run_batch(DeviceState& ds, const cutqc_problem* problems, int n, void* const* out, int algo,
                      double* sum_p, cudaStream_t s) {
  // a call identical to an earlier one whose graph, workspace and plans
  // still stand: replay its graph
  const std::string sig = batch_signature(problems, n, out, algo, sum_p);
  {
    auto f = ds.batch_fast.find(sig);
    if (f != ds.batch_fast.end() && f->second.ws_gen == ds.ws_gen && f->second.plan_gen == ds.plan_gen) {
      auto g = ds.graphs.find(f->second.gk);
      if (g != ds.graphs.end() && g->second.gen == ds.ws_gen) {
        CUTQC_CUDA(cudaGraphLaunch(g->second.exec, s));
        return;
      }
    }
  }
  std::vector<Plan*> plans(n);
  std::string key;
  put_int(key, algo);
  key += '#';
  auto put_ptr = [&](const void* p) {
    char buf[24];
    const auto r = std::to_chars(buf, buf + sizeof buf, (unsigned long long)(uintptr_t)p, 16);
    key.append(buf, r.ptr);
  };
  for (int i = 0; i < n; ++i) {
    const cutqc_problem* p = &problems[i];
    const std::string k = fd_key(p, 0, nullptr, 0);
    plans[i] = &get_plan(ds, k, [&](Plan& P) { build_fd_plan(P, p); });
    key += k;
    key += '@';
    for (int c = 0; c < p->n_sub; ++c) {
      put_ptr(p->sub[c].tensor);
      key += ',';
    }
    put_ptr(out[i]);
    key += ',';
    put_ptr(sum_p ? (const void*)(sum_p + i) : nullptr);
    key += ';';
  }
  auto tensors_of = [](const cutqc_problem* p) {
    return [p](char*) {
      std::vector<const void*> t(p->n_sub);
      for (int c = 0; c < p->n_sub; ++c) t[c] = p->sub[c].tensor;
      return t;
    };
  };
  // autotune the final form once per plan (eager, outside any capture); a
  // choice measured before (this process, or a cache file named by
  // CUTQC_AUTOTUNE_CACHE) is reused
  for (int i = 0; i < n; ++i) {
    Plan& P = *plans[i];
    if (algo != CUTQC_AUTO || P.dtype != CUTQC_F32 || P.tuned >= 0) continue;
    const std::string tkey = fd_key(&problems[i], 0, nullptr, 0);
    const int cached = autotune_lookup(tkey);
    if (cached >= 0) {
      P.tuned = cached;
      continue;
    }
    cudaEvent_t e0, e1;
    CUTQC_CUDA(cudaEventCreate(&e0));
    CUTQC_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int choice = CUTQC_CC;
    for (int form : {CUTQC_CC, CUTQC_TC_BF16X3}) {
      float t = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        CUTQC_CUDA(cudaEventRecord(e0, s));
        run_plan(ds, P, 0, 0, tensors_of(&problems[i]), out[i], sum_p ? sum_p + i : nullptr,
                 form == CUTQC_TC_BF16X3 ? CUTQC_AUTO : form, s);
        CUTQC_CUDA(cudaEventRecord(e1, s));
        CUTQC_CUDA(cudaEventSynchronize(e1));
        CUTQC_CUDA(cudaEventElapsedTime(&t, e0, e1));
      }
      if (g_last_algo == CUTQC_CC && form != CUTQC_CC) t = 1e30f;   // the shape has no tensor-core form
      if (t < best) {
        best = t;
        choice = form;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    P.tuned = choice == CUTQC_CC ? CUTQC_CC : CUTQC_AUTO;
    autotune_store(tkey, P.tuned);
  }
  // workspace regions
  std::vector<size_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    size_t b = 0;
    int a = algo;
    if (a == CUTQC_AUTO && plans[i]->tuned == CUTQC_CC) a = CUTQC_CC;
    run_plan(ds, *plans[i], 0, 0, tensors_of(&problems[i]), out[i], nullptr, a, s, nullptr, &b);
    off[i + 1] = off[i] + align_up(b);
  }
  char* ws = static_cast<char*>(workspace(ds, off[n]));
  key += "|gen";
  put_int(key, (long long)ds.ws_gen);
  const std::string gk = key;
  auto it = ds.graphs.find(gk);
  if (it != ds.graphs.end() && it->second.gen == ds.ws_gen) {
    if (ds.batch_fast.size() >= 64) ds.batch_fast.clear();
    ds.batch_fast[sig] = DeviceState::BatchFast{gk, ds.ws_gen, ds.plan_gen};
    CUTQC_CUDA(cudaGraphLaunch(it->second.exec, s));
    return;
  }
  auto algo_of = [&](int i) {
    return (algo == CUTQC_AUTO && plans[i]->tuned == CUTQC_CC) ? (int)CUTQC_CC : algo;
  };
  // Low-rank CUDA-core final contractions are not launched per problem: they
  // are collected (per dtype) and run as one launch over a device work list.
  std::vector<Contraction> lr[2];
  auto launch_deferred = [&](cudaStream_t st, const char* group) {
    for (int d = 0; d < 2; ++d) {
      if (lr[d].empty()) continue;
      const std::string tk = gk + "#lr" + group + std::to_string(d);
      std::vector<char> host;
      int64_t items = 0;
      lowrank_batch_tables(lr[d], host, &items);
      auto it2 = ds.lr_tables.find(tk);
      if (it2 == ds.lr_tables.end()) {
        // first (eager) call: upload the work list; captured replays reuse it
        void* dev = nullptr;
        CUTQC_CUDA(cudaMalloc(&dev, host.size()));
        CUTQC_CUDA(cudaMemcpy(dev, host.data(), host.size(), cudaMemcpyHostToDevice));
        it2 = ds.lr_tables.emplace(tk, dev).first;
      }
      launch_lowrank_batch(it2->second, lr[d], items, st);
      lr[d].clear();
    }
  };
  auto run_one = [&](int i, cudaStream_t st, char* w, bool defer) {
    std::vector<Contraction> d;
    run_plan(ds, *plans[i], 0, 0, tensors_of(&problems[i]), out[i], sum_p ? sum_p + i : nullptr, algo_of(i), st, w,
             nullptr, SIZE_MAX, nullptr, false, nullptr, defer ? &d : nullptr);
    for (const Contraction& c : d) lr[c.dtype == CUTQC_F64 ? 1 : 0].push_back(c);
  };
  // the problems whose final contraction is deferred into the batched
  // low-rank launches (the same decision run_plan takes), and the rest
  std::vector<int> direct;
  std::vector<char> is_deferred(n, 0);
  for (int i = 0; i < n; ++i) {
    const Plan& P = *plans[i];
    const Step& st = P.steps.back();
    Contraction c;
    c.batch = st.batch;
    c.kmax = st.kmax;
    c.fA = P.nodes[st.a].f();
    c.fB = P.nodes[st.b].f();
    c.vecB = st.vecB;
    c.dtype = P.dtype;
    const int a = algo_of(i);
    const bool cc_final = a == CUTQC_CC || (a == CUTQC_AUTO && (lowrank_eligible(c) || P.dtype != CUTQC_F32)) ||
                          !tc_supported(c);
    const bool defer = cc_final && lowrank_eligible(c) && !is_host_memory(out[i]);
    // a deferred problem without group builds launches nothing of its own
    if (defer && P.steps.size() == 1)
      direct.push_back(i);
    else
      is_deferred[i] = defer;
  }
  // the other problems over the side branches, largest output first onto
  // the least loaded branch; each branch runs its deferred problems' group
  // builds, then one batched low-rank launch of their final contractions,
  // then its other problems, so no branch waits for another's group builds
  // (the large low-rank launches of different branches, of different term
  // classes, then run beside each other and beside the short launches)
  std::vector<int> rest;
  for (int i = 0; i < n; ++i)
    if (std::find(direct.begin(), direct.end(), i) == direct.end()) rest.push_back(i);
  std::stable_sort(rest.begin(), rest.end(), [&](int x, int y) { return plans[x]->n_out > plans[y]->n_out; });
  std::vector<std::vector<int>> on(kBranches);
  std::vector<double> load(kBranches, 0.0);
  for (int i : rest) {
    int bmin = 1;
    for (int b = 2; b < kBranches; ++b)
      if (load[b] < load[bmin]) bmin = b;
    on[bmin].push_back(i);
    load[bmin] += std::ldexp(1.0, plans[i]->n_out);
  }
  auto run_branch = [&](int b, cudaStream_t st) {
    for (int i : on[b])
      if (is_deferred[i]) run_one(i, st, ws + off[i], true);
    launch_deferred(st, ("b" + std::to_string(b)).c_str());
    for (int i : on[b])
      if (!is_deferred[i]) run_one(i, st, ws + off[i], false);
  };
  // eager run of the whole batch on the caller's stream (it also uploads the
  // work lists that the captured launches reuse)
  for (int i : direct) run_one(i, s, ws + off[i], true);
  launch_deferred(s, "a");
  for (int b = 1; b < kBranches; ++b) run_branch(b, s);
  // capture the same launches over parallel branches for later calls
  if (!ds.fork) {
    for (int b = 0; b < kBranches; ++b) {
      CUTQC_CUDA(cudaStreamCreateWithFlags(&ds.branch[b], cudaStreamNonBlocking));
      CUTQC_CUDA(cudaEventCreateWithFlags(&ds.join[b], cudaEventDisableTiming));
      CUTQC_CUDA(cudaEventCreateWithFlags(&ds.mid[b], cudaEventDisableTiming));
    }
    CUTQC_CUDA(cudaEventCreateWithFlags(&ds.fork, cudaEventDisableTiming));
  }
  cudaGraph_t graph = nullptr;
  g_capturing = true;
  try {
    CUTQC_CUDA(cudaStreamBeginCapture(ds.branch[0], cudaStreamCaptureModeThreadLocal));
    CUTQC_CUDA(cudaEventRecord(ds.fork, ds.branch[0]));
    for (int b = 1; b < kBranches; ++b) CUTQC_CUDA(cudaStreamWaitEvent(ds.branch[b], ds.fork, 0));
    // branch 0: the batched low-rank launch of the problems without group
    // builds, at once; branches 1..: the rest, beside it
    for (int i : direct) run_one(i, ds.branch[0], ws + off[i], true);
    launch_deferred(ds.branch[0], "a");
    for (int b = 1; b < kBranches; ++b) run_branch(b, ds.branch[b]);
    for (int b = 1; b < kBranches; ++b) {
      CUTQC_CUDA(cudaEventRecord(ds.join[b], ds.branch[b]));
      CUTQC_CUDA(cudaStreamWaitEvent(ds.branch[0], ds.join[b], 0));
    }
    CUTQC_CUDA(cudaStreamEndCapture(ds.branch[0], &graph));
  } catch (...) {
    g_capturing = false;
    cudaGraph_t g2 = nullptr;
    cudaStreamEndCapture(ds.branch[0], &g2);
    if (g2) cudaGraphDestroy(g2);
    throw;
  }
  g_capturing = false;
  GraphEntry e;
  e.gen = ds.ws_gen;
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  CUTQC_CUDA(ie);
  if (ds.graphs.size() >= 16) drop_graphs(ds);
  ds.graphs[gk] = e;
}

// The pre-step of a dynamic-definition plan: merge every subcircuit's tensor
// over its merged outputs with the zoomed outputs fixed (Algorithm 1), into
// the front region of the workspace; returns the merged tensors.
static std::function<std::vector<const void*>(char*)> dd_merge_pre(const Plan& P, const cutqc_problem* p,
                                                                   cudaStream_t s, char** front_out) {
  return [&P, p, s, front_out](char* front) {
    if (front_out) *front_out = front;
    char* ddtab = static_cast<char*>(P.ddtab);
    std::vector<const void*> t(p->n_sub);
    for (int c = 0; c < p->n_sub; ++c) {
      const DdSubPlan& d = P.dd[c];
      launch_dd_merge(p->sub[c].tensor, P.dtype, d.rows, d.f, d.a, d.mg,
                      reinterpret_cast<const uint64_t*>(ddtab + d.off_act),
                      reinterpret_cast<const uint64_t*>(ddtab + d.off_mrg), d.zoom, d.run, d.dense,
                      front + d.ws_merged, reinterpret_cast<float*>(front + d.ws_mc), front + d.ws_part, s, d.blk);
      t[c] = front + d.ws_merged;
    }
    return t;
  };
}

}  // namespace cutqc

using namespace cutqc;

extern "C" {

int cutqc_reconstruct_fd(const cutqc_problem* problems, int32_t n_problems, void* const* out, int32_t algo,
                         double* sum_p, void* stream) {
  return guarded([&] {
    if (!problems || n_problems < 1) fail(CUTQC_ERR_ARG, "need n_problems >= 1 problems");
    if (!out) fail(CUTQC_ERR_ARG, "out is NULL");
    if (algo < CUTQC_AUTO || algo > CUTQC_TC_TF32X3) fail(CUTQC_ERR_ARG, "unknown algo");
    for (int i = 0; i < n_problems; ++i) {
      validate(&problems[i], true);
      if (problems[i].n_qubits > kMaxFD) fail(CUTQC_ERR_UNSUPPORTED, "full definition needs n_qubits <= 34");
      if (!out[i]) fail(CUTQC_ERR_ARG, "out[i] is NULL");
      need_aligned(out[i], 16, "out[i]");
    }
    need_aligned(sum_p, 8, "sum_p");
    std::vector<void*> dout(n_problems);
    for (int i = 0; i < n_problems; ++i) dout[i] = resolve_out(out[i]);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceState& ds = device_state();
    auto tensors_of = [&](const cutqc_problem* p) {
      return [p](char*) {
        std::vector<const void*> t(p->n_sub);
        for (int c = 0; c < p->n_sub; ++c) t[c] = p->sub[c].tensor;
        return t;
      };
    };
    if (n_problems == 1) {
      const cutqc_problem* p = &problems[0];
      Plan& P = get_plan(ds, fd_key(p, 0, nullptr, 0), [&](Plan& P) { build_fd_plan(P, p); });
      run_plan(ds, P, 0, 0, tensors_of(p), dout[0], sum_p, algo, s);
      return;
    }
    run_batch(ds, problems, n_problems, dout.data(), algo, sum_p, s);
  });
}

int cutqc_reconstruct_fd_slab(const cutqc_problem* problem, int32_t slab_bits, int64_t slab_index, void* out,
                              int32_t algo, double* sum_p, void* stream) {
  return guarded([&] {
    validate(problem, true);
    const cutqc_problem* p = problem;
    if (p->n_qubits > kMaxFD) fail(CUTQC_ERR_UNSUPPORTED, "full definition needs n_qubits <= 34");
    if (slab_bits < 0 || slab_bits >= p->n_qubits) fail(CUTQC_ERR_ARG, "slab_bits must be in 0 .. n_qubits - 1");
    if (slab_index < 0 || slab_index >= (int64_t(1) << slab_bits)) fail(CUTQC_ERR_ARG, "slab_index out of range");
    if (algo < CUTQC_AUTO || algo > CUTQC_TC_TF32X3) fail(CUTQC_ERR_ARG, "unknown algo");
    if (!out) fail(CUTQC_ERR_ARG, "out is NULL");
    need_aligned(out, 16, "out");
    need_aligned(sum_p, 8, "sum_p");
    void* dout = resolve_out(out);
    // qubits 0 .. slab_bits-1 (the most significant output bits) fixed at the
    // slab's bits, the rest active: the recursion's bins are the slab
    std::vector<int8_t> role(p->n_qubits, 0);
    for (int q = 0; q < slab_bits; ++q) role[q] = (int8_t)(((slab_index >> (slab_bits - 1 - q)) & 1) ? 3 : 2);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceState& ds = device_state();
    Plan& P = get_plan(ds, fd_key(p, 1, role.data(), 0), [&](Plan& P) { build_dd_plan(P, p, role.data()); });
    run_plan(ds, P, P.dd_front, 0, dd_merge_pre(P, p, s, nullptr), dout, sum_p, algo, s);
  });
}

int cutqc_attribute(const void* variant_probs, int32_t d, int32_t k_in, const int32_t* meas_qubit, int32_t k_out,
                    const int32_t* out_local, int32_t n_eff, int32_t dtype, void* tensor, void* stream) {
  return guarded([&] {
    if (d < 1 || d > 30) fail(CUTQC_ERR_UNSUPPORTED, "attribution needs 1 <= d <= 30");
    if (k_in < 0 || k_out < 0 || n_eff < 0 || k_in + k_out > kMaxCuts) fail(CUTQC_ERR_SHAPE, "bad slot counts");
    if (k_out + n_eff != d) fail(CUTQC_ERR_SHAPE, "every local qubit must be an output or a measured cut qubit");
    if (!variant_probs || !tensor || (k_out && !meas_qubit) || (n_eff && !out_local)) fail(CUTQC_ERR_ARG, "NULL array");
    // the attribution kernels pick 16-byte or scalar accesses themselves
    need_aligned(variant_probs, dtype == CUTQC_F64 ? 8 : 4, "variant_probs");
    need_aligned(tensor, dtype == CUTQC_F64 ? 8 : 4, "tensor");
    if (dtype != CUTQC_F32 && dtype != CUTQC_F64) fail(CUTQC_ERR_ARG, "bad dtype");
    std::vector<int> seen(d, 0), mq(k_out), oq(n_eff);
    for (int j = 0; j < k_out; ++j) {
      if (meas_qubit[j] < 0 || meas_qubit[j] >= d || seen[meas_qubit[j]]++) fail(CUTQC_ERR_SHAPE, "bad measured qubit");
      mq[j] = meas_qubit[j];
    }
    for (int j = 0; j < n_eff; ++j) {
      if (out_local[j] < 0 || out_local[j] >= d || seen[out_local[j]]++) fail(CUTQC_ERR_SHAPE, "bad output qubit");
      oq[j] = out_local[j];
    }
    launch_attribute(variant_probs, dtype, d, k_in, mq.data(), k_out, oq.data(), n_eff, tensor,
                     static_cast<cudaStream_t>(stream));
  });
}

int cutqc_attribute_merged(const void* variant_probs, int32_t d, int32_t k_in, const int32_t* meas_qubit,
                           int32_t k_out, const int32_t* out_local, int32_t n_eff, const int8_t* role_out,
                           int32_t dtype, void* tensor, void* stream) {
  return guarded([&] {
    if (d < 1 || d > 30) fail(CUTQC_ERR_UNSUPPORTED, "attribution needs 1 <= d <= 30");
    if (k_in < 0 || k_out < 0 || n_eff < 0 || k_in + k_out > kMaxCuts) fail(CUTQC_ERR_SHAPE, "bad slot counts");
    if (k_out + n_eff != d) fail(CUTQC_ERR_SHAPE, "every local qubit must be an output or a measured cut qubit");
    if (!variant_probs || !tensor || (k_out && !meas_qubit) || (n_eff && (!out_local || !role_out)))
      fail(CUTQC_ERR_ARG, "NULL array");
    if (dtype != CUTQC_F32 && dtype != CUTQC_F64) fail(CUTQC_ERR_ARG, "bad dtype");
    const size_t es = dtype == CUTQC_F64 ? 8 : 4;
    need_aligned(variant_probs, es, "variant_probs");
    need_aligned(tensor, es, "tensor");
    // role of each local qubit: 0 kept (a measured cut qubit or an active
    // output), 1 merged, 2 / 3 zoomed at 0 / 1
    std::vector<int> seen(d, 0), lrole(d, 0), mq(k_out);
    for (int j = 0; j < k_out; ++j) {
      if (meas_qubit[j] < 0 || meas_qubit[j] >= d || seen[meas_qubit[j]]++) fail(CUTQC_ERR_SHAPE, "bad measured qubit");
      mq[j] = meas_qubit[j];
    }
    for (int i = 0; i < n_eff; ++i) {
      if (out_local[i] < 0 || out_local[i] >= d || seen[out_local[i]]++) fail(CUTQC_ERR_SHAPE, "bad output qubit");
      if (role_out[i] < 0 || role_out[i] > 3) fail(CUTQC_ERR_ARG, "role_out must be 0, 1, 2 or 3");
      lrole[out_local[i]] = role_out[i];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int> kept, oq;
    int mg = 0;
    bool zoomed = false;
    for (int j = 0; j < d; ++j) {
      if (lrole[j] == 0) kept.push_back(j);
      if (lrole[j] == 1) ++mg;
      if (lrole[j] >= 2) zoomed = true;
    }
    for (int i = 0; i < n_eff; ++i)
      if (role_out[i] == 0) oq.push_back(out_local[i]);
    if (mg == 0 && !zoomed) {   // nothing to merge: plain attribution
      launch_attribute(variant_probs, dtype, d, k_in, mq.data(), k_out, oq.data(), n_eff, tensor, s);
      return;
    }
    if (kept.empty()) fail(CUTQC_ERR_UNSUPPORTED, "no measured cut qubit or active output left to attribute");
    // merge the variant distributions over the merged outputs, zoomed ones
    // fixed, keeping the local qubits of `kept` in order (local qubit j is
    // bit d-1-j of a distribution's index); Eq. 3 and Eq. 2 act only on the
    // cut qubits and the init variants, so attributing the merged
    // distributions gives the merged tensor (Algorithm 1) without forming
    // the full one
    std::vector<uint64_t> act_val, mrg_val;
    uint64_t zoom = 0, mm = 0, am = 0;
    for (int j = d - 1; j >= 0; --j) {   // least significant index bit first
      const uint64_t xbit = uint64_t(1) << (d - 1 - j);
      if (lrole[j] == 0) {
        act_val.push_back(xbit);
        am |= xbit;
      } else if (lrole[j] == 1) {
        mrg_val.push_back(xbit);
        mm |= xbit;
      } else if (lrole[j] == 3) {
        zoom |= xbit;
      }
    }
    const int a = (int)kept.size();
    const bool run = mg > 0 && mm == ((uint64_t(1) << mg) - 1);
    const bool dense = run && am == (((uint64_t(1) << a) - 1) << mg);
    const size_t tab_act = (size_t)std::max((a + 7) / 8, 1) * 256, tab_mrg = (size_t)std::max((mg + 7) / 8, 1) * 256;
    int64_t rows = 1;
    for (int j = 0; j < k_in; ++j) rows *= 4;
    for (int j = 0; j < k_out; ++j) rows *= 3;
    const size_t nq = (size_t)rows << a;
    size_t off = 0;
    const size_t o_q = off;
    off = align_up(off + nq * es);
    const size_t o_mc = off;
    off = align_up(off + nq * 4);
    const size_t o_part = off;
    if (run) off = align_up(off + ((size_t)rows << (a + dd_merge_chunks(rows, a, mg))) * 8);
    const size_t o_act = off;
    off = align_up(off + tab_act * 8);
    const size_t o_mrg = off;
    off = align_up(off + tab_mrg * 8);
    DeviceState& ds = device_state();
    char* w = aux_buffer(ds, off) + aux_distance_bytes();
    launch_deposit_tables(act_val.data(), a, mrg_val.data(), mg, reinterpret_cast<uint64_t*>(w + o_act),
                          reinterpret_cast<uint64_t*>(w + o_mrg), s);
    launch_dd_merge(variant_probs, dtype, rows, d, a, mg, reinterpret_cast<const uint64_t*>(w + o_act),
                    reinterpret_cast<const uint64_t*>(w + o_mrg), zoom, run, dense, w + o_q,
                    reinterpret_cast<float*>(w + o_mc), w + o_part, s, run ? 0 : dd_merge_block(mm, mg, am, zoom));
    // the merged distributions' local qubits are `kept`, in order
    std::vector<int> pos(d, -1);
    for (int i = 0; i < a; ++i) pos[kept[i]] = i;
    for (int& q : mq) q = pos[q];
    for (int& q : oq) q = pos[q];
    launch_attribute(w + o_q, dtype, a, k_in, mq.data(), k_out, oq.data(), (int)oq.size(), tensor, s);
  });
}

int cutqc_simulate_subcircuit(const cutqc_gate* gates, int32_t n_gates, int32_t d, const int32_t* init_qubit,
                              int32_t k_in, const int32_t* meas_qubit, int32_t k_out, const int32_t* out_local,
                              int32_t n_eff, int32_t dtype, void* tensor, void* stream) {
  return guarded([&] {
    if (d < 1 || d > 30) fail(CUTQC_ERR_UNSUPPORTED, "simulator needs 1 <= d <= 30");
    if (n_gates < 0 || (n_gates && !gates)) fail(CUTQC_ERR_ARG, "bad gate list");
    if (k_in < 0 || k_out < 0 || n_eff < 0 || k_in + k_out > kMaxCuts) fail(CUTQC_ERR_SHAPE, "bad slot counts");
    if (k_out + n_eff != d) fail(CUTQC_ERR_SHAPE, "every local qubit must be an output or a measured cut qubit");
    if ((k_in && !init_qubit) || (k_out && !meas_qubit) || (n_eff && !out_local) || !tensor)
      fail(CUTQC_ERR_ARG, "NULL array");
    need_aligned(tensor, dtype == CUTQC_F64 ? 8 : 4, "tensor");   // written by the attribution kernels
    if (dtype != CUTQC_F32 && dtype != CUTQC_F64) fail(CUTQC_ERR_ARG, "bad dtype");
    std::vector<int> seen(d, 0);
    SimPlan sp;
    sp.d = d;
    sp.k_in = k_in;
    sp.k_out = k_out;
    sp.n_eff = n_eff;
    for (int j = 0; j < k_in; ++j) {
      if (init_qubit[j] < 0 || init_qubit[j] >= d) fail(CUTQC_ERR_SHAPE, "init qubit out of range");
      sp.init_q.push_back(init_qubit[j]);
    }
    for (int j = 0; j < k_out; ++j) {
      if (meas_qubit[j] < 0 || meas_qubit[j] >= d || seen[meas_qubit[j]]++) fail(CUTQC_ERR_SHAPE, "bad measured qubit");
      sp.meas_q.push_back(meas_qubit[j]);
    }
    for (int j = 0; j < n_eff; ++j) {
      if (out_local[j] < 0 || out_local[j] >= d || seen[out_local[j]]++) fail(CUTQC_ERR_SHAPE, "bad output qubit");
      sp.out_q.push_back(out_local[j]);
    }
    for (int g = 0; g < n_gates; ++g) {
      const cutqc_gate& gt = gates[g];
      if (gt.op < CUTQC_GATE_H || gt.op > CUTQC_GATE_CP) fail(CUTQC_ERR_ARG, "unknown gate op");
      if (gt.q0 < 0 || gt.q0 >= d) fail(CUTQC_ERR_SHAPE, "gate qubit out of range");
      if (gt.op >= CUTQC_GATE_CZ && (gt.q1 < 0 || gt.q1 >= d || gt.q1 == gt.q0)) fail(CUTQC_ERR_SHAPE, "bad two-qubit gate");
      sp.gates.push_back(gt);
    }
    run_subcircuit_sim(sp, dtype, tensor, static_cast<cudaStream_t>(stream));
  });
}

int cutqc_reconstruct_dd(const cutqc_problem* problem, const int8_t* role, void* bins, int32_t topk,
                         int64_t* top_idx, double* top_val, int32_t algo, void* stream) {
  return guarded([&] {
    validate(problem, true);
    if (!role) fail(CUTQC_ERR_ARG, "role is NULL");
    if (!bins) fail(CUTQC_ERR_ARG, "bins is NULL");
    need_aligned(bins, 16, "bins");
    if (algo < CUTQC_AUTO || algo > CUTQC_TC_TF32X3) fail(CUTQC_ERR_ARG, "unknown algo");
    if (topk < 0 || topk > 32) fail(CUTQC_ERR_UNSUPPORTED, "topk must be in 0..32");
    if (topk > 0 && (!top_idx || !top_val)) fail(CUTQC_ERR_ARG, "NULL top_idx / top_val");
    int na = 0;
    for (int q = 0; q < problem->n_qubits; ++q) {
      if (role[q] < 0 || role[q] > 3) fail(CUTQC_ERR_ARG, "role values must be 0..3");
      na += role[q] == 0;
    }
    if (na < 1) fail(CUTQC_ERR_SHAPE, "dynamic definition needs at least one active qubit");
    if (na > kMaxFD) fail(CUTQC_ERR_UNSUPPORTED, "more than 34 active qubits");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceState& ds = device_state();
    const cutqc_problem* p = problem;
    Plan& P = get_plan(ds, fd_key(p, 1, role, 0), [&](Plan& P) { build_dd_plan(P, p, role); });
    const int64_t nbins = int64_t(1) << na;
    int64_t max_rows = 1;
    for (const DdSubPlan& d : P.dd) max_rows = std::max(max_rows, d.rows);
    constexpr int NC = 32;
    size_t back = 0, off_tk = 0, off_cv = 0, off_ci = 0, off_m64 = 0, off_val = 0, off_part = 0;
    if (topk > 0) {
      off_tk = 0;
      back = align_up(topk_workspace_bytes(nbins));
      off_cv = back;
      back = align_up(back + NC * 4);
      off_ci = back;
      back = align_up(back + NC * 8);
      off_m64 = back;
      back = align_up(back + (size_t)NC * p->n_sub * max_rows * 8);
      off_val = back;
      back = align_up(back + NC * 8);
      off_part = back;
      back = align_up(back + (size_t)NC * dd_eval_chunks(p->n_cuts) * 8);
    }
    char* ddtab = static_cast<char*>(P.ddtab);
    char* front_ptr = nullptr;
    int fused_lists = 0;
    char* back_ptr = run_plan(ds, P, P.dd_front, back, dd_merge_pre(P, p, s, &front_ptr), bins, nullptr, algo, s,
                              nullptr, nullptr, topk > 0 ? off_tk : SIZE_MAX, &fused_lists);
    if (topk > 0) {
      float* cv = reinterpret_cast<float*>(back_ptr + off_cv);
      int64_t* ci = reinterpret_cast<int64_t*>(back_ptr + off_ci);
      if (fused_lists > 0)   // the tensor-core contraction kept the candidates while writing the bins
        launch_topk_lists(back_ptr + off_tk, fused_lists, cv, ci, s);
      else
        launch_topk(bins, P.dtype, nbins, back_ptr + off_tk, cv, ci, s);
      DdEvalArgs ea{};
      ea.n_sub = p->n_sub;
      ea.n_cuts = p->n_cuts;
      ea.n_active = na;
      ea.n_cand = NC;
      ea.f64 = P.dtype == CUTQC_F64;
      ea.max_rows = max_rows;
      ea.scale = std::ldexp(1.0, -p->n_cuts);
      ea.cand_idx = ci;
      for (int c = 0; c < p->n_sub; ++c) {
        const DdSubPlan& d = P.dd[c];
        DdEvalSub& e = ea.sub[c];
        ea.tens[c] = p->sub[c].tensor;
        e.m = front_ptr + d.ws_merged;
        e.mc = reinterpret_cast<const float*>(front_ptr + d.ws_mc);
        e.rows = d.rows;
        e.cols = int64_t(1) << d.f;
        e.a = d.a;
        e.mg = d.mg;
        e.nbA = (d.a + 7) / 8;
        e.nbM = (d.mg + 7) / 8;
        e.zoom = d.zoom;
        e.depAct = reinterpret_cast<const uint64_t*>(ddtab + d.off_act);
        e.depMrg = reinterpret_cast<const uint64_t*>(ddtab + d.off_mrg);
        for (int i = 0; i < d.a; ++i) e.act_rank[i] = d.act_rank[i];
        e.ncuts = (int)d.cuts.size();
        for (int j = 0; j < e.ncuts; ++j) e.cuts[j] = d.cuts[j];
      }
      double* m64 = reinterpret_cast<double*>(back_ptr + off_m64);
      double* val = reinterpret_cast<double*>(back_ptr + off_val);
      launch_dd_rerank(ea, P.dtype, m64, reinterpret_cast<double*>(back_ptr + off_part), val, s);
      std::vector<int64_t> hi(NC);
      std::vector<double> hv(NC);
      CUTQC_CUDA(cudaMemcpyAsync(hi.data(), ci, NC * 8, cudaMemcpyDeviceToHost, s));
      CUTQC_CUDA(cudaMemcpyAsync(hv.data(), val, NC * 8, cudaMemcpyDeviceToHost, s));
      CUTQC_CUDA(cudaStreamSynchronize(s));
      check_status(ds);
      std::vector<std::pair<double, int64_t>> cand;
      for (int j = 0; j < NC; ++j)
        if (hi[j] >= 0 && hi[j] < nbins) cand.emplace_back(hv[j], hi[j]);
      std::sort(cand.begin(), cand.end(), [](const std::pair<double, int64_t>& x, const std::pair<double, int64_t>& y) {
        return x.first > y.first || (x.first == y.first && x.second < y.second);
      });
      for (int j = 0; j < topk; ++j) {
        if (j < (int)cand.size()) {
          top_idx[j] = cand[j].second;
          top_val[j] = cand[j].first;
        } else {
          top_idx[j] = -1;
          top_val[j] = 0.0;
        }
      }
    }
  });
}

int cutqc_reconstruct_backward(const cutqc_problem* problem, const void* grad_out, const cutqc_loss* loss,
                               void* const* grad_tensor, double* loss_value, void* stream) {
  return guarded([&] {
    validate(problem, true);
    const cutqc_problem* p = problem;
    if (p->n_qubits > kMaxFD) fail(CUTQC_ERR_UNSUPPORTED, "the adjoint needs n_qubits <= 34");
    if (p->n_sub < 2) fail(CUTQC_ERR_UNSUPPORTED, "the adjoint needs at least two subcircuits");
    if (!grad_tensor) fail(CUTQC_ERR_ARG, "NULL gradient pointer");
    for (int c = 0; c < p->n_sub; ++c) {
      if (!grad_tensor[c]) fail(CUTQC_ERR_ARG, "NULL gradient pointer");
      need_aligned(grad_tensor[c], 16, "grad_tensor[c]");
    }
    need_aligned(grad_out, 16, "grad_out");
    need_aligned(loss_value, 8, "loss_value");
    const bool maxcut = loss && loss->kind == CUTQC_LOSS_MAXCUT;
    if (loss && loss->kind != CUTQC_LOSS_NONE && !maxcut) fail(CUTQC_ERR_ARG, "unknown loss kind");
    if (!maxcut && !grad_out) fail(CUTQC_ERR_ARG, "need grad_out or a loss");
    if (maxcut && (loss->n_edges < 0 || (loss->n_edges && !loss->edges))) fail(CUTQC_ERR_ARG, "bad edge list");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceState& ds = device_state();
    const double scale = std::ldexp(1.0, -p->n_cuts);
    // MaxCut bookkeeping of a pair of sides: the edges inside each side and
    // the bridge endpoints, as index bits (least significant = 0)
    struct Sides {
      BwdEdges inA{}, inB{};
      BwdBits brA{}, brB{};
    };
    auto split_edges = [&](const Node& A, const Node& B) {
      Sides sd;
      const int fA = A.f(), fB = B.f();
      std::vector<int> side(p->n_qubits, -1), bit(p->n_qubits, -1);
      for (int i = 0; i < fA; ++i) {
        side[A.bits[fA - 1 - i]] = 0;
        bit[A.bits[fA - 1 - i]] = i;
      }
      for (int i = 0; i < fB; ++i) {
        side[B.bits[fB - 1 - i]] = 1;
        bit[B.bits[fB - 1 - i]] = i;
      }
      for (int k = 0; k < loss->n_edges; ++k) {
        const int u = loss->edges[2 * k], v = loss->edges[2 * k + 1];
        if (u < 0 || v < 0 || u >= p->n_qubits || v >= p->n_qubits || u == v) fail(CUTQC_ERR_ARG, "bad edge");
        if (side[u] == side[v]) {
          BwdEdges& E = side[u] == 0 ? sd.inA : sd.inB;
          if (E.n >= 96) fail(CUTQC_ERR_UNSUPPORTED, "more than 96 edges inside one side");
          E.p[E.n] = bit[u];
          E.q[E.n] = bit[v];
          ++E.n;
        } else {
          if (sd.brA.n >= 16) fail(CUTQC_ERR_UNSUPPORTED, "more than 16 edges between the sides");
          const int ua = side[u] == 0 ? u : v, ub = side[u] == 0 ? v : u;
          sd.brA.p[sd.brA.n++] = bit[ua];
          sd.brB.p[sd.brB.n++] = bit[ub];
        }
      }
      return sd;
    };
    if (p->n_sub > 2) {
      // every subcircuit c against the group tensor R_c of all the others,
      // rebuilt by the forward's group builds (recomputation: nothing of the
      // forward is stored); the workspace is sized for the largest c first so
      // it is not reallocated while earlier work is in flight
      std::vector<Plan*> plans(p->n_sub);
      size_t need = 0;
      for (int c = 0; c < p->n_sub; ++c) {
        const std::string key = fd_key(p, 2, nullptr, 0) + "#bwd" + std::to_string(c);
        plans[c] = &get_plan(ds, key, [&](Plan& P) { build_bwd_plan(P, p, c); });
        const Step& st = plans[c]->steps.back();
        // per-row sums of both sides, then room for both sides' keys (f <= 24)
        auto key_room = [](int f) { return f <= 24 ? align_up(size_t(2) << f) : size_t(0); };
        const size_t back = maxcut ? align_up((size_t)(2 + 16) * plans[c]->nodes[st.a].rows() * 8) +
                                         align_up((size_t)(2 + 16) * plans[c]->nodes[st.b].rows() * 8) +
                                         key_room(plans[c]->nodes[st.a].f()) + key_room(plans[c]->nodes[st.b].f())
                                   : 0;
        size_t b = 0;
        run_plan(ds, *plans[c], 0, back, [](char*) { return std::vector<const void*>(); }, nullptr, nullptr,
                 CUTQC_CC, s, nullptr, &b, SIZE_MAX, nullptr, true);
        need = std::max(need, b);
      }
      char* ws = static_cast<char*>(workspace(ds, need));
      auto originals = [p](char*) {
        std::vector<const void*> t(p->n_sub);
        for (int c = 0; c < p->n_sub; ++c) t[c] = p->sub[c].tensor;
        return t;
      };
      for (int c = 0; c < p->n_sub; ++c) {
        Plan& P = *plans[c];
        const Step& st = P.steps.back();
        const Node& A = P.nodes[st.a];
        const Node& B = P.nodes[st.b];
        if ((int64_t)st.kmax != A.rows() || (int64_t)st.kmax != B.rows())
          fail(CUTQC_ERR_SHAPE, "internal: a subcircuit's cuts do not all join it to the rest");
        char* base = nullptr;
        char* back = run_plan(ds, P, 0, 0, originals, nullptr, nullptr, CUTQC_CC, s, ws, nullptr, SIZE_MAX, nullptr,
                              true, &base);
        const void* TR = B.orig >= 0 ? p->sub[B.orig].tensor : static_cast<const void*>(base + P.ws_node[st.b]);
        char* dtab = static_cast<char*>(P.dtab);
        const int32_t* rowC = reinterpret_cast<const int32_t*>(dtab + st.off_rows);
        const int32_t* rowR = rowC + st.kmax;
        if (maxcut) {
          const Sides sd = split_edges(A, B);
          double* sumsC = reinterpret_cast<double*>(back);
          const size_t offR = align_up((size_t)(2 + 16) * A.rows() * 8);
          double* sumsR = reinterpret_cast<double*>(back + offR);
          char* kbase = back + offR + align_up((size_t)(2 + 16) * B.rows() * 8);
          const size_t kbA = bwd_keys_bytes(A.f(), sd.inA, sd.brA), kbB = bwd_keys_bytes(B.f(), sd.inB, sd.brB);
          uint16_t* keysC = kbA ? reinterpret_cast<uint16_t*>(kbase) : nullptr;
          uint16_t* keysR = kbB ? reinterpret_cast<uint16_t*>(kbase + (A.f() <= 24 ? align_up(size_t(2) << A.f()) : 0))
                                : nullptr;
          if (keysC) launch_bwd_keys(A.f(), sd.inA, sd.brA, keysC, s);
          if (keysR) launch_bwd_keys(B.f(), sd.inB, sd.brB, keysR, s);
          launch_bwd_rowsums(p->sub[c].tensor, P.dtype, A.rows(), A.f(), sd.inA, sd.brA, sumsC, s, keysC);
          launch_bwd_rowsums(TR, P.dtype, B.rows(), B.f(), sd.inB, sd.brB, sumsR, s, keysR);
          launch_bwd_maxcut_grad(rowC, rowR, st.kmax, A.f(), sd.inA, sd.brA, sumsR, B.rows(), scale, grad_tensor[c],
                                 P.dtype, s, keysC);
          if (c == 0 && loss_value)
            launch_bwd_maxcut_loss(rowC, rowR, st.kmax, sumsC, A.rows(), sumsR, B.rows(), sd.brA.n, scale,
                                   loss_value, s);
        } else {
          const uint64_t* depC = reinterpret_cast<const uint64_t*>(dtab + st.off_depA);
          const uint64_t* depR = reinterpret_cast<const uint64_t*>(dtab + st.off_depB);
          launch_bwd_cc(TR, grad_out, rowC, rowR, st.kmax, A.f(), B.f(), depC, depR, scale, grad_tensor[c], P.dtype,
                        s);
        }
      }
      if (!maxcut && loss_value) {
        // L = sum_x G(x) p(x) = sum dL/dT_0 . T_0 (p is linear in each tensor)
        CUTQC_CUDA(cudaMemsetAsync(loss_value, 0, sizeof(double), s));
        launch_dot(grad_tensor[0], p->sub[0].tensor,
                   (int64_t(1) << (2 * (p->sub[0].k_in + p->sub[0].k_out))) << p->sub[0].n_eff, p->dtype, loss_value,
                   s);
      }
      return;
    }
    Plan& P = get_plan(ds, fd_key(p, 0, nullptr, 0), [&](Plan& P) { build_fd_plan(P, p); });
    if (P.steps.size() != 1) fail(CUTQC_ERR_UNSUPPORTED, "the adjoint supports a single final contraction");
    const Step& st = P.steps[0];
    const Node& A = P.nodes[st.a];
    const Node& B = P.nodes[st.b];
    const int sa = A.orig, sb = B.orig;
    if (sa < 0 || sb < 0) fail(CUTQC_ERR_UNSUPPORTED, "the adjoint needs two original subcircuits");
    const int fA = A.f(), fB = B.f();
    const int64_t rowsA = A.rows(), rowsB = B.rows();
    char* dtab = static_cast<char*>(P.dtab);
    const int32_t* rowA = reinterpret_cast<const int32_t*>(dtab + st.off_rows);
    const int32_t* rowB = rowA + st.kmax;
    if ((int64_t)st.kmax != rowsA || (int64_t)st.kmax != rowsB)
      fail(CUTQC_ERR_UNSUPPORTED, "the adjoint needs every slot of both subcircuits joined by a cut");
    void* dA = grad_tensor[sa];
    void* dB = grad_tensor[sb];
    const void* TA = p->sub[sa].tensor;
    const void* TB = p->sub[sb].tensor;
    if (maxcut) {
      // index bit (least significant = 0) of each qubit on its side
      std::vector<int> side(p->n_qubits, -1), bit(p->n_qubits, -1);
      for (int i = 0; i < fA; ++i) {
        side[A.bits[fA - 1 - i]] = 0;
        bit[A.bits[fA - 1 - i]] = i;
      }
      for (int i = 0; i < fB; ++i) {
        side[B.bits[fB - 1 - i]] = 1;
        bit[B.bits[fB - 1 - i]] = i;
      }
      BwdEdges inA{}, inB{};
      BwdBits brA{}, brB{};
      for (int k = 0; k < loss->n_edges; ++k) {
        const int u = loss->edges[2 * k], v = loss->edges[2 * k + 1];
        if (u < 0 || v < 0 || u >= p->n_qubits || v >= p->n_qubits || u == v) fail(CUTQC_ERR_ARG, "bad edge");
        if (side[u] == side[v]) {
          BwdEdges& E = side[u] == 0 ? inA : inB;
          if (E.n >= 96) fail(CUTQC_ERR_UNSUPPORTED, "more than 96 edges inside one subcircuit");
          E.p[E.n] = bit[u];
          E.q[E.n] = bit[v];
          ++E.n;
        } else {
          if (brA.n >= 16) fail(CUTQC_ERR_UNSUPPORTED, "more than 16 edges between the subcircuits");
          const int ua = side[u] == 0 ? u : v, ub = side[u] == 0 ? v : u;
          brA.p[brA.n++] = bit[ua];
          brB.p[brB.n++] = bit[ub];
        }
      }
      const size_t bytesA = align_up((size_t)(2 + brA.n) * rowsA * 8);
      const size_t bytesB = align_up((size_t)(2 + brB.n) * rowsB * 8);
      const size_t kbA = bwd_keys_bytes(fA, inA, brA), kbB = bwd_keys_bytes(fB, inB, brB);
      char* ws = static_cast<char*>(workspace(ds, bytesA + bytesB + kbA + kbB));
      double* sumsA = reinterpret_cast<double*>(ws);
      double* sumsB = reinterpret_cast<double*>(ws + bytesA);
      uint16_t* keysA = kbA ? reinterpret_cast<uint16_t*>(ws + bytesA + bytesB) : nullptr;
      uint16_t* keysB = kbB ? reinterpret_cast<uint16_t*>(ws + bytesA + bytesB + kbA) : nullptr;
      if (keysA) launch_bwd_keys(fA, inA, brA, keysA, s);
      if (keysB) launch_bwd_keys(fB, inB, brB, keysB, s);
      launch_bwd_rowsums(TA, P.dtype, rowsA, fA, inA, brA, sumsA, s, keysA);
      launch_bwd_rowsums(TB, P.dtype, rowsB, fB, inB, brB, sumsB, s, keysB);
      launch_bwd_maxcut_grad(rowA, rowB, st.kmax, fA, inA, brA, sumsB, rowsB, scale, dA, P.dtype, s, keysA);
      launch_bwd_maxcut_grad(rowB, rowA, st.kmax, fB, inB, brB, sumsA, rowsA, scale, dB, P.dtype, s, keysB);
      if (loss_value)
        launch_bwd_maxcut_loss(rowA, rowB, st.kmax, sumsA, rowsA, sumsB, rowsB, brA.n, scale, loss_value, s);
    } else {
      const uint64_t* depA = reinterpret_cast<const uint64_t*>(dtab + st.off_depA);
      const uint64_t* depB = reinterpret_cast<const uint64_t*>(dtab + st.off_depB);
      launch_bwd_cc(TB, grad_out, rowA, rowB, st.kmax, fA, fB, depA, depB, scale, dA, P.dtype, s);
      launch_bwd_cc(TA, grad_out, rowB, rowA, st.kmax, fB, fA, depB, depA, scale, dB, P.dtype, s);
      if (loss_value) {
        CUTQC_CUDA(cudaMemsetAsync(loss_value, 0, sizeof(double), s));
        launch_dot(dA, TA, rowsA << fA, P.dtype, loss_value, s);
      }
    }
  });
}

const char* cutqc_last_error(void) { return g_last_error.c_str(); }

void cutqc_release(void) {
  std::lock_guard<std::recursive_mutex> lk(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_dev) {
    cudaSetDevice(kv.first);
    drop_graphs(kv.second);
    for (int b = 0; b < kBranches; ++b) {
      if (kv.second.branch[b]) cudaStreamDestroy(kv.second.branch[b]);
      if (kv.second.join[b]) cudaEventDestroy(kv.second.join[b]);
      if (kv.second.mid[b]) cudaEventDestroy(kv.second.mid[b]);
    }
    if (kv.second.fork) cudaEventDestroy(kv.second.fork);
    kv.second.plans.clear();
    kv.second.order.clear();
    if (kv.second.ws) cudaFree(kv.second.ws);
    if (kv.second.one) cudaFree(kv.second.one);
    if (kv.second.status) cudaFree(kv.second.status);
    kv.second.status = nullptr;
    if (kv.second.aux) cudaFree(kv.second.aux);
    kv.second.aux = nullptr;
    kv.second.aux_bytes = 0;
    kv.second.ws = nullptr;
    kv.second.one = nullptr;
    kv.second.ws_bytes = 0;
  }
  g_dev.clear();
  cudaSetDevice(cur);
  release_sim_scratch();
}

int64_t cutqc_launch_count(void) { return g_launches.load(); }

int32_t cutqc_last_algo(void) { return g_last_algo; }

int cutqc_last_split(int32_t* nseg, double* bound) {
  return guarded([&] {
    if (!nseg || !bound) fail(CUTQC_ERR_ARG, "NULL output");
    if (!g_last_nseg || g_last_algo == CUTQC_CC) fail(CUTQC_ERR_ARG, "no tensor-core contraction has run");
    CUTQC_CUDA(cudaStreamSynchronize(g_last_stream));
    check_status(device_state());
    CUTQC_CUDA(cudaMemcpy(nseg, g_last_nseg, sizeof(int32_t), cudaMemcpyDeviceToHost));
    CUTQC_CUDA(cudaMemcpy(bound, g_last_bound, sizeof(double), cudaMemcpyDeviceToHost));
  });
}

int cutqc_distance(const void* a, const void* b, int64_t n, int32_t dtype, double* chi2, double* tv,
                   void* stream) {
  return guarded([&] {
    if (!a || !b || !chi2 || !tv) fail(CUTQC_ERR_ARG, "NULL pointer");
    need_aligned(a, dtype == CUTQC_F64 ? 8 : 4, "a");
    need_aligned(b, dtype == CUTQC_F64 ? 8 : 4, "b");
    need_aligned(chi2, 8, "chi2");
    need_aligned(tv, 8, "tv");
    if (n < 1 || n > (int64_t(1) << 40)) fail(CUTQC_ERR_UNSUPPORTED, "distance needs 1 <= n <= 2^40");
    if (dtype != CUTQC_F32 && dtype != CUTQC_F64) fail(CUTQC_ERR_ARG, "bad dtype");
    DeviceState& ds = device_state();
    char* scratch = aux_buffer(ds, 0);
    launch_distance(a, b, n, dtype, chi2, tv, scratch, static_cast<cudaStream_t>(stream));
  });
}

int cutqc_sample(const void* p, int64_t n, int32_t dtype, const double* u, int64_t n_samples, int64_t* out,
                 void* stream) {
  return guarded([&] {
    if (!p) fail(CUTQC_ERR_ARG, "p is NULL");
    if (n < 1 || n > (int64_t(1) << 40)) fail(CUTQC_ERR_UNSUPPORTED, "sampling needs 1 <= n <= 2^40");
    if (n_samples < 0) fail(CUTQC_ERR_ARG, "n_samples < 0");
    if (n_samples > 0 && (!u || !out)) fail(CUTQC_ERR_ARG, "NULL u or out");
    need_aligned(p, dtype == CUTQC_F64 ? 8 : 4, "p");
    need_aligned(u, 8, "u");
    need_aligned(out, 8, "out");
    if (dtype != CUTQC_F32 && dtype != CUTQC_F64) fail(CUTQC_ERR_ARG, "bad dtype");
    DeviceState& ds = device_state();
    char* scratch = aux_buffer(ds, sample_scratch_bytes(n)) + aux_distance_bytes();
    launch_sample(p, n, dtype, u, n_samples, out, scratch, static_cast<cudaStream_t>(stream));
  });
}

int cutqc_device_status(void* stream) {
  return guarded([&] {
    DeviceState& ds = device_state();
    CUTQC_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    check_status(ds);
  });
}

int cutqc_selftest_wait(int32_t limit_us, void* stream) {
  return guarded([&] {
    if (limit_us < 0 || limit_us > 2000000) fail(CUTQC_ERR_ARG, "limit_us outside [0, 2000000]");
    DeviceState& ds = device_state();
    launch_wait_selftest(status_word(ds), limit_us, static_cast<cudaStream_t>(stream));
  });
}

int cutqc_profile(int32_t enable) {
  return guarded([&] { g_profile = enable != 0; });
}

int cutqc_profile_read(int64_t* launches, double* total_ms) {
  return guarded([&] {
    if (!launches || !total_ms) fail(CUTQC_ERR_ARG, "NULL output");
    double ms = 0.0;
    for (auto& ab : g_prof_events) {
      CUTQC_CUDA(cudaEventSynchronize(ab.second));
      float t = 0.f;
      CUTQC_CUDA(cudaEventElapsedTime(&t, ab.first, ab.second));
      ms += t;
      cudaEventDestroy(ab.first);
      cudaEventDestroy(ab.second);
    }
    *launches = (int64_t)g_prof_events.size();
    *total_ms = ms;
    g_prof_events.clear();
  });
}

}  // extern "C"

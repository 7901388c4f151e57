/*
 * cutqc.h - C ABI of the GB300 reconstruction library for CutQC
 * (Tang et al., "CutQC: Using Small Quantum Computers for Large Quantum
 * Circuit Evaluations", arXiv 2012.02333).
 *
 * The library rebuilds an uncut circuit's output distribution from the
 * attributed probability tensors of its subcircuits (Sec. 3.2.3, Sec. 3.3):
 *
 *     p(x) = 2^-K  sum_{e in {I,X,Y,Z}^K}  prod_c  T_c[e|c][x|c]
 *
 * in full-definition mode (Sec. 4.2: all 2^n entries), in dynamic-definition
 * mode (Sec. 4.3, Algorithm 1: active qubits binned, merged qubits summed,
 * zoomed qubits fixed), and as an adjoint that gives dL/dT_c for a loss
 * L = sum_x G(x) p(x) over the reconstructed distribution.
 *
 * Conventions shared by every call
 *  - Qubit 0 is the most significant bit of every output index (the paper's
 *    |q_0 ... q_{n-1}> notation, Sec. 3.2).
 *  - Pauli digits: I=0, X=1, Y=2, Z=3.  A cut assignment e over K cuts is
 *    the base-4 number whose most significant digit is cut 0.
 *  - Subcircuit tensor T_c (caller-owned, device memory, row-major):
 *        [4^k_in][4^k_out][2^n_eff]
 *    k_in = init slots (rho_c, Eq. 5), k_out = measurement slots (O_c,
 *    Eq. 6), n_eff = effective output qubits (f_c, Eq. 7).  Row (a, b):
 *    a = digits of the init slots, b = digits of the measurement slots,
 *    slot 0 most significant; in_cut[j] / out_cut[j] name the global cut id
 *    of slot j.  Column x: bit i of x (bit 0 = most significant) is global
 *    qubit out_qubit[i].  Entry = Tr[(P_x (x) P_b) U (rho_0 (x) P_a) U^+]
 *    (Eq. 1-3): the Pauli-basis attribution of the subcircuit's variants.
 *  - Every call is stream-ordered and asynchronous on `stream` (a
 *    cudaStream_t; NULL = the legacy default stream) unless it says
 *    otherwise.  Device pointers must be on the current device.  The caller
 *    keeps inputs alive and unmodified until the stream has passed the call.
 *  - Alignment: device arrays given to the reconstruction calls (subcircuit
 *    tensors, out, bins, grad_out, grad_tensor) must be 16-byte aligned, as
 *    cudaMalloc and PyTorch allocations are (a tensor view at an element
 *    offset may not be); cutqc_attribute, cutqc_attribute_merged,
 *    cutqc_simulate_subcircuit, cutqc_distance and cutqc_sample take any
 *    element-aligned array; device
 *    scalars (sum_p, loss_value, chi2, tv) and the u / out arrays of
 *    cutqc_sample need their natural alignment.  Anything else is rejected
 *    with CUTQC_ERR_ARG before anything is launched.
 *  - The library owns a per-device workspace and a plan cache (device tables
 *    derived from the problem's structure).  Both grow on demand with
 *    cudaMalloc and persist until cutqc_release().  Calls from several host
 *    threads are serialised internally.
 *  - Errors: every entry point returns a cutqc_status.  Argument and shape
 *    errors are detected on the host before anything is launched; the
 *    message is available from cutqc_last_error() (thread-local).  No C++
 *    exception crosses this boundary.  Kernels never trap: a device-side
 *    check that fails writes a status word that the next synchronising
 *    call reports as CUTQC_ERR_DEVICE.
 *  - Limits: n_qubits <= 34 in full definition, #active <= 34 in dynamic
 *    definition, n_qubits <= 4096 overall, K <= 12, n_sub <= 16.  Outside
 *    them the call returns CUTQC_ERR_UNSUPPORTED.
 */
#ifndef CUTQC_H
#define CUTQC_H

#include <stdint.h>

#if defined(__GNUC__)
#define CUTQC_API __attribute__((visibility("default")))
#else
#define CUTQC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CUTQC_OK = 0,
  CUTQC_ERR_ARG = -1,          /* null pointer, bad enum, bad count            */
  CUTQC_ERR_SHAPE = -2,        /* inconsistent subcircuit / cut structure      */
  CUTQC_ERR_OOM = -3,          /* workspace allocation failed                  */
  CUTQC_ERR_CUDA = -4,         /* a CUDA runtime call failed                   */
  CUTQC_ERR_UNSUPPORTED = -5,  /* outside the documented limits                */
  CUTQC_ERR_TIMEOUT = -6,      /* a bounded device wait ran out                */
  CUTQC_ERR_DEVICE = -7        /* a device-side check failed                   */
} cutqc_status;

typedef enum { CUTQC_F64 = 0, CUTQC_F32 = 1 } cutqc_dtype;

/* How the main contraction (the 4^K sum) is computed.
 *  CUTQC_CC        CUDA-core FMA in the tensors' dtype (FP64 or FP32): the
 *                  plain baseline.
 *  CUTQC_TC_BF16X3 tcgen05 tensor cores, FP32 tensors only: each operand x
 *                  split into h = bf16(x), m = bf16(x - h); the products
 *                  h*h + h*m + m*h accumulate in FP32 in tensor memory.
 *                  Error per product <= ~3 * 2^-18 |a||b|.
 *  CUTQC_TC_BF16X6 as above with a third piece l = bf16(x - h - m) and the
 *                  six products hh, hm, mh, hl, lh, mm: FP32-level accuracy
 *                  at twice the tensor work.
 *  CUTQC_TC_TF32X3 tcgen05 tensor cores, FP32 tensors only: each operand x
 *                  split into hi = tf32(x), lo = tf32(x - hi) (round to
 *                  nearest; Ootomo and Yokota's split with TF32 pieces); the
 *                  products hi*hi + hi*lo + lo*hi accumulate in FP32 in
 *                  tensor memory.  Error per product <= ~3 * 2^-22 |a||b|, at
 *                  half the BF16 tensor rate and 4/3 of the BF16 x3 operand
 *                  bytes.  Never chosen by CUTQC_AUTO.
 *  CUTQC_AUTO      FP64 tensors: CUTQC_CC.  FP32 tensors: CUTQC_CC when the
 *                  final contraction has at most 16 Kronecker terms (a
 *                  streaming form whose output stream is all the work) and
 *                  no top bins are asked for (cutqc_reconstruct_dd with
 *                  topk > 0 keeps them in the tensor-core epilogue),
 *                  otherwise the tensor-core path when the shape allows it
 *                  (else CUTQC_CC), with the
 *                  number of products chosen on the device per call from
 *                  the a-priori bound S = 2^-K sum_e max|A_e| max|B_e|:
 *                  x3 when 3 * 2^-18 * S <= 2.5e-7, otherwise x6, so the
 *                  split error stays within a quarter of 1e-6 absolute. */
typedef enum {
  CUTQC_AUTO = 0,
  CUTQC_CC = 1,
  CUTQC_TC_BF16X3 = 2,
  CUTQC_TC_BF16X6 = 3,
  CUTQC_TC_TF32X3 = 4
} cutqc_algo;

/* One subcircuit (host struct; `tensor` is a device pointer). */
typedef struct {
  int32_t k_in, k_out, n_eff;
  const int32_t* in_cut;     /* host [k_in]  cut id of each init slot        */
  const int32_t* out_cut;    /* host [k_out] cut id of each measurement slot */
  const int32_t* out_qubit;  /* host [n_eff] global qubit of each output bit */
  const void* tensor;        /* device [4^k_in][4^k_out][2^n_eff], dtype     */
} cutqc_subcircuit;

/* One cut circuit.  Every cut id 0..n_cuts-1 must appear in exactly one
 * in_cut and one out_cut; the out_qubit lists must partition 0..n_qubits-1. */
typedef struct {
  int32_t n_qubits, n_cuts, n_sub;
  int32_t dtype;                  /* cutqc_dtype, the same for all tensors */
  const cutqc_subcircuit* sub;    /* host [n_sub] */
} cutqc_problem;

/* Full definition (Sec. 4.2).  For each of n_problems cut circuits write all
 * 2^n_qubits probabilities to out[i] (the problem's dtype, index = bit string
 * with qubit 0 most significant).  out[i] is device memory of the current
 * device, or pinned host memory mapped for the device (cudaHostAlloc /
 * cudaHostRegister, or a pinned torch tensor): the contraction then writes
 * the probabilities straight into host memory over the host link, with no
 * separate copy; they are there once the stream has passed the call.  Any
 * other pointer (unregistered host memory, another device's memory) is
 * rejected with CUTQC_ERR_ARG before anything runs.  Kronecker terms whose
 * factor rows are all zero are skipped (early termination, Sec. 4.2).
 * sum_p: device double [n_problems] receiving sum_x p(x) accumulated in FP64,
 * or NULL.  No host synchronisation for a single problem.  Several problems
 * (a batch) run together: the first call with a given set of shapes and
 * pointers runs eagerly and is captured into a CUDA graph that identical later
 * calls replay; every final contraction of at most 16 terms runs in one
 * launch over all such problems; under CUTQC_AUTO the first call times the
 * CUDA-core and tensor-core forms of every other FP32 problem's final
 * contraction once (this synchronises the stream) and keeps the faster per
 * problem structure, also across processes when the environment variable
 * CUTQC_AUTOTUNE_CACHE names a file (read on first use, appended to). */
CUTQC_API int cutqc_reconstruct_fd(const cutqc_problem* problems, int32_t n_problems,
                         void* const* out, int32_t algo, double* sum_p,
                         void* stream);

/* One slab of a full definition (Sec. 4.2, whose parallel processing has no
 * data dependency between output entries): the 2^(n_qubits - slab_bits)
 * probabilities whose slab_bits most significant output bits (qubits
 * 0 .. slab_bits-1) read slab_index, written to out in output order (out[j] =
 * p(slab_index * 2^(n_qubits - slab_bits) + j)).  G ranks that each compute
 * slab r of slab_bits = log2(G) together produce the whole distribution, and
 * the FP64 partial sums they write to sum_p (device double, or NULL) add up
 * to sum_x p(x): an 8-byte all-reduce is the only exchange.  Computed as a
 * recursion of the dynamic definition whose zoomed qubits are the slab's (no
 * merged qubits).  out as in cutqc_reconstruct_fd; algo as there.  No host
 * synchronisation.  0 <= slab_bits < n_qubits, else CUTQC_ERR_ARG. */
CUTQC_API int cutqc_reconstruct_fd_slab(const cutqc_problem* problem, int32_t slab_bits, int64_t slab_index,
                                        void* out, int32_t algo, double* sum_p, void* stream);

/* Dynamic definition, one recursion (Sec. 4.3, Algorithm 1).
 * role[q] (host, n_qubits entries): 0 active, 1 merged, 2 zoomed at 0,
 * 3 zoomed at 1.  Writes the 2^#active bins (device, the problem's dtype;
 * bin bit 0 = the lowest-numbered active qubit = most significant) = the
 * probability summed over the merged qubits with the zoomed qubits fixed.
 * If topk > 0, also returns on the host the topk heaviest bins ranked in FP64
 * (each candidate re-evaluated from the tensors in FP64; ties to the lower
 * index) in top_idx / top_val; this synchronises the stream. */
CUTQC_API int cutqc_reconstruct_dd(const cutqc_problem* problem, const int8_t* role,
                         void* bins, int32_t topk, int64_t* top_idx,
                         double* top_val, int32_t algo, void* stream);

/* Loss kinds for the adjoint. */
typedef enum { CUTQC_LOSS_NONE = 0, CUTQC_LOSS_MAXCUT = 1 } cutqc_loss_kind;

typedef struct {
  int32_t kind;              /* cutqc_loss_kind                                  */
  int32_t n_edges;           /* MAXCUT: G(x) = number of edges cut by x          */
  const int32_t* edges;      /* host [2*n_edges] qubit pairs                     */
} cutqc_loss;

/* Adjoint of the full definition: grad_tensor[c] (device, shape and dtype of
 * T_c) receives dL/dT_c for L = sum_x G(x) p(x), where G = grad_out (device,
 * 2^n entries, problem dtype) when loss is NULL or kind NONE, else the loss's
 * G(x) generated on the fly.  loss_value: device double receiving L in FP64,
 * or NULL.  No host synchronisation.  (Not in the paper: the gradient of an
 * expectation value over the reconstructed distribution.) */
CUTQC_API int cutqc_reconstruct_backward(const cutqc_problem* problem,
                               const void* grad_out, const cutqc_loss* loss,
                               void* const* grad_tensor, double* loss_value,
                               void* stream);

/* Full definition that allocates no device memory.  The paper has no
 * counterpart: this exists for callers that cannot let the library call
 * cudaMalloc - processes whose device memory is entirely reserved up front by
 * another allocator, and latency-sensitive callers that forbid device
 * allocation after start-up because cudaMalloc / cudaFree can synchronise the
 * device and stall other streams.  It computes what cutqc_reconstruct_fd
 * computes with CUTQC_CC (CUDA-core contraction in the tensors' dtype, early
 * termination, FP64 sum) for a problem of exactly two subcircuits, writing
 * out (2^n_qubits entries: device memory of the current device, or pinned
 * host memory mapped for the device, as for cutqc_reconstruct_fd) and, if
 * sum_p is not NULL, the FP64 sum to sum_p (device double on the current
 * device); other pointers are rejected with CUTQC_ERR_ARG before anything
 * runs.  The plan's tables are written on the device by a kernel from its
 * launch parameters: no host buffer is read after the call returns and no
 * host-to-device copy is made.  All of its scratch lives in one 4 MiB array in
 * device global memory that the library declares statically; every GPU that
 * loads the library holds it until the process exits.  Problems that need
 * more scratch (roughly K > 8 cuts) are rejected with CUTQC_ERR_UNSUPPORTED
 * and a message giving the bytes needed.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  Every call
 * shares the array: calls whose work overlaps on the GPU (for instance on two
 * streams) race and must not be issued. */
CUTQC_API int cutqc_reconstruct_fd_noalloc(const cutqc_problem* problem, void* out, double* sum_p,
                                           void* stream);

/* ---- input preparation: the GPU subcircuit simulator -------------------- */

typedef enum {
  CUTQC_GATE_H = 0, CUTQC_GATE_X, CUTQC_GATE_Y, CUTQC_GATE_Z, CUTQC_GATE_S,
  CUTQC_GATE_SDG, CUTQC_GATE_T, CUTQC_GATE_SX, CUTQC_GATE_SY, CUTQC_GATE_SW,
  CUTQC_GATE_RX, CUTQC_GATE_RY, CUTQC_GATE_RZ,
  CUTQC_GATE_CZ, CUTQC_GATE_CX, CUTQC_GATE_CP
} cutqc_gate_op;

typedef struct {
  int32_t op;        /* cutqc_gate_op                                         */
  int32_t q0, q1;    /* local qubits (q1 unused for 1-qubit gates; for CX q0
                        is the control)                                        */
  double param;      /* angle for RX/RY/RZ/CP                                 */
} cutqc_gate;

/* Exact cut search (Sec. 4.1, Eqs. 4-15), on the host.  The circuit's
 * multi-qubit gates (CZ, CX, CP, in order) are the vertices, the qubit wires
 * between consecutive multi-qubit gates the edges; single-qubit gates are
 * ignored.  Among the assignments of vertices to max_subcircuits (= n_C)
 * subcircuits with vertex k in a subcircuit <= k (Eq. 12) and every
 * subcircuit's width alpha + rho <= max_width (= D, Eq. 9), finds one of least
 * reconstruction cost L = 4^K sum_{c=2}^{n_C} prod_{i<=c} 2^{f_i} (Eq. 14; K
 * cut wires, f_i the outputs of subcircuit i, Eq. 7) by branch and bound; ties
 * go to the first assignment in vertex order.  Qubits no multi-qubit gate
 * touches belong to no vertex.  cluster: host int32 with room for one entry
 * per gate; receives the subcircuit of each multi-qubit gate, in gate order;
 * *n_vertices the number of them, *n_cuts K, *cost L (exact below 2^53).  The
 * search visits at most max_nodes nodes; beyond that, or when no assignment
 * fits the width, it returns CUTQC_ERR_UNSUPPORTED.  The paper solves the
 * same model with a MIP solver; this exhaustive form is for small circuits.
 * No GPU work. */
CUTQC_API int cutqc_cut_search(const cutqc_gate* gates, int32_t n_gates, int32_t n_qubits, int32_t max_width,
                               int32_t max_subcircuits, int64_t max_nodes, int32_t* cluster,
                               int32_t* n_vertices, int32_t* n_cuts, double* cost);

/* Attribution of measured variant distributions (Sec. 3.2.2, Eq. 2 and
 * Eq. 3): the tensor T[4^k_in][4^k_out][2^n_eff] of one subcircuit from the
 * output distributions of its 4^k_in x 3^k_out physical variants (Fig. 3),
 * for example normalised shot counts from a quantum device.
 * variant_probs: device [4^k_in][3^k_out][2^d] in `dtype`; variant index s
 * has one base-4 digit per init slot (slot 0 most significant; 0 = |0>,
 * 1 = |1>, 2 = |+>, 3 = |+i>), then one base-3 digit per measurement slot
 * (0 = Z basis, 1 = X, 2 = Y; X measured after H, Y after S^dagger then H),
 * then the d local qubits (local qubit 0 most significant).  meas_qubit[j]:
 * the local qubit measured for slot j; out_local[i]: the local qubit of output
 * i (output 0 = most significant bit of x); every local qubit is exactly one
 * of the two.  Eq. 3 weights outcome 0 by +1 and 1 by -1 for X, Y, Z and both
 * by +1 for I (I and Z read the Z-basis variant); Eq. 2 combines the inits
 * as I = |0><0| + |1><1|, Z = |0><0| - |1><1|, X = 2|+><+| - I,
 * Y = 2|+i><+i| - I.  Entries below 2^-40 in magnitude are written as 0.
 * tensor: device, caller-owned.  No workspace, no host synchronisation.
 * Shape errors are returned before anything is launched; d <= 30. */
CUTQC_API int cutqc_attribute(const void* variant_probs, int32_t d, int32_t k_in, const int32_t* meas_qubit,
                              int32_t k_out, const int32_t* out_local, int32_t n_eff, int32_t dtype,
                              void* tensor, void* stream);

/* The merged tensor one recursion of the dynamic definition (Sec. 4.3,
 * Algorithm 1) contracts for one subcircuit, straight from its variants'
 * measured distributions: [4^k_in][4^k_out][2^a] in `dtype`, a = the number
 * of active outputs, kept in output order (output 0 most significant).
 * Arguments as cutqc_attribute, plus role_out[n_eff] (host): the role of each
 * output in the recursion, 0 active, 1 merged (summed out), 2 zoomed at 0,
 * 3 zoomed at 1.  Merging sums over output qubits and fixes zoomed ones,
 * while Eq. 3 and Eq. 2 act only on the measured cut qubits' outcomes and the
 * init variants, so the library sums the variant distributions over the
 * merged outputs first (one read of variant_probs) and attributes the merged
 * distributions: the full 2^n_eff tensor is never formed.  Equals
 * attributing, then merging, up to rounding.  Uses a per-device buffer of the
 * library (the merged distributions, 4^k_in * 3^k_out * 2^(k_out + a)
 * entries); calls that overlap on the GPU race on it.  When nothing is merged
 * or zoomed this is cutqc_attribute.  Rejected with CUTQC_ERR_UNSUPPORTED
 * when no measured cut qubit and no active output remains. */
CUTQC_API int cutqc_attribute_merged(const void* variant_probs, int32_t d, int32_t k_in,
                                     const int32_t* meas_qubit, int32_t k_out, const int32_t* out_local,
                                     int32_t n_eff, const int8_t* role_out, int32_t dtype, void* tensor,
                                     void* stream);

/* Produce one subcircuit's attributed tensor on the GPU (Fig. 3, Eq. 2-3):
 * simulates every variant (state stored in complex FP64, gates evaluated in
 * double-float arithmetic of about 48 significant bits, attribution in FP64;
 * each init slot in |0>, |1>,
 * |+>, |+i>; each measurement slot measured in the Z, X, Y basis) of a
 * d-qubit subcircuit whose other qubits start in |0>, attributes the measured
 * cut qubits' outcomes with +-1 (Eq. 3) and combines the init variants into
 * Pauli operators (Eq. 2).  Entries below 2^-40 in magnitude become 0.
 * init_qubit[k_in], meas_qubit[k_out], out_local[n_eff]: host arrays of local
 * qubits (local qubit 0 = most significant).  tensor: device
 * [4^k_in][4^k_out][2^n_eff] of `dtype`.  d <= 30.  Synchronises the stream
 * before it returns; its scratch (state, attributed rows, gate tables) is kept
 * per device between calls up to 256 MiB (freed by cutqc_release), larger
 * scratch is allocated and freed per call. */
CUTQC_API int cutqc_simulate_subcircuit(const cutqc_gate* gates, int32_t n_gates,
                              int32_t d, const int32_t* init_qubit,
                              int32_t k_in, const int32_t* meas_qubit,
                              int32_t k_out, const int32_t* out_local,
                              int32_t n_eff, int32_t dtype, void* tensor,
                              void* stream);

/* ---- housekeeping -------------------------------------------------------- */

/* Message for the last non-OK status returned on this thread. */
CUTQC_API const char* cutqc_last_error(void);

/* Free the workspace and plan cache of every device. */
CUTQC_API void cutqc_release(void);

/* Number of kernels this library has launched since load (all devices). */
CUTQC_API int64_t cutqc_launch_count(void);

/* The cutqc_algo that computed the final contraction of the most recent
 * full-definition call on this thread: CUTQC_CC, or CUTQC_TC_BF16X3 for the
 * tensor-core path under CUTQC_AUTO (whose x3 / x6 choice is made on the
 * device), or the tensor-core form that was forced. */
CUTQC_API int32_t cutqc_last_algo(void);

/* Diagnostics of the most recent tensor-core final contraction on this
 * thread: the number of split products the device chose (3 or 6) and the
 * a-priori magnitude S = 2^-K sum_e max|A_e| max|B_e| it was chosen from.
 * Synchronises the stream of that call.  Returns CUTQC_ERR_ARG if no
 * tensor-core contraction has run on this thread. */
CUTQC_API int cutqc_last_split(int32_t* nseg, double* bound);

/* The chi^2 loss of Eq. 16 between two distributions of n entries (device,
 * `dtype`), sum_i (a_i - b_i)^2 / (a_i + b_i), into *chi2, and their total
 * variation (1/2) sum_i |a_i - b_i| into *tv (both device doubles).  A term
 * with a_i + b_i = 0 counts 0 (the paper leaves it undefined).  FP32 inputs:
 * terms in FP32, summed in compensated FP32 then FP64.  The result does not
 * depend on scheduling.  Uses a small per-device buffer of the library;
 * calls that overlap on the GPU (several streams) race on it. */
CUTQC_API int cutqc_distance(const void* a, const void* b, int64_t n, int32_t dtype, double* chi2, double* tv,
                             void* stream);

/* Draw n_samples outcomes from the distribution p of n entries (device,
 * `dtype`; for example a full-definition output or dynamic-definition bins) by
 * inverse transform: weights w_i = max(p_i, 0) (negative entries are rounding
 * residue), and for each uniform u[k] in [0, 1) (device doubles, supplied by
 * the caller) the smallest x whose running weight sum exceeds u[k] times the
 * total.  out: device int64 [n_samples].  An outcome with zero weight is never
 * drawn; if no outcome has weight every draw is -1.  Uses a per-device
 * buffer of the library (grows to 16 bytes per 1024 entries); calls that
 * overlap on the GPU race on it. */
CUTQC_API int cutqc_sample(const void* p, int64_t n, int32_t dtype, const double* u, int64_t n_samples,
                           int64_t* out, void* stream);

/* Every kernel that waits (on an mbarrier, a grid barrier or a flag) gives
 * up after a bounded time instead of hanging the GPU, and records that in a
 * per-device status word; its outputs are then invalid.  cutqc_device_status
 * synchronises `stream` and reports the word: CUTQC_OK, CUTQC_ERR_TIMEOUT (a
 * bounded wait ran out) or CUTQC_ERR_DEVICE (another device-side check
 * failed), then clears it.  cutqc_reconstruct_dd (when it returns a top
 * list) and cutqc_last_split check it themselves, as they synchronise.  The
 * full-definition and backward calls are asynchronous and do not: a caller
 * that needs the guarantee calls cutqc_device_status after them. */
CUTQC_API int cutqc_device_status(void* stream);

/* Failure-path self-test: launches one thread that waits on a device flag
 * nothing ever sets, with a limit of `limit_us` microseconds (0 .. 2e6);
 * when the limit runs out it records CUTQC_ERR_TIMEOUT in the status word,
 * exactly as a timed-out wait in the reconstruction kernels does, and ends
 * normally, so the context stays usable.  The paper has no counterpart: it
 * exists so the error path can be tested without a fault. */
CUTQC_API int cutqc_selftest_wait(int32_t limit_us, void* stream);

/* Kernel timing for roofline measurement.  While enabled, every launch of
 * the main contraction kernel of a full-definition call (the 4^K sum of the
 * final step) is bracketed by CUDA events recorded on the stream it is
 * launched on.  cutqc_profile_read() waits for the recorded events, returns
 * the number of bracketed launches and their summed duration in
 * milliseconds, and clears the record.  Not thread-safe against concurrent
 * calls on other threads. */
CUTQC_API int cutqc_profile(int32_t enable);
CUTQC_API int cutqc_profile_read(int64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* CUTQC_H */

/*
 * qaoa.h -- C ABI of the GB300 (sm_103a) QAOA state-vector simulator.
 *
 * The method is "Fast Simulation of High-Depth QAOA Circuits" (arXiv
 * 2309.04841): precompute the diagonal cost vector f(x) over all 2^n basis
 * states (Sec. 3.1), then apply p layers of the phase operator
 * exp(-i gamma_l f) (elementwise, Algorithm 3) and the transverse-field mixer
 * exp(-i beta_l sum_q X_q) (Algorithms 1-2), and reduce the objective
 * <psi|diag(f)|psi> and the ground-state overlap (Sec. 3.1, Sec. 4).
 *
 * Conventions (all entry points):
 *   - qubit q (0 <= q < n) is bit q of the basis index x; spin
 *     s_q(x) = +1 if bit q is 0, -1 if it is 1.
 *   - the mixer gate is exp(-i beta X) = [[cos b, -i sin b], [-i sin b, cos b]].
 *   - states are interleaved complex: float2 (QAOA_C64) or double2
 *     (QAOA_C128) per amplitude, 2^n amplitudes, index x.
 *   - cost vectors hold 2^n values of type int32, float32 or float64.
 *   - every device pointer is owned by the caller (allocate it with any CUDA
 *     allocator, e.g. a torch tensor); the library never allocates device
 *     memory and never frees a pointer it is given.  Cost and state buffers
 *     must be 16-byte aligned, workspaces 256-byte aligned.
 *   - calls enqueue work on `stream` and return without synchronising, unless
 *     the comment says "synchronises".  Results written to device pointers
 *     are valid once the stream reaches that point.
 *   - on any error the call returns a status, enqueues nothing further and
 *     leaves the outputs untouched; it never aborts or traps.  Errors of
 *     kernels that already ran asynchronously surface as QAOA_ERR_CUDA at the
 *     next synchronising call.
 *   - 1 <= n <= QAOA_MAX_N.  Calls are thread-safe if they use distinct
 *     workspaces; calls that share a workspace must be ordered on one stream.
 */
#ifndef QAOA_H
#define QAOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QAOA_MAX_N 34

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *qaoa_stream_t;

typedef enum {
    QAOA_OK = 0,
    QAOA_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum, angle or term  */
    QAOA_ERR_OUT_OF_MEMORY = 2, /* caller-provided buffer too small        */
    QAOA_ERR_OVERFLOW = 3,      /* integer cost would not fit int32        */
    QAOA_ERR_CUDA = 4,          /* a CUDA runtime call or kernel failed    */
    QAOA_ERR_TIMEOUT = 5,       /* a bounded wait ran out                  */
    QAOA_ERR_REJECTED = 6,      /* serving: request can never be admitted  */
    QAOA_ERR_CANCELLED = 7,     /* serving: request was cancelled          */
    QAOA_ERR_NOT_FOUND = 8,     /* serving: unknown ticket                 */
    QAOA_ERR_BUSY = 9           /* serving: queue full, retry later        */
} qaoa_status;

/* Cost vector element types.  QAOA_COST_U16 holds integer values 0..65535,
 * the paper's compact LABS storage (Sec. 5.2, distributed simulation:
 * f < 2^16 for the problems it simulates); half the memory and HBM traffic
 * of int32. */
typedef enum {
    QAOA_COST_I32 = 0,
    QAOA_COST_F32 = 1,
    QAOA_COST_F64 = 2,
    QAOA_COST_U16 = 3
} qaoa_cost_type;
typedef enum { QAOA_C64 = 0, QAOA_C128 = 1 } qaoa_state_type;

/*
 * One term of the cost polynomial f(s) = sum_k w_k prod_{i in t_k} s_i
 * (Eq. 1).  Bit i of `mask` set <=> variable i is in t_k.  mask == 0 is the
 * constant offset term.
 */
typedef struct {
    double weight;
    uint64_t mask;
} qaoa_term;

/* Statistics of a cost vector that later calls need. */
typedef struct {
    double f_min;       /* min_x f[x]                                    */
    double f_max;       /* max_x f[x]                                    */
    uint64_t n_min;     /* number of x with f[x] == f_min (ground states) */
    uint32_t step_log2; /* int32 / uint16 costs: largest k with 2^k
                           dividing every f[x] - f_min (LABS: at least 2); 0
                           for float costs and for a constant vector.  0 is
                           always valid. */
    uint32_t reserved;  /* 0 */
} qaoa_cost_stats;

/* Human-readable name of a status code (static string, never NULL). */
const char *qaoa_status_string(qaoa_status st);

/* Library version as major * 10000 + minor * 100 + patch. */
int qaoa_version(void);

/* Message describing the last error returned on the calling thread (static
 * thread-local buffer, "" if none). */
const char *qaoa_last_error_message(void);

/* ------------------------------------------------------------ host helpers */

/*
 * LABS terms (Background, "Low Autocorrelation Binary Sequences"):
 * f = sum_{k=1}^{n-1} C_k^2 with C_k = sum_i s_i s_{i+k}, written as
 * 4-body terms of weight 4, 2-body terms of weight 2 and a constant n(n-1)/2
 * (twice the paper's reduced polynomial plus n(n-1)/2).  Writes at most `cap`
 * terms to `out` (host) and the total count to *n_out; if cap is too small
 * returns QAOA_ERR_OUT_OF_MEMORY with *n_out set.  `out` may be NULL when
 * cap == 0.  n <= 64.
 */
qaoa_status qaoa_labs_terms(int n, qaoa_term *out, size_t cap, size_t *n_out);

/*
 * Weighted MaxCut terms (Background): f = sum_{(i,j)} (w_ij / 2)(s_i s_j - 1)
 * = -(cut weight), as m two-body terms of weight w/2 and one constant
 * -sum(w)/2.  edges: host array of 2m int32 (i, j), 0 <= i, j < n, i != j;
 * w: host array of m doubles (NULL means all 1).  Output as qaoa_labs_terms.
 */
qaoa_status qaoa_maxcut_terms(int n, const int32_t *edges, const double *w,
                              size_t m, qaoa_term *out, size_t cap,
                              size_t *n_out);

/* --------------------------------------------------------- a1: cost vector */

/*
 * Cost vector from terms (Sec. 3.1, Eq. 1; Algorithm 3 step 1):
 * d_costs[x] = sum_k w_k (-1)^popcount(x & mask_k), for all x < 2^n.
 *   terms: host array of n_terms terms; every mask < 2^n.
 *   QAOA_COST_I32: every weight must be an integer and sum |w_k| < 2^31
 *     (QAOA_ERR_OVERFLOW otherwise); the result is exact.
 *   QAOA_COST_F32 / F64: the sum is formed as in float64 in term order and
 *     rounded once to the output type; when every weight is a multiple of
 *     2^-e with sum |w_k| 2^e < 2^53 the sum is exact (order-independent).
 *     QAOA_COST_F32 takes at most 1024 terms.
 *   d_costs: device, 2^n elements of the cost type (not QAOA_COST_U16: build
 *     int32, then qaoa_convert_costs).
 */
qaoa_status qaoa_precompute_costs(int n, const qaoa_term *terms, size_t n_terms,
                                  qaoa_cost_type ct, void *d_costs,
                                  qaoa_stream_t stream);

/*
 * LABS cost vector directly from the autocorrelations (Background):
 * d_costs[x] = sum_{k=1}^{n-1} (n - k - 2 popcount((x ^ (x >> k)) & (2^{n-k}-1)))^2,
 * int32, exact; O(n) per x instead of O(n^2) terms.  n <= 32.
 */
qaoa_status qaoa_labs_costs(int n, int32_t *d_costs, qaoa_stream_t stream);

/*
 * The same LABS values stored as uint16 (QAOA_COST_U16; Sec. 5.2 stores the
 * precomputed diagonal this way, its maximum (n-1)n(2n-1)/6 being below 2^16
 * for every n <= 32 taken here).  d_costs: device, 2^n uint16, 16-byte
 * aligned.  n <= 32.  Asynchronous.
 */
qaoa_status qaoa_labs_costs_u16(int n, uint16_t *d_costs, qaoa_stream_t stream);

/*
 * Element-type conversion of a cost vector: int32 -> uint16 or uint16 ->
 * int32 (no other pair).  stats: of the source vector (host; for int32 ->
 * uint16 every value must lie in [0, 65535], else QAOA_ERR_OVERFLOW before any
 * launch).  d_src, d_dst: device, 2^n elements each, 16-byte aligned, not
 * overlapping.  The statistics of the result are the source's.  Asynchronous.
 */
qaoa_status qaoa_convert_costs(int n, const void *d_src, qaoa_cost_type src_ct,
                               const qaoa_cost_stats *stats, void *d_dst,
                               qaoa_cost_type dst_ct, qaoa_stream_t stream);

/*
 * Weighted MaxCut cost vector directly from the edge list (Background):
 * d_costs[x] = -sum_{(i,j) cut by x} w_ij, accumulated in edge order as in
 * float64 (exact when the weights are dyadic as for qaoa_precompute_costs).
 * edges/w as qaoa_maxcut_terms (host).  QAOA_COST_I32 needs integer weights
 * with sum |w| < 2^31.  m <= 1536.
 */
qaoa_status qaoa_maxcut_costs(int n, const int32_t *edges, const double *w,
                              size_t m, qaoa_cost_type ct, void *d_costs,
                              qaoa_stream_t stream);

/*
 * Minimum, maximum and number of minimisers of a cost vector, and for int32
 * costs the largest power of two dividing every f[x] - f_min (the phase
 * tables of later calls index (f - f_min) >> step_log2).  d_work is a device
 * workspace of at least qaoa_workspace_bytes(n) bytes.  Writes the result to
 * *h_out (host).  Synchronises `stream`.
 */
qaoa_status qaoa_cost_stats_compute(int n, const void *d_costs,
                                    qaoa_cost_type ct, void *d_work,
                                    size_t work_bytes, qaoa_cost_stats *h_out,
                                    qaoa_stream_t stream);

/* ------------------------------------------------------------- XY mixers */

/*
 * Hamming-weight-preserving XY mixer M = sum_{<i,j>} (X_i X_j + Y_i Y_j) / 2
 * over the edges of a ring or a complete graph on the qubits (Sec. 3.2, the
 * SU(4) extension of Algorithms 1-2).  exp(-i beta M) is taken as the
 * product of the edge gates exp(-i beta (X_i X_j + Y_i Y_j) / 2), first edge
 * first: ring (0,1), (1,2), ..., (n-2,n-1), (n-1,0) (the last one for n >= 3);
 * complete (i,j), i < j, in lexicographic order.
 */
typedef enum { QAOA_XY_RING = 1, QAOA_XY_COMPLETE = 2 } qaoa_xy_graph;

/*
 * Algorithm 3 with the XY mixer of `graph`: p layers of phase then mixer on
 * the state in d_state (the start state is the caller's, e.g. a Dicke state
 * from qaoa_dicke_state, since the mixer keeps the Hamming weight).  Other
 * arguments as qaoa_simulate (init_plus does not exist here; stats is needed
 * only with d_out, which receives [E, O] of the final state).  n >= 2.
 * Asynchronous.
 */
qaoa_status qaoa_simulate_xy(int n, const void *d_costs, qaoa_cost_type ct,
                             const qaoa_cost_stats *stats, const double *gammas,
                             const double *betas, int p, int graph, void *d_state,
                             qaoa_state_type st, void *d_work, size_t work_bytes,
                             double *d_out, qaoa_stream_t stream);

/*
 * Dicke state |D^n_k>: amplitude C(n,k)^{-1/2} on every basis state of
 * Hamming weight k, 0 elsewhere.  d_state: device, 2^n amplitudes of type st,
 * 16-byte aligned.  0 <= k <= n.  Asynchronous.
 */
qaoa_status qaoa_dicke_state(int n, int k, void *d_state, qaoa_state_type st,
                             qaoa_stream_t stream);

/* ------------------------------------------------------------- workspace */

/*
 * Bytes of device workspace (reduction partials and counters) that the calls
 * below need for n qubits; the same workspace serves every call on one stream.
 */
size_t qaoa_workspace_bytes(int n);

/*
 * Waits for `stream`, then reports whether a kernel that used this workspace
 * since the last qaoa_simulate / qaoa_grad call started gave up on a bounded
 * device-side wait (QAOA_ERR_TIMEOUT; the flag is then cleared).  Kernels
 * never trap or hang: a wait that runs out (about one second) records the
 * flag and the kernel returns, leaving its outputs incomplete.
 * d_work = NULL with work_bytes = 0 checks the library's built-in scratch on
 * the current device instead, the one qaoa_simulate_noalloc uses: this is how
 * a caller of that entry point learns that one of its calls timed out (check
 * before the next qaoa_simulate_noalloc call, which clears the flag).
 * Synchronises `stream`.
 */
qaoa_status qaoa_workspace_check(void *d_work, size_t work_bytes, qaoa_stream_t stream);

/*
 * Diagnostic for the path above: enqueues on `stream` one kernel whose
 * bounded device-side wait nothing completes (an mbarrier expecting bytes
 * that no copy delivers).  It gives up after about one second and records
 * the flag, so the next qaoa_workspace_check on this workspace returns
 * QAOA_ERR_TIMEOUT and the context stays usable.  d_work = NULL with
 * work_bytes = 0 targets the built-in scratch of the current device, as in
 * qaoa_workspace_check.  Asynchronous; errors: QAOA_ERR_INVALID_ARG
 * (workspace NULL with a nonzero size, or smaller than its 512-byte header
 * of counters), QAOA_ERR_CUDA (launch failure).
 */
qaoa_status qaoa_selftest_timeout(void *d_work, size_t work_bytes, qaoa_stream_t stream);

/* ---------------------------------------------------- a2-a4: simulation */

/*
 * Algorithm 3: p layers of  psi <- exp(-i beta_l sum X) exp(-i gamma_l f) psi.
 *   d_costs/ct: the cost vector; stats: from qaoa_cost_stats_compute on it
 *     (host struct; f_min, f_max and step_log2 are read; a struct filled by
 *     hand must satisfy f_min <= f[x] <= f_max, and step_log2 = 0 is always
 *     valid).
 *   gammas, betas: host arrays of p finite doubles, 1 <= p <= 100000.
 *   d_state: device, 2^n amplitudes of type st, updated in place.  If
 *     init_plus != 0 the input is ignored and the simulation starts from
 *     |+>^n (Background), otherwise from the state in d_state.
 *   d_work/work_bytes: device workspace (qaoa_workspace_bytes(n)).
 *   d_out: device, 2 doubles, or NULL.  If non-NULL, receives
 *     [E, O] = [sum_x |psi_x|^2 f_x, sum_{x: f_x = f_min} |psi_x|^2] of the
 *     final state (Sec. 3.1 inner product; Sec. 4 get_overlap), fused into
 *     the last pass.
 * Asynchronous.
 */
qaoa_status qaoa_simulate(int n, const void *d_costs, qaoa_cost_type ct,
                          const qaoa_cost_stats *stats, const double *gammas,
                          const double *betas, int p, void *d_state,
                          qaoa_state_type st, int init_plus, void *d_work,
                          size_t work_bytes, double *d_out,
                          qaoa_stream_t stream);

/*
 * qaoa_simulate without a workspace argument, for callers that cannot
 * allocate device memory (the paper has no counterpart): for example a plugin
 * whose host application owns every device allocation and forbids any outside
 * its own pool, or a caller whose fixed device-memory budget is already fully
 * committed.  The caller still provides d_costs, d_state and d_out exactly as
 * for qaoa_simulate; the scratch (reduction partials, counters, error word)
 * is a fixed 128.5 KiB device array inside the library, which every GPU that
 * loads the library holds until the process exits.
 *   - Maximum n = 23; a larger n returns QAOA_ERR_OUT_OF_MEMORY with a
 *     message, before anything is enqueued.
 *   - Every call looks up that array's device address (cudaGetSymbolAddress)
 *     with the device current.  The driver commits the array's memory when
 *     it loads this library's device code on a device; with CUDA's lazy
 *     module loading (the default) that can be the first call, so a caller
 *     whose memory budget will later be full should make its first call (or
 *     a qaoa_workspace_check(NULL, 0, stream)) while memory is still free;
 *     make that first call before any stream capture too.
 *   - All calls share the one array and each call clears the parts that must
 *     start at zero.  Calls that overlap on the GPU (different streams,
 *     different host threads) race on it: order them on one stream.
 *   - A bounded device-side wait that runs out sets the error word in the
 *     built-in scratch: qaoa_workspace_check(NULL, 0, stream) reports it
 *     (QAOA_ERR_TIMEOUT) until the next call of this entry point clears it.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Arguments, results and errors otherwise as qaoa_simulate.
 */
qaoa_status qaoa_simulate_noalloc(int n, const void *d_costs, qaoa_cost_type ct,
                                  const qaoa_cost_stats *stats, const double *gammas,
                                  const double *betas, int p, void *d_state,
                                  qaoa_state_type st, int init_plus, double *d_out,
                                  qaoa_stream_t stream);

/* ---------------------------------------------------- a5: reductions */

/*
 * Probabilities |psi_x|^2 of the state in d_state (Sec. 4, get_probabilities).
 *   d_probs: device, 2^n reals (float for QAOA_C64, double for QAOA_C128),
 *     16-byte aligned; or NULL for in place: every amplitude of d_state is
 *     replaced by |psi_x|^2 + 0i (the paper's preserve_state = False).
 * Asynchronous.
 */
qaoa_status qaoa_probabilities(int n, void *d_state, qaoa_state_type st, void *d_probs,
                               qaoa_stream_t stream);

/*
 * Expectation sum_x |psi_x|^2 f_x (Sec. 3.1) of the state in d_state, written
 * to d_out[0] (device double).  Deterministic order.  Asynchronous.
 * Precision: complex128 states are summed in double; for complex64 states
 * |psi_x|^2 f_x is formed exactly as a pair of floats and summed with the
 * rounding error of every add kept, runs of 32 terms then added in double,
 * which agrees with a double evaluation of the same state to about 1e-14
 * relative (the same holds for qaoa_overlap).
 */
qaoa_status qaoa_expectation(int n, const void *d_state, qaoa_state_type st,
                             const void *d_costs, qaoa_cost_type ct,
                             void *d_work, size_t work_bytes, double *d_out,
                             qaoa_stream_t stream);

/*
 * Ground-state overlap sum_{x: f_x = stats->f_min} |psi_x|^2 (Sec. 4,
 * get_overlap with the cost vector as the default), written to d_out[0].
 * Asynchronous.
 */
qaoa_status qaoa_overlap(int n, const void *d_state, qaoa_state_type st,
                         const void *d_costs, qaoa_cost_type ct,
                         const qaoa_cost_stats *stats, void *d_work,
                         size_t work_bytes, double *d_out,
                         qaoa_stream_t stream);

/* ---------------------------------------------------- a6: adjoint gradient */

/*
 * Objective and gradient with respect to all 2p angles (not in the paper):
 * forward simulation from |+>^n, then one backward sweep that un-applies the
 * layers in place on two state vectors (psi and lambda = d E / d psi^*),
 * accumulating
 *   dE/dbeta_l  = 2 Im <lambda| sum_q X_q |psi>   inside the un-mixer passes,
 *   dE/dgamma_l = 2 Im <lambda| f |psi>          before each un-phase.
 *   d_state, d_lambda: device, 2^n amplitudes each (contents ignored and
 *     overwritten; on return d_state holds approximately |+>^n).
 *   d_out: device, 2 + 2p doubles: [E, O, dE/dgamma_1..p, dE/dbeta_1..p],
 *     E and O of the forward final state.
 * Asynchronous.
 * Plan (complex64, n >= 13): the backward passes rotate the qubits in
 * groups; a group of up to 9 qubits on a 2^13-amplitude tile is taken where
 * it saves a group (n = 21, 29, 30).  Its passes run on one 512-thread CTA
 * per tile, the last pass on a pair of CTAs that exchange halves of the tile.
 * Environment variables, read at each call: QAOA_ADJOINT_PAIRS = "never" (no
 * such groups) or "always" (every group above the lowest 12 qubits is one);
 * QAOA_ADJOINT_WIDE = "pair" (every pass of those groups on CTA pairs) or
 * "all" (every pass, the last one too, on the 512-thread CTA).
 * Results agree across plans to rounding.
 */
qaoa_status qaoa_grad(int n, const void *d_costs, qaoa_cost_type ct,
                      const qaoa_cost_stats *stats, const double *gammas,
                      const double *betas, int p, void *d_state,
                      void *d_lambda, qaoa_state_type st, void *d_work,
                      size_t work_bytes, double *d_out, qaoa_stream_t stream);

/* ------------------------------------------------------ a7: serving loop */

/*
 * Continuous-batching request server (not in the paper).  Objective or
 * objective + gradient requests of any n (2..32) and p arrive at any time
 * (qaoa_server_submit returns at once).  A scheduler thread admits them as
 * GPU slots and device memory free up and runs admitted work concurrently:
 * requests with n <= 12 and p <= 128 are packed many per kernel launch (one
 * CTA each, state on chip); larger ones run on their own CUDA streams, up to
 * max_inflight units at a time.  All device memory comes from one
 * caller-owned arena (d_arena, arena_bytes), sub-allocated by the server:
 * a running request holds its state (8 B x 2^n, complex64), lambda (the same,
 * gradient requests only), workspace and outputs; cost vectors are cached per
 * (problem, n, problem_key) and evicted least recently used.  A request that
 * cannot fit the arena even when it is empty is rejected (its ticket reports
 * QAOA_ERR_REJECTED).  Results depend only on the request: the same
 * request gives bit-identical results alone and in any mix.
 */
typedef struct qaoa_server qaoa_server;

typedef enum { QAOA_PROBLEM_LABS = 0, QAOA_PROBLEM_MAXCUT = 1 } qaoa_problem;

typedef struct {
    int max_inflight;  /* GPU work units (streams) at once, 1..64           */
    int max_queue;     /* pending requests accepted before QAOA_ERR_BUSY    */
    int small_batch;   /* most n <= 12 requests packed into one launch      */
} qaoa_server_config;

typedef struct {
    qaoa_problem problem;
    int n, p;
    const int32_t *edges;   /* MaxCut: host, 2m vertex indices (copied)      */
    const double *weights;  /* MaxCut: host, m weights or NULL for 1 (copied) */
    size_t m;               /* MaxCut edge count, <= 1536                     */
    uint64_t problem_key;   /* equal (problem, n, key) => same cost vector    */
    const double *gammas;   /* host, p angles (copied)                        */
    const double *betas;    /* host, p angles (copied)                        */
    int want_grad;          /* 0: E and O only; 1: also all 2p derivatives    */
} qaoa_request;

typedef struct {
    qaoa_status status;     /* QAOA_OK, _REJECTED, _CANCELLED or an error   */
    double energy, overlap; /* E and O of the final state                     */
    double submit_s, admit_s, finish_s; /* host steady-clock seconds         */
} qaoa_result;

typedef struct {
    uint64_t submitted, completed, rejected, cancelled;
    double p50_ms, p99_ms;  /* latency (finish - submit) of completed ones    */
    double evals_per_s;     /* completed / (last finish - first submit)       */
    size_t arena_bytes, arena_peak_bytes, cached_cost_vectors;
} qaoa_server_stats_t;

/* Creates the server and its scheduler thread on the current device.  The
 * arena (device, 256-byte aligned, >= 1 MiB) stays owned by the caller and
 * must outlive the server. */
qaoa_status qaoa_server_create(const qaoa_server_config *cfg, void *d_arena, size_t arena_bytes,
                               qaoa_server **out);

/* Queues a request (all inputs copied) and returns its ticket; never blocks
 * on the GPU.  QAOA_ERR_BUSY when max_queue requests are pending. */
qaoa_status qaoa_server_submit(qaoa_server *srv, const qaoa_request *req, uint64_t *ticket);

/* Waits up to timeout_ms (< 0: forever) for the ticket, fills *out and, for
 * gradient requests, h_dgamma / h_dbeta (host, p each, may be NULL), then
 * forgets the ticket.  QAOA_ERR_TIMEOUT leaves the ticket valid. */
qaoa_status qaoa_server_wait(qaoa_server *srv, uint64_t ticket, qaoa_result *out,
                             double *h_dgamma, double *h_dbeta, int timeout_ms);

/* Cancels a pending request; a running one finishes on the GPU and reports
 * QAOA_ERR_CANCELLED. */
qaoa_status qaoa_server_cancel(qaoa_server *srv, uint64_t ticket);

qaoa_status qaoa_server_stats(qaoa_server *srv, qaoa_server_stats_t *out);

/* Stops the scheduler, waits for running work, releases streams and pinned
 * host buffers (the arena is the caller's). */
qaoa_status qaoa_server_destroy(qaoa_server *srv);

/* ------------------------------------------------------------ profiling */

/* Per-kernel-kind launch statistics (not in the paper; measurement aid). */
typedef struct {
    char name[24];      /* kernel kind, e.g. "fwd_low", "bwd_high"          */
    uint64_t launches;  /* launches recorded since the last reset            */
    double ms;          /* summed device time between the bracketing events  */
    double bytes;       /* summed algorithmic HBM bytes of those launches:
                           every state vector read and written once, the cost
                           vector read once where the launch needs it        */
} qaoa_prof_entry;

/*
 * When `on` is nonzero every kernel launch of this library is bracketed by
 * two CUDA events recorded on the launching stream (events come from a pool
 * created here; up to 65536 launches are recorded, later ones are counted
 * but not timed).  Turning it off keeps the records for qaoa_profile_read.
 */
qaoa_status qaoa_profile_enable(int on);

/*
 * Aggregates the recorded launches per kernel kind into out[0..cap) (host),
 * sets *n_out to the number of kinds, and if reset != 0 clears the records.
 * Waits for the recorded events (synchronises with the launches).
 */
qaoa_status qaoa_profile_read(qaoa_prof_entry *out, int cap, int *n_out, int reset);

#ifdef __cplusplus
}
#endif

#endif /* QAOA_H */

/*
 * ace.h - C ABI of the GB300 (sm_103a) implementation of the recursive
 * contraction of sparse symmetric tensors for symmetry-adapted n-correlations
 * (Kaliuzhnyi & Ortner, arXiv 2202.04140).
 *
 * The library evaluates, for a batch of environments e,
 *     phi[e][ch] = sum_{k in K} c[k][ch] * prod_{t=1}^{nu(k)} A[e][k_t]        (Eq. 1, Eq. 2)
 * over a sparse, permutation-sorted, degree-truncated set K of invariant
 * multi-indices, by the recursive computational graph of section 2.6: every
 * node AA_k of order >= 2 is the product AA_{k1} * AA_{k2} of two earlier nodes
 * (Eq. 4), auxiliary nodes (c = 0) fill in the sub-products that are not in K,
 * and the graph is built by Algorithm 1 (section 3.2) or Algorithm 2
 * (section 3.3).  It also evaluates the adjoint dphi/dA and, for O(3) bases,
 * the neighbour pooling A_nlm = sum_j R_n(r_j) Y_lm(r_j/|r_j|) and its adjoint
 * (the forces).
 *
 * Conventions for every entry point:
 *  - Every function returns an ace_status and never throws or aborts; on error
 *    a thread-local message is available from ace_last_error().
 *  - Handles (ace_spec, ace_dag) are owned by the library; free them with
 *    ace_spec_free / ace_dag_free.  Device buffers of a handle are allocated by
 *    the library with cudaMalloc on the current device, the first time the
 *    handle is used on that device (ace_dag_upload does it explicitly).
 *  - Tensors passed by pointer are owned by the caller.  "dev" pointers are
 *    CUDA device pointers on the current device, contiguous, 16-byte aligned;
 *    "host" pointers are ordinary host memory.  Row-major layouts throughout.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *    work is enqueued asynchronously; the calls that wait are
 *    ace_stream_status, the first use of a handle on a device (the plan upload
 *    waits for its copies), and calls that allocate or replace a buffer of the
 *    handle (cudaMalloc / cudaFree may synchronise the device): the first
 *    request of a kind, or one larger than any before.  Launch errors are
 *    reported at enqueue time.
 *  - One-particle ids: O(3) id = (n - nmin)(lmax+1)^2 + l^2 + (l + m);
 *    SO(2) id = (n - nmin)(2 lmax + 1) + (m + lmax); torus id = m + lmax.
 *  - Basis order ("canonical"): by correlation order nu, then lexicographic on
 *    the non-decreasing id tuple.  c is given in this order.
 */
#ifndef ACE_H_
#define ACE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ACE_ABI_VERSION 2

typedef enum {
  ACE_OK = 0,
  ACE_ERR_INVALID_ARG = -1, /* bad pointer, size, shape, alignment or parameter */
  ACE_ERR_OOM = -2,         /* host or device allocation failed */
  ACE_ERR_CUDA = -3,        /* a CUDA runtime call or kernel launch failed */
  ACE_ERR_TIMEOUT = -4,     /* a bounded device wait gave up (status word) */
  ACE_ERR_BOUNDS = -5,      /* a checked kernel saw an out-of-range index (status word) */
  ACE_ERR_UNSUPPORTED = -6, /* valid request this build does not implement */
  ACE_ERR_NO_DEVICE = -7    /* no CUDA device is available */
} ace_status;

enum { ACE_GROUP_O3 = 0, ACE_GROUP_SO2 = 1, ACE_GROUP_TORUS = 2 };
enum { ACE_ALGO_1 = 1, ACE_ALGO_2 = 2 };
enum { ACE_SPLIT_BALANCED = 0, ACE_SPLIT_PEEL = 1 };
enum { ACE_F32 = 0, ACE_F64 = 1 };
enum { ACE_READOUT_PLAIN = 0, ACE_READOUT_COMPENSATED = 1, ACE_READOUT_FP64_FINAL = 2 };

typedef struct ace_spec ace_spec; /* the index set K (library-owned) */
typedef struct ace_dag ace_dag;   /* the graph G and its device plan (library-owned) */

/* Index-set parameters (sections 2.2-2.5, Eq. 3, with p = 1 on the evaluated path).
 *  O(3):  k = (n, l, m), nmin <= n <= nmax, 0 <= l <= lmax, |m| <= l,
 *         degree wn*n + wl*l; invariance sum m = 0 and (if require_l_even) sum l even.
 *         With invariant features (section "Invariant features", phi_nlmk =
 *         R_n Y_l^m T_k(mu)): 0 <= k <= kmax, degree wn*n + wl*l + wk*k; the
 *         one-particle id is ((n - nmin)(kmax+1) + k)(lmax+1)^2 + l^2 + l + m
 *         (kmax = 0: no feature index).  kmax and wk are ignored by SO(2) and torus.
 *  SO(2): k = (n, m), |m| <= lmax, degree wn*n + wl*|m|; invariance sum m = 0.
 *  Torus: k = m, |m| <= lmax, degree |m|; invariance sum m = 0.
 *  p_norm: 1 (sum of one-particle degrees), 2, or 0 for the maximum.
 *  nu_max in [1, 8]. */
typedef struct {
  int32_t group;
  int32_t nmin, nmax;
  int32_t lmax;
  int32_t nu_max;
  int32_t deg_max;
  int32_t wn, wl;
  int32_t p_norm;
  int32_t require_l_even;
  int32_t kmax, wk;  /* invariant-feature degree range and weight (O(3)); ABI 2 */
} ace_spec_params;

/* ---- library ---------------------------------------------------------------- */

/* Thread-local message for the last error of this thread (never NULL). */
const char* ace_last_error(void);
/* ACE_ABI_VERSION of the loaded library. */
int32_t ace_abi_version(void);

/* ---- index set (host only, no GPU needed) ----------------------------------- */

/* Build K_G^p(D) (section 2.5, Eq. 3; invariance of sections 2.2-2.4).
 * params: host, read only.  *out receives a new handle.
 * Errors: INVALID_ARG for out-of-range parameters, OOM. */
ace_status ace_build_spec(const ace_spec_params* params, ace_spec** out);

/* Sizes of the set.  n_basis = |K|; K = number of one-particle functions;
 * counts_per_nu (host, may be NULL) receives nu_max entries: |K| per order 1..nu_max. */
ace_status ace_spec_info(const ace_spec* spec, int64_t* n_basis, int32_t* K, int64_t* counts_per_nu);

/* Copy the canonical tuples (host int32 [n_basis][nu_max], -1 padded) and the
 * total degree of each tuple (host int32 [n_basis]).  Either pointer may be NULL. */
ace_status ace_spec_tuples(const ace_spec* spec, int32_t* tuples, int32_t* deg);

void ace_spec_free(ace_spec* spec);

/* ---- graph (host only) --------------------------------------------------------- */

/* Build the computational graph G (section 2.6) with Algorithm 1 (algo = 1,
 * section 3.2) or Algorithm 2 (algo = 2, section 3.3, parameter n_split >= 1).
 * Leaves are the K one-particle nodes (ids 0..K-1); the basis is inserted in
 * canonical order; node ids are insertion order.  split_rule fixes the order in
 * which decompositions are tried (ACE_SPLIT_BALANCED: part sizes nu/2 down to
 * 1; ACE_SPLIT_PEEL: 1 up to nu/2).  Also builds the evaluation plan (host side).
 * Errors: INVALID_ARG, OOM. */
ace_status ace_build_dag(const ace_spec* spec, int32_t algo, int32_t split_rule, int32_t n_split,
                         ace_dag** out);

/* Counts: n_nodes (all nodes incl. leaves), n_aux (auxiliary nodes, c = 0,
 * section 2.6), n_operands (nodes of order >= 2 used as a factor of another
 * node), n_levels (highest correlation order = number of topological levels).
 * Any pointer may be NULL. */
ace_status ace_dag_info(const ace_dag* dag, int64_t* n_nodes, int64_t* n_aux, int64_t* n_operands,
                        int32_t* n_levels);

/* Export G in canonical ids (host buffers of n_nodes entries, any may be NULL):
 * left/right factor ids (-1 for leaves), level = correlation order, is_aux;
 * basis_node (host int32 [n_basis], may be NULL) = node id of each basis tuple. */
ace_status ace_dag_export(const ace_dag* dag, int32_t* left, int32_t* right, int32_t* level,
                          uint8_t* is_aux, int32_t* basis_node);

/* Plan statistics: n_slots (values stored per environment: leaves + operand
 * nodes), n_sinks (nodes of order >= 2 without consumers, folded into the
 * readout), n_entries (entries of the symmetric sink matrix), smem_bytes_f32
 * (shared memory per environment of the tile-per-lane FP32 forward+adjoint
 * kernel, which keeps the plan's "stored" slots: when a graph's operands do
 * not all fit a tile of four environments in shared memory, its least-used top
 * operands are left out and read through their two factors; the
 * "n_stored" plan array gives their number).  Any pointer may be NULL. */
ace_status ace_dag_plan_info(const ace_dag* dag, int64_t* n_slots, int64_t* n_sinks, int64_t* n_entries,
                             int64_t* smem_bytes_f32);

/* Copy one array of the evaluation plan, for inspection and tests.  `name` is
 * one of: "slot_node", "slot_basis", "n_g", "fwd_slot", "fwd_l", "fwd_r",
 * "fwd_off", "rev_slot", "rev_l", "rev_r", "rev_off", and for the symmetric
 * ("sym_") and one-sided ("one_") sink forms: "tasks" (4 int32 per task: row,
 * flags, factor slots), "slice_off", "slice_steps", "col", "ebasis", "ew2", and
 * their row-major copies "rm_tasks", "rm_off", "rm_col", "rm_ebasis", "rm_ew2",
 * and the cold tasks "cold_tasks", "cold_slice_off", "cold_slice_steps",
 * "cold_ca", "cold_cb" (factor slots of the operand read), "cold_ebasis",
 * "cold_ew2"; also "n_stored" and the stored forward levels "fwd_stored_slot",
 * "fwd_stored_l", "fwd_stored_r", "fwd_stored_off"; and per sink form the layout
 * of the row-major tasks as one stream per warp of the one-environment-per-lane
 * kernel: "loe_wbeg" (33 values: first 16-byte item of each of the 32 warps'
 * streams, then the total) and "loe_hpos" (item of each task's header; task t
 * belongs to warp t mod 32 and its entry pairs follow its header); "g_perm"
 * (the tile-per-lane kernel's adjoint row of each of the n_g slots with an adjoint,
 * a permutation chosen so that the adjoint updates one warp issues together fall
 * in different shared-memory banks).
 * Every array is exported as int32.  *count receives the number of int32
 * values; out (host) may be NULL to query the size.  Errors: INVALID_ARG for an
 * unknown name. */
ace_status ace_dag_plan_array(const ace_dag* dag, const char* name, int32_t* out, int64_t* count);

/* Host-side check of every plan index a kernel reads (forward and adjoint levels, tasks and
 * their slices, cold entries, the adjoint gather list, the row-major tasks and the per-warp
 * streams): the check the first upload performs before anything reaches a device.  Needs no
 * device.  Errors: INVALID_ARG (NULL dag), BOUNDS (an index out of range or an inconsistent
 * layout; the message names which). */
ace_status ace_dag_validate(const ace_dag* dag);

/* Write a graph to the file `path`: the parameters of its index set, the options it was built
 * with, and the graph itself (left factor, right factor and correlation order of every node, and
 * the node of every basis function), as a versioned little-endian file ending in the FNV-1a
 * 64-bit checksum of everything before it.  The evaluation plan is not stored (ace_dag_load
 * rebuilds it).  `spec` must be the index set the graph was built from.  Host only.
 * Errors: INVALID_ARG (NULL argument, a graph of another index set, the file cannot be
 * written), OOM. */
ace_status ace_dag_save(const ace_spec* spec, const ace_dag* dag, const char* path);

/* Read a file written by ace_dag_save into a new index set and graph (both owned by the caller:
 * ace_spec_free, ace_dag_free).  The index set is rebuilt from the stored parameters and must
 * equal the stored one (size and checksum of its tuples); the graph is checked before use:
 * leaves first, every other node the product of two earlier nodes with the sum of their orders,
 * every basis function's node distinct, of its order and of its tuple (by a multiset hash); the
 * plan is then rebuilt.  *params (may be NULL) receives the index set's parameters.  Host only.
 * Errors: INVALID_ARG (unreadable file, wrong magic or version, checksum mismatch, sizes that do
 * not match, an index set this library builds differently, a graph that fails a check), OOM. */
ace_status ace_dag_load(const char* path, ace_spec_params* params, ace_spec** spec_out, ace_dag** dag_out);

void ace_dag_free(ace_dag* dag);

/* ---- evaluation (device) ------------------------------------------------------ */

/* Allocate and upload the device plan on the current device (done implicitly
 * by the first evaluation; call it first when the evaluation is to be captured
 * in a CUDA graph). */
ace_status ace_dag_upload(ace_dag* dag, void* stream);

/* Forward: phi = sum_k c_k AA_k (Eq. 2) evaluated through G (Eq. 4).
 *  A   : dev [n_env][K] in dtype (ACE_F32 float, ACE_F64 double).
 *  c   : dev [n_basis][n_out] in dtype, canonical basis order.  Bound into the
 *        plan by a small gather kernel on `stream`; NULL reuses the
 *        coefficients bound by the previous call with the same n_out and dtype.
 *        A CUDA graph that captured an evaluation reads the coefficients bound
 *        when it was captured, from buffers of the handle: binding other
 *        coefficients (another c, dtype or n_out) to the handle afterwards
 *        changes what a replay reads.  Buffers replaced by a larger binding stay
 *        allocated until ace_dag_free, so a replay never reads freed memory; a
 *        global workspace replaced by a larger request is freed, so replaying a
 *        graph captured before such a request is not valid.
 *  phi : dev [n_env][n_out] in dtype, written.
 *  n_out in {1, 2, 4, 8, 16}.  readout: ACE_READOUT_PLAIN (FP32 sums),
 *  ACE_READOUT_COMPENSATED (per-task partial sums in FP32, combined by Kahan's
 *  compensated FP32 summation), ACE_READOUT_FP64_FINAL (partials
 *  combined in FP64).  For ACE_F64 all arithmetic is FP64 and readout is ignored.
 * Kernel forms (chosen by the autotuner's result, else automatically): one
 * environment per lane with the stored values of 32 environments in shared
 * memory (FP32, one channel, graph small enough); a tile of E environments per
 * CTA with the stored values in shared memory (any dtype and n_out, up to
 * 65535 stored values per environment); and, for graphs whose stored values do
 * not fit on chip (e.g. millions of basis functions), the stored values in a
 * global-memory workspace allocated by the first such call and kept in the graph
 * handle (FP32, one channel): by default two environments per lane, 64 per CTA,
 * grid x (n_slots + n_g) x 64 floats, or one environment per lane, 32 per CTA,
 * grid x (n_slots + n_g) x 32 floats; for FP32 forward requests with several
 * channels, one environment per lane with the stored values in that workspace and
 * each entry's coefficient row read once per warp.  ACE_KERNEL=lon|loe|loeg|loeg2|loem
 * forces one (loeg2: two environments per lane).
 * Errors: INVALID_ARG (null/misaligned pointer, n_env < 0, n_out), UNSUPPORTED,
 * NO_DEVICE, CUDA, OOM.  n_env = 0 is a no-op. */
ace_status ace_eval(ace_dag* dag, const void* A, const void* c, int64_t n_env, int32_t n_out,
                    int32_t dtype, int32_t readout, void* phi, void* stream);

/* Forward and reverse sweep (the adjoint of Eq. 4; not in the paper) fused in
 * one kernel: dA[e][k] = sum_ch phi_bar[e][ch] dphi[e][ch]/dA[e][k].
 *  phi_bar: dev [n_env][n_out] in dtype, or NULL meaning all ones.
 *  phi    : dev [n_env][n_out] or NULL (then phi is not written).
 *  dA     : dev [n_env][K] in dtype, written.
 * Other arguments and errors as ace_eval. */
ace_status ace_eval_grad(ace_dag* dag, const void* A, const void* c, const void* phi_bar,
                         int64_t n_env, int32_t n_out, int32_t dtype, int32_t readout, void* phi,
                         void* dA, void* stream);

/* ace_eval / ace_eval_grad with HOST buffers: the copies to and from the device
 * overlap the evaluation.  The batch is cut into chunks of chunk_env
 * environments.  Chunk i's rows of A
 * (and phi_bar) are copied to a device staging slot on one library stream, the
 * chunk is evaluated on a second, and its phi (and dA) copied back on a third:
 * while chunk i is evaluated, chunk i+1 is copied in and chunk i-1 out (two
 * staging slots).  Evaluations run one after another, as ace_eval_grad would.
 * chunk_env = 0 takes a short first and last chunk (whole waves of the kernel
 * form, SMs x environments per tile, at least 2 MiB of A: their copy-in and
 * copy-out overlap nothing) around two long chunks that take the rest; a batch
 * too small for that takes a third of the batch but at least 8 MiB of A and 4
 * waves per chunk (a smaller batch is one chunk).
 *  A       : host [n_env][K] in dtype, read.
 *  c       : dev [n_basis][n_out] in dtype, or NULL (bound coefficients), as ace_eval.
 *  phi_bar : host [n_env][n_out] in dtype, or NULL (ones); ace_eval_grad_host only.
 *  phi     : host [n_env][n_out] in dtype, written (may be NULL for the adjoint form).
 *  dA      : host [n_env][K] in dtype, written; ace_eval_grad_host only.
 * Host buffers should be page-locked (pinned): with pageable memory the copies
 * are correct but do not overlap.  Asynchronous with respect to `stream`: the
 * library streams first wait for the work queued on `stream`, and `stream` then
 * waits for every chunk, so the host outputs are complete once `stream` is
 * synchronised; the call can be captured in a CUDA graph (after a first call
 * of the same chunk size, which allocates the staging slots kept in the
 * handle).  The staging slots and streams belong to the handle: calls on one
 * handle must not overlap in time (issue them on one stream, or synchronise
 * between them).  Errors: as ace_eval / ace_eval_grad; INVALID_ARG for
 * chunk_env < 0. */
ace_status ace_eval_host(ace_dag* dag, const void* A, const void* c, int64_t n_env, int32_t n_out,
                         int32_t dtype, int32_t readout, void* phi, int64_t chunk_env, void* stream);
ace_status ace_eval_grad_host(ace_dag* dag, const void* A, const void* c, const void* phi_bar,
                              int64_t n_env, int32_t n_out, int32_t dtype, int32_t readout, void* phi,
                              void* dA, int64_t chunk_env, void* stream);

/* Autotuner (not in the paper): time every compiled kernel configuration for
 * this request — the one-environment-per-lane kernel with its stored values in
 * shared memory and in a global workspace (one or two environments per lane), its
 * several-channel forward form, and
 * the tile-per-lane kernel with each tile size E of 1, 2, 4, 8, 16 environments — on n_env
 * environments of small constant inputs, and keep the fastest in the graph handle; later
 * ace_eval / ace_eval_grad calls with the same dtype, n_out and mode use it.
 * Allocates and frees temporary device buffers (inputs, outputs, coefficients)
 * and leaves no coefficients bound.  best_kind (1 tile per lane, 2 one
 * environment per lane, 3 one environment per lane with the global workspace,
 * 4 one environment per lane with several channels: FP32 forward, n_out > 1,
 * stored values in the global workspace, coefficient rows read once per warp,
 * 5 two environments per lane with the global workspace), best_E and best_ms
 * (mean of 3 launches) may be NULL.
 * Environment variables ACE_KERNEL=lon|loe|loeg|loeg2|loem and ACE_TILE_E=<E> override both
 * the tuned and the default choice.  Errors: as ace_eval, UNSUPPORTED when no
 * configuration runs. */
ace_status ace_dag_autotune(ace_dag* dag, int64_t n_env, int32_t n_out, int32_t dtype, int32_t grad, int32_t readout,
                            void* stream, int32_t* best_kind, int32_t* best_E, float* best_ms);

/* The plain FP64 GPU evaluation of G: one thread per environment walks every
 * node in id order (Eq. 4), keeping every node value in global memory, reads
 * out phi and, if dA != NULL, runs the reverse sweep.  It is the baseline the
 * fused kernels are compared with.
 *  workspace: dev, at least ace_eval_plain_workspace_bytes(...) bytes, owned by
 *  the caller, contents irrelevant on entry.
 * Other arguments as ace_eval_grad (FP64 only, n_out in {1..16}). */
ace_status ace_eval_plain_workspace_bytes(const ace_dag* dag, int64_t n_env, int32_t with_grad,
                                          size_t* bytes);
ace_status ace_eval_plain_f64(ace_dag* dag, const double* A, const double* c, const double* phi_bar,
                              int64_t n_env, int32_t n_out, double* phi, double* dA, void* workspace,
                              size_t workspace_bytes, void* stream);

/* The same plain FP64 graph walk without any device allocation.
 * The paper has no counterpart to this entry point.  It exists for callers that
 * must not call cudaMalloc: code that runs where the device heap is owned by
 * another allocator (a framework's caching allocator reserving the memory),
 * code on latency-critical paths where an allocation call, which may
 * synchronise the device, is not acceptable, and hosts that only hand out
 * input and output buffers.  Its scratch is one array of 32 MiB that lives in
 * the library image on every GPU that loads libace, until the process exits.
 * Inside it go the graph (three int32 arrays of n_nodes, copied on each call
 * with cudaMemcpyAsync from pageable host memory held by the handle, so the
 * call returns once those bytes are staged) and the node values (n_nodes x
 * n_env doubles, twice that when dA != NULL).  A request larger than the array
 * fails with ACE_ERR_INVALID_ARG before any CUDA call, with a message giving
 * the bytes needed and the largest n_env that fits; nothing is truncated or
 * split.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it for the life of the process.  The
 * cached address does not survive cudaDeviceReset (or any other teardown of
 * the device's primary context): after one, do not call this entry point
 * again in the same process.  Every call on a device shares the array and the
 * kernel writes each scratch value before reading it, so nothing is cleared between
 * calls; calls whose work overlaps on the GPU (other streams, other threads)
 * race on the array and must be serialised by the caller.  The graph handle is
 * used on the host only (no upload).  Arguments and results are those of
 * ace_eval_plain_f64, minus the workspace. */
ace_status ace_eval_plain_f64_static(ace_dag* dag, const double* A, const double* c, const double* phi_bar,
                                     int64_t n_env, int32_t n_out, double* phi, double* dA, void* stream);

/* ---- neighbour pooling (device, O(3) only) ------------------------------------ */

/* A[e][id(n,l,m)] = sum_{j in env e} R_n(|r_j|) Y_lm(r_j/|r_j|)   (Eq. 2, section 2.4)
 * with R_n(r) = T_n(2r/rc - 1)(1 - r/rc)^2 (Chebyshev T_n, n = nmin..nmax) and
 * real orthonormal spherical harmonics without Condon-Shortley phase.
 *  pos     : dev float [n_pairs][3], neighbour positions relative to the centre.
 *  offsets : dev int64 [n_env + 1], CSR ranges of the neighbours of each env
 *            (offsets[0] = 0, non-decreasing, offsets[n_env] = n_pairs).
 *  A       : dev float [n_env][K], K = (nmax-nmin+1)(lmax+1)^2, written.
 * Neighbours with |r| >= rc or |r| = 0 contribute zero.  lmax <= 8.
 * Errors: INVALID_ARG, UNSUPPORTED (lmax > 8), CUDA. */
ace_status ace_pool_A(const float* pos, const int64_t* offsets, int64_t n_env, int64_t n_pairs,
                      float rc, int32_t nmin, int32_t nmax, int32_t lmax, float* A, void* stream);

/* Adjoint of ace_pool_A: dpos[j] = alpha * sum_k dA[e(j)][k] grad_{r_j} (R_n Y_lm)(r_j).
 * With dA = dphi/dA and alpha = -1 this writes the forces F_j = -dphi/dr_j.
 *  dA   : dev float [n_env][K];  dpos : dev float [n_pairs][3], written. */
ace_status ace_pool_A_grad(const float* pos, const int64_t* offsets, int64_t n_env, int64_t n_pairs,
                           float rc, int32_t nmin, int32_t nmax, int32_t lmax, const float* dA,
                           float alpha, float* dpos, void* stream);

/* Pooling with one invariant feature per neighbour (section "Invariant
 * features", phi_nlmk(r, mu) = R_n(r) Y_l^m(r/|r|) T_k(mu), T_k the Chebyshev
 * polynomial of degree k, 0 <= k <= kmax):
 *   A[e][id] = sum_{j in env e} R_n(|r_j|) T_k(mu_j) Y_lm(r_j/|r_j|),
 *   id = ((n - nmin)(kmax+1) + k)(lmax+1)^2 + l^2 + l + m  (the ids of a spec
 *   built with the same kmax).
 *  mu : dev float [n_pairs], feature value of each neighbour (in [-1, 1] for a
 *       well-conditioned T_k); may be NULL when kmax = 0.
 *  A  : dev float [n_env][K], K = (nmax-nmin+1)(kmax+1)(lmax+1)^2, written.
 * Limits: kmax <= 3, (nmax-nmin+1)(kmax+1) <= 16, lmax <= 8 (UNSUPPORTED
 * beyond).  kmax = 0 is ace_pool_A.  Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
ace_status ace_pool_A_feat(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env,
                           int64_t n_pairs, float rc, int32_t nmin, int32_t nmax, int32_t lmax, int32_t kmax,
                           float* A, void* stream);

/* Adjoint of ace_pool_A_feat with respect to the positions (the feature is a
 * label, not a coordinate): dpos[j] = alpha sum_id dA[e(j)][id] T_k(mu_j)
 * grad_{r_j}(R_n Y_lm)(r_j); alpha = -1 with dA = dphi/dA gives the forces. */
ace_status ace_pool_A_feat_grad(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env,
                                int64_t n_pairs, float rc, int32_t nmin, int32_t nmax, int32_t lmax, int32_t kmax,
                                const float* dA, float alpha, float* dpos, void* stream);

/* Energy and forces of a batch of environments, DEVICE buffers: pooling (Eq. 2, section 2.4),
 * the graph's forward and adjoint with phi_bar = 1 (Eq. 4, FP32, one channel) and the pooling
 * adjoint with alpha = -1: F_j = -dphi/dr_j.  Two forms compute it:
 *   fused       one kernel per tile of 32 environments: pooling into shared memory, the graph,
 *               the pooling adjoint from the adjoints still in shared memory (A and dA never
 *               reach global memory).  Needs no invariant features (kmax = 0), lmax = 6, at most
 *               8 radial functions and the graph's 32-environment layout in shared memory.
 *   three-kernel ace_pool_A_feat -> ace_eval_grad -> ace_pool_A_feat_grad through A and dA
 *               buffers of the batch kept in the handle (allocated by the first such call).
 * The three-kernel form runs by default (measured faster on GB300 with 50,000 environments of
 * 10-60 neighbours and K = 392: 0.645 ms against 0.759 ms); ACE_FORCES=fused selects the fused
 * form where it applies.  ace_energy_forces_plan tells which one runs.  Calls on one handle share
 * its A and dA buffers and its bound coefficients, so calls that overlap on the GPU (several
 * streams or threads) race and must be serialised by the caller; the buffers are replaced (the
 * old ones freed) when a larger batch arrives.
 *  pos, mu, offsets : dev, as ace_pool_A_feat (offsets are not checked: device memory).
 *  c       : dev [n_basis] float, or NULL (the bound coefficients of the adjoint form).
 *  phi     : dev [n_env] float, written.  forces: dev [n_pairs][3] float, written.
 * The graph must be built over the pooling's one-particle set:
 * K = (nmax - nmin + 1)(kmax + 1)(lmax + 1)^2.  Asynchronous on `stream`.  The fused form sums
 * an environment whose neighbours fall into several warps' ranges with shared-memory atomics, so
 * its last bits can differ between runs when an environment spans three or more ranges.
 * Errors: as ace_pool_A_feat and ace_eval_grad; INVALID_ARG for a graph whose K does not match. */
ace_status ace_energy_forces(ace_dag* dag, const float* pos, const float* mu, const int64_t* offsets, int64_t n_env,
                             int64_t n_pairs, const void* c, int32_t readout, float rc, int32_t nmin, int32_t nmax,
                             int32_t lmax, int32_t kmax, float* phi, float* forces, void* stream);

/* Which form ace_energy_forces (and ace_energy_forces_host) takes for these pooling parameters
 * on the current device: *fused = 1 and *smem_bytes = the fused kernel's shared memory per CTA,
 * or 0 and 0 for the three kernels.  Reads device attributes only.  Either output may be NULL.
 * Errors: INVALID_ARG (NULL dag), NO_DEVICE. */
ace_status ace_energy_forces_plan(ace_dag* dag, int32_t nmin, int32_t nmax, int32_t lmax, int32_t kmax,
                                  int32_t* fused, int64_t* smem_bytes);

/* Energy and forces of a batch of environments with HOST buffers: pooling
 * (ace_pool_A_feat), forward + adjoint with phi_bar = 1 (ace_eval_grad, FP32, one
 * channel) and the pooling adjoint with alpha = -1 (ace_pool_A_feat_grad), the
 * batch cut into chunks of chunk_env environments (0: as ace_eval_grad_host).  Positions (and mu) of chunk i are copied in on one
 * library stream, its forces pipeline runs on a second (the form of ace_energy_forces), its
 * forces and phi are copied out on a third: the copies overlap the kernels of neighbouring chunks.
 *  pos     : host [n_pairs][3] float, neighbour positions relative to their centre.
 *  mu      : host [n_pairs] float (invariant feature per neighbour) or NULL (kmax = 0).
 *  offsets : host [n_env + 1] int64, CSR: environment e owns pairs offsets[e] ..
 *            offsets[e+1]; checked here (offsets[0] = 0, non-decreasing,
 *            offsets[n_env] = n_pairs).
 *  c       : dev [n_basis] float, or NULL (the bound coefficients of the adjoint form).
 *  phi     : host [n_env] float, written.  forces: host [n_pairs][3] float, written
 *            (F_j = -dphi/dr_j).
 * The graph must be built over the pooling's one-particle set:
 * K = (nmax - nmin + 1)(kmax + 1)(lmax + 1)^2.  Device buffers (positions, offsets,
 * forces and phi of the whole batch, A and dA of two chunks for the three-kernel form) belong to the
 * handle and grow on demand.  Asynchronous and capturable as ace_eval_grad_host.
 * Errors: as ace_pool_A_feat and ace_eval_grad; INVALID_ARG for inconsistent offsets
 * or a graph whose K does not match. */
ace_status ace_energy_forces_host(ace_dag* dag, const float* pos, const float* mu, const int64_t* offsets,
                                  int64_t n_env, int64_t n_pairs, const void* c, int32_t readout, float rc,
                                  int32_t nmin, int32_t nmax, int32_t lmax, int32_t kmax, float* phi,
                                  float* forces, int64_t chunk_env, void* stream);

/* ---- status / utilities --------------------------------------------------------- */

/* Synchronise `stream` and read the device status word of `dag` (written by
 * kernels that check DAG indices or bound their waits).  Returns ACE_OK,
 * ACE_ERR_BOUNDS or ACE_ERR_TIMEOUT, and clears the word. */
ace_status ace_stream_status(ace_dag* dag, void* stream);

/* Device properties the planner uses: SM count and opt-in shared memory per block. */
ace_status ace_device_info(int32_t* sm_count, int32_t* smem_optin_bytes, int32_t* cc_major,
                           int32_t* cc_minor);

/* FP32 FMA throughput microbenchmark: runs `iters` dependent FMA chains per
 * thread on every SM and writes the elapsed device time (ms) and the FMA
 * count; used to measure the ALU roofline on the device. */
ace_status ace_fma_peak(int64_t iters, double* ms, double* fma_count, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ACE_H_ */

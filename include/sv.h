/*
 * sv.h -- C ABI of the GB300 state-vector core (libsv.so).
 *
 * The library applies parameterised gates to a 2^n complex amplitude vector,
 * reduces Pauli-sum expectation values and computes the adjoint-method
 * Jacobian, all on one NVIDIA GB300 (sm_103a), with hand-written CUDA kernels.
 * It follows the problem statement of arXiv 2403.02512:
 *   - a state is 2^n complex amplitudes, 32- or 64-bit floating point
 *     (Sec. 2: "fully templated end-to-end ... 32-bit or 64-bit");
 *   - wire w is bit (n - 1 - w) of an amplitude index: wire 0 is the most
 *     significant bit (Alg. 1, q_offset = n - q - 1);
 *   - a gate is (kind, wires, angles, inverse flag) (Listing 1), optionally
 *     controlled by wires that must hold prescribed values (Alg. 2);
 *   - an observable is a Hamiltonian: coefficients times Pauli words
 *     (Sec. 2.2, Listing 2);
 *   - gradients come from the adjoint method as a Jacobian matrix (Sec. 2.2,
 *     Sec. 4.3: "build and return the Jacobian matrix"), parameters in,
 *     results and Jacobian out (Sec. 2).
 *
 * Conventions for every entry point:
 *   - no C++ exception crosses this boundary; every call returns sv_status;
 *   - on SV_ERR_ARG / SV_ERR_UNSUPPORTED nothing was launched and the state
 *     is unchanged; sv_last_error() holds a message for the calling thread;
 *   - host pointers are plain host memory unless a parameter says "device";
 *     the library never keeps a caller pointer after the call returns, except
 *     the device buffer given to sv_create_from_device_ptr / sv_set_workspace;
 *   - all GPU work is issued on the state's stream (sv_set_stream); calls that
 *     return host results synchronise that stream before returning;
 *   - angles, expectation values and Jacobians are FP64 on the host side
 *     whatever the state's precision.
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SV_MAX_QUBITS 34      /* 2^34 complex128 = 256 GiB, the largest that can fit */
#define SV_MAX_TARGETS 6      /* target wires of one op (dense matrices up to 64 x 64) */
#define SV_MAX_CONTROLS 8

typedef struct sv_state sv_state;     /* opaque: one state vector on one GPU */
typedef struct sv_program sv_program; /* opaque: a planned circuit + observables */

typedef enum {
    SV_C64 = 0,  /* complex64: FP32 amplitudes, FP32 gate arithmetic, FP64 / compensated reductions */
    SV_C128 = 1  /* complex128: FP64 amplitudes and arithmetic */
} sv_dtype;

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = 1,          /* invalid argument (bad wire, size, pointer, NaN angle ...) */
    SV_ERR_OOM = 2,          /* device allocation failed or exceeds the allocation cap */
    SV_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    SV_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    SV_ERR_UNSUPPORTED = 5,  /* valid request the library does not implement */
    SV_ERR_STATE = 6         /* an earlier asynchronous device error is latched; sv_reset clears it */
} sv_status;

/* Base gates of Sec. 2.1.2 and Sec. 3.2.  Matrices (c = cos(t/2), s = sin(t/2)):
 *   RX(t)=exp(-i t X/2), RY(t)=exp(-i t Y/2), RZ(t)=exp(-i t Z/2);
 *   PhaseShift(t)=diag(1, e^{it}) (Listing 1); Rot(a,b,c)=RZ(c) RY(b) RZ(a);
 *   IsingXX(t)=exp(-i t XX/2) (Eq. 1), IsingYY(t)=exp(-i t YY/2),
 *   IsingZZ(t)=exp(-i t ZZ/2), IsingXY(t)=exp(i t (XX+YY)/4);
 *   SingleExcitation(t): [[c,-s],[s,c]] on (|01>,|10>), identity elsewhere;
 *   DoubleExcitation(t): the same on (|0011>,|1100>).
 * The first target wire is the most significant bit of a gate's local index. */
typedef enum {
    SV_IDENTITY = 0,
    SV_PAULI_X = 1,
    SV_PAULI_Y = 2,
    SV_PAULI_Z = 3,
    SV_HADAMARD = 4,
    SV_S = 5,
    SV_T = 6,
    SV_PHASE_SHIFT = 7,
    SV_RX = 8,
    SV_RY = 9,
    SV_RZ = 10,
    SV_ROT = 11,
    SV_SWAP = 12,
    SV_ISING_XX = 13,
    SV_ISING_YY = 14,
    SV_ISING_ZZ = 15,
    SV_ISING_XY = 16,
    SV_SINGLE_EXCITATION = 17,
    SV_DOUBLE_EXCITATION = 18,
    SV_MATRIX = 19,          /* dense 2^k x 2^k matrix supplied by the tape */
    SV_OP_KIND_COUNT = 20
} sv_op_kind;

/* One operation of a tape.
 *   angle[a] = scale * params[param_index[a]]  if param_index[a] >= 0,
 *            = const_angle[a]                   otherwise.
 * A parameter may be used by several ops; its Jacobian column sums them.
 * adjoint != 0 applies the conjugate transpose (the "inverse" flag of
 * Listing 1).  Controls (Alg. 2): the op acts only on amplitudes whose control
 * wires hold control_values (0 or 1).  SV_MATRIX ops read 4^k complex entries,
 * row-major, interleaved (re, im), from tape->matrices + 2 * matrix_offset. */
typedef struct {
    int32_t kind;
    int32_t n_targets;
    int32_t targets[SV_MAX_TARGETS];
    int32_t n_controls;
    int32_t controls[SV_MAX_CONTROLS];
    int32_t control_values[SV_MAX_CONTROLS];
    int32_t param_index[3];
    double const_angle[3];
    double scale;
    int32_t adjoint;
    int64_t matrix_offset;
} sv_op;

typedef struct {
    int32_t n_ops;
    const sv_op *ops;
    int32_t n_params;         /* length of the parameter vector = Jacobian columns */
    const double *matrices;   /* SV_MATRIX data, may be NULL if no such op */
    int64_t n_matrix_entries; /* complex entries available in matrices */
} sv_tape;

/* A Hamiltonian sum_t coeffs[t] * P_t (Listing 2).  Pauli word t acts with X on
 * the wires in x_mask & ~z_mask, Y on x_mask & z_mask, Z on z_mask & ~x_mask;
 * bit w of a mask is wire w (NOT an amplitude-index bit).  n_terms may be 0. */
typedef struct {
    int32_t n_terms;
    const double *coeffs;
    const uint64_t *x_mask;
    const uint64_t *z_mask;
} sv_pauli_sum;

/* ---- library ------------------------------------------------------------ */

/* Message of the last failed call on this thread ("" if none).  Owned by the
 * library, valid until the next call on this thread. */
const char *sv_last_error(void);

/* Build identification string (compile flags, arch).  Static storage. */
const char *sv_version(void);

/* Cap on the device bytes the library itself allocates (0 = no cap).  Allocations
 * that would exceed it fail with SV_ERR_OOM (used to test the OOM path). */
sv_status sv_set_alloc_cap(size_t bytes);

/* ---- state ---------------------------------------------------------------- */

/* Allocate a 2^n state on the current CUDA device, initialised to |0...0>.
 * 1 <= n <= SV_MAX_QUBITS.  *out owns its device buffer; free with sv_destroy. */
sv_status sv_create(int n, sv_dtype dtype, sv_state **out);

/* Wrap a caller-owned device buffer of 2^n amplitudes (interleaved re/im of the
 * dtype's width, 256-byte aligned).  Contents are used as they are; the buffer
 * must outlive the state. */
sv_status sv_create_from_device_ptr(int n, sv_dtype dtype, void *device_ptr, sv_state **out);

/* Release the state, its workspace and any library-owned buffer.  NULL is a no-op.
 * Programs created for the state refer to it: destroy them first. */
sv_status sv_destroy(sv_state *s);

/* Issue all further work for s on this CUDA stream (cudaStream_t; NULL = legacy default). */
sv_status sv_set_stream(sv_state *s, void *cuda_stream);

/* Optional caller-owned device workspace (256-byte aligned, `bytes` long): a
 * call whose temporaries fit in it uses it instead of library allocations; a
 * call that needs more allocates its own, as if none were set.  A Jacobian or
 * VJP needs about (2 + m_c) state vectors (phi buffers and m_c lambda
 * vectors) plus small tables; probabilities, samples and sparse expectation
 * values need a few partial-sum arrays.  NULL / 0 returns to library-owned
 * workspace.  The buffer must outlive every call that uses it. */
sv_status sv_set_workspace(sv_state *s, void *device_ptr, size_t bytes);

/* Arithmetic of a complex128 state (its storage stays IEEE complex128):
 *   SV_COMPUTE_NATIVE (default) -- FP64;
 *   SV_COMPUTE_DOUBLE_FLOAT     -- double-float: each real as an unevaluated sum of two
 *     FP32 values (~48 significant bits, errors ~1e-14 relative per operation), run on the
 *     FP32 pipe, which is 62x the FP64 rate on a GB300; expectation values and Jacobians
 *     are still reduced in FP64.
 * complex64 states accept only SV_COMPUTE_NATIVE.  Planned programs follow the state's
 * current mode (their gate matrices are rebuilt when it changes). */
typedef enum { SV_COMPUTE_NATIVE = 0, SV_COMPUTE_DOUBLE_FLOAT = 1 } sv_compute;
sv_status sv_set_compute(sv_state *s, int compute);

/* Renormalisation after a circuit's forward pass (the complex64 precision
 * reading of the method: only norms, expectation values and adjoint inner
 * products are reduced in FP64).  When on, sv_forward and sv_program_forward
 * end with psi <- psi / ||psi||, ||psi||^2 summed in FP64 in a fixed order, all
 * on the device (no host synchronisation).  Single-gate calls (sv_apply,
 * sv_apply_op, sv_apply_matrix) never renormalise.  Default: on for complex64
 * states, off for complex128 states (their drift from 1 is what sv_norm2
 * reports).  on: 0 or 1; SV_ERR_ARG for a NULL state or another value. */
sv_status sv_set_renormalize(sv_state *s, int on);

/* Dense 5-qubit blocks on complex64 states run on the tensor cores (tcgen05,
 * three TF32 products per FP32 product, FP32 accumulation in tensor memory)
 * unless this library-wide switch is 0; then they run on the CUDA cores.
 * Default 1.  A tensor-core wait that runs out (bounded at 1 s) makes the
 * next synchronising call on the state return SV_ERR_TIMEOUT. */
sv_status sv_set_dense_tensor_cores(int on);

/* Query: n, dtype and the device pointer of the amplitudes (any may be NULL). */
sv_status sv_info(const sv_state *s, int *n, sv_dtype *dtype, void **device_ptr);

/* |basis_index> (index bits: wire 0 = MSB).  Clears a latched SV_ERR_STATE. */
sv_status sv_reset(sv_state *s, uint64_t basis_index);

/* Copy 2^n amplitudes (interleaved re/im in the state's dtype) host -> state / state -> host. */
sv_status sv_set_state(sv_state *s, const void *host_amplitudes);
sv_status sv_get_state(sv_state *s, void *host_amplitudes);

/* Wait for all work issued on the state's stream; reports latched device errors. */
sv_status sv_synchronize(sv_state *s);

/* ---- gates ------------------------------------------------------------------ */

/* Apply one base gate (Sec. 2.1.1, Alg. 1; Listing 1 inverse flag):
 * wires = its n_targets target wires, angles = its angles (NULL if none). */
sv_status sv_apply(sv_state *s, int kind, const int *wires, int n_wires,
                   const double *angles, int adjoint);

/* Apply one tape op (controls and control values per Alg. 2); params is the
 * parameter vector its param_index entries refer to (may be NULL if none). */
sv_status sv_apply_op(sv_state *s, const sv_op *op, const double *params,
                      const double *matrices);

/* Apply a dense 2^k x 2^k matrix (row-major, interleaved re/im, k <= SV_MAX_TARGETS)
 * to the k wires (Sec. 2.1.2, generic many-qubit gate). */
sv_status sv_apply_matrix(sv_state *s, const int *wires, int k, const double *matrix, int adjoint);

/* ---- measurements ------------------------------------------------------------ */

/* out[j] = <psi|H_j|psi> for j < n_obs (Sec. 2.2), FP64 accumulation (complex64:
 * compensated FP32 per thread, FP64 across threads), fixed summation order:
 * repeated calls give bitwise-equal results.  complex128 Hamiltonians of many
 * words (on average >= 4 per observable, <= 64 observables) are summed as
 * Re<psi|(H_j psi)> with (H_j psi) formed per amplitude in FP64 registers. */
sv_status sv_expval(sv_state *s, const sv_pauli_sum *obs, int n_obs, double *out);

/* out = <psi|psi> in FP64. */
sv_status sv_norm2(sv_state *s, double *out);

/* Variances (the GPU device's variance measurement, Sec. 2.2):
 *   out[j] = <psi|H_j^2|psi> - <psi|H_j|psi>^2 = ||H_j psi||^2 - <H_j>^2
 * (real coefficients make H_j Hermitian).  lambda_j = H_j psi is formed by the
 * same passes as the adjoint method's lambda vectors; ||lambda_j||^2 is summed
 * in FP64 over a fixed set of partial sums, so results repeat bitwise.  out is
 * a host array of n_obs doubles.  Device workspace: min(n_obs, what fits) state
 * vectors (the rest in chunks).  Same argument errors as sv_expval; the state
 * is not modified. */
sv_status sv_var(sv_state *s, const sv_pauli_sum *obs, int n_obs, double *out);

/* Marginal probabilities of k wires (the device's probability measurement,
 * Sec. 2.2; Listing 3 reads probabilities out of a circuit):
 *   out[b] = sum of |psi_i|^2 over indices i whose bits at wires[0..k) spell b,
 * with wires[0] the most significant bit of b (wire w = index bit n-1-w).
 * 0 <= k <= min(n, SV_MAX_PROB_WIRES); wires distinct and in [0, n); out is a
 * host array of 2^k doubles.  FP64 sums in a fixed order (bitwise repeatable).
 * k = 0 gives out[0] = <psi|psi>.  SV_ERR_ARG on bad wires; the state is not
 * modified. */
#define SV_MAX_PROB_WIRES 24
sv_status sv_probs(sv_state *s, const int *wires, int k, double *out);

/* Samples of k wires by inverse transform: for each caller-drawn uniform
 * u[t] in [0, 1) (host array of `shots`), out[t] (host, uint64) is the first
 * outcome b whose cumulative probability -- the marginal probabilities of
 * sv_probs summed in ascending b by a fixed-order scan -- exceeds u[t] times
 * their total.  The caller owns the random numbers (seeded, reproducible);
 * the same uniforms give the same samples.  SV_ERR_ARG for a uniform outside
 * [0, 1), bad wires or shots < 0; the state is not modified. */
sv_status sv_sample(sv_state *s, const int *wires, int k, const double *uniforms, int64_t shots, uint64_t *out);

/* ---- circuits ---------------------------------------------------------------- */

/* psi <- U_N ... U_1 psi for the tape with the given parameters.  Ops are fused
 * into shared-memory passes (gate fusion) without changing the result
 * beyond rounding. */
sv_status sv_forward(sv_state *s, const sv_tape *tape, const double *params);

/* Adjoint-method Jacobian (the method the paper cites for Lightning's gradients,
 * Sec. 2.1 / 3.1.1):  the state must hold psi = U(params)|psi0>, e.g. from
 * sv_forward.  expvals_out[j] = <psi|H_j|psi> (may be NULL);
 * jacobian_out[j * n_params + p] = d<H_j>/d params[p].  psi is not modified. */
sv_status sv_adjoint_jacobian(sv_state *s, const sv_tape *tape, const double *params,
                              const sv_pauli_sum *obs, int n_obs,
                              double *expvals_out, double *jacobian_out);

/* Vector-Jacobian product sum_j grad_out[j] * d<H_j>/d params (one backward
 * sweep with lambda = sum_j grad_out[j] H_j psi).  Same precondition as above. */
sv_status sv_adjoint_vjp(sv_state *s, const sv_tape *tape, const double *params,
                         const sv_pauli_sum *obs, int n_obs, const double *grad_out,
                         double *vjp_out);

/* ---- planned programs (device-resident re-execution) --------------------------- */

/* Plan a tape and observables once for state s: fusion passes, device tables and
 * workspace are built here; later calls only move parameters.  The program keeps
 * copies of everything it needs; tape and obs may be freed after the call.  The
 * program runs on s (its buffer and stream) and must be destroyed before s. */
sv_status sv_program_create(sv_state *s, const sv_tape *tape, const sv_pauli_sum *obs,
                            int n_obs, sv_program **out);
sv_status sv_program_destroy(sv_program *p);

/* Parameters: n_params doubles, on the host (params_on_device = 0) or in device
 * memory (1).  Gate matrices are rebuilt on the device from them. */
sv_status sv_program_set_params(sv_program *p, const double *params, int params_on_device);

/* Forward pass on the program's state (from its current contents). */
sv_status sv_program_forward(sv_program *p);

/* Expectation values and full Jacobian of the program's observables; outputs on
 * the host (outputs_on_device = 0, the call synchronises) or device pointers (1,
 * asynchronous on the state's stream).  expvals_out may be NULL. */
sv_status sv_program_jacobian(sv_program *p, double *expvals_out, double *jacobian_out,
                              int outputs_on_device);

/* Expectation values of the program's observables for the current state
 * (outputs on the host, synchronising, or device pointers, asynchronous). */
sv_status sv_program_expval(sv_program *p, double *expvals_out, int outputs_on_device);

/* Vector-Jacobian product of the program's observables for the current state:
 * vjp_out[p] = sum_j grad_out[j] d<H_j>/d params[p], one backward sweep with
 * lambda = sum_j grad_out[j] H_j psi (grad_out: m host doubles).  Output on the
 * host (outputs_on_device = 0, synchronising) or in device memory (1).
 * Device memory: psi plus two vectors (phi, lambda). */
sv_status sv_program_vjp(sv_program *p, const double *grad_out, double *vjp_out, int outputs_on_device);

/* Jacobian-vector product in forward mode (the JVP integration the paper
 * names as future work, Sec. 5): jvp_out[j] = sum_p d<H_j>/d params[p]
 * tangent[p] (tangent: n_params host doubles, finite).  One tangent pass runs
 * the tape from the state's CURRENT contents (as sv_program_forward does)
 * while carrying d psi / dt, starting at 0; each trainable gate
 * U = exp(i s theta G) adds i s scale tangent[p] G psi after it; then
 * jvp_out[j] = 2 Re <H_j psi | d psi> with FP64 fixed-order sums.  The state
 * ends holding the forward output (not renormalised).  Cost: one pass over two
 * vectors plus one lambda per observable, whatever the number of parameters
 * (the full Jacobian by forward mode is n_params such calls; by reverse mode,
 * sv_program_jacobian, one sweep per observable).  Output m doubles on the host
 * (synchronising) or in device memory (outputs_on_device = 1).
 * SV_ERR_ARG: no observables, NULL or non-finite tangent; SV_ERR_STATE:
 * parameters never set. */
sv_status sv_program_jvp(sv_program *p, const double *tangent, double *jvp_out, int outputs_on_device);

/* ---- sparse observables -----------------------------------------------------
 * A general sparse observable in CSR form (the SparseHamiltonian the paper's
 * GPU device accepts for expectation values and the adjoint method, Sec. 2.2):
 * indptr[0..2^n] (indptr[0] = 0, non-decreasing, indptr[2^n] = nnz), column
 * indices[0..nnz) in [0, 2^n), values[0..2*nnz) complex (re, im) interleaved.
 * sv_sparse_create validates and copies the arrays to the current device
 * (one allocation; SV_ERR_ARG on a malformed matrix, SV_ERR_OOM).  The matrix
 * is taken as given: Hermitian matrices give real expectation values. */
typedef struct sv_sparse sv_sparse;
sv_status sv_sparse_create(int n, const int64_t *indptr, const int64_t *indices, const double *values, int64_t nnz,
                           sv_sparse **out);
sv_status sv_sparse_destroy(sv_sparse *h);

/* out = Re <psi|H psi> (one warp per row, FP64 sums in a fixed order). */
sv_status sv_sparse_expval(sv_state *s, const sv_sparse *h, double *out);

/* Adjoint Jacobian of <H> for a sparse H: the state holds psi = U(params)|.>
 * (as for sv_adjoint_jacobian); lambda = H psi from the SpMV, then the usual
 * reverse sweep.  expval_out (may be NULL): 1 double; jacobian_out:
 * n_params doubles, host. */
sv_status sv_adjoint_jacobian_sparse(sv_state *s, const sv_tape *tape, const double *params, const sv_sparse *h,
                                     double *expval_out, double *jacobian_out);

/* Kernel launches issued by the last program call (for launch accounting). */
sv_status sv_program_stats(const sv_program *p, int *n_forward_passes, int *n_adjoint_passes,
                           int *launches_last_call);

/* Kernel timing for roofline accounting.  While enabled, every kernel launch of
 * the library is bracketed by CUDA events on the stream it runs on, grouped by
 * kernel class: 0 tile_forward, 1 tile_adjoint, 2 expval, 3 lambda, 4 reduce
 * (all deterministic reductions), 5 build_matrices, 6 dense_k, 7 other.
 * sv_kernel_timing_read synchronises the device, adds the elapsed times of the
 * completed launches to per-class totals and reports them (ms, launches).
 * SV_KERNEL_CLASSES entries each; NULL outputs are skipped.  Reset clears totals.
 * The totals are process-wide: launches of every state and host thread are
 * recorded (under a lock, so concurrent threads may launch while timing). */
#define SV_KERNEL_CLASSES 8
sv_status sv_kernel_timing_enable(int enable);
sv_status sv_kernel_timing_reset(void);
sv_status sv_kernel_timing_read(double *total_ms, int64_t *launches);

/* ---- batched circuits ------------------------------------------------------------- */

typedef struct sv_batch sv_batch; /* opaque: many circuits in one persistent launch */

/* Plan n_circuits circuits for one persistent, CUDA-graph-captured launch
 * (many independent circuits on one device, as in the paper's batched
 * execution of cut-circuit fragments of mixed sizes, Sec. 4.1).  Circuit i acts
 * on n_qubits[i] wires (1..30), runs tapes[i] from |basis_states[i]> (NULL = all
 * |0>) and measures obs[i], one Pauli sum of Z-only words (x_mask = 0;
 * otherwise SV_ERR_UNSUPPORTED), giving one expectation value per circuit.
 * Parameters of circuit i are the next tapes[i].n_params entries of the
 * concatenated parameter vector.  Tapes may repeat (one tape, many parameter
 * sets).  The batch owns its device memory (states of all circuits, tables).
 * SV_MATRIX ops wider than 4 wires are not supported in a batch. */
sv_status sv_batch_create(sv_dtype dtype, int n_circuits, const int *n_qubits, const sv_tape *tapes,
                          const sv_pauli_sum *obs, const uint64_t *basis_states, sv_batch **out);
sv_status sv_batch_destroy(sv_batch *b);
/* Stream for all batch work (NULL: a stream the batch creates; graph capture
 * needs a non-default stream). */
sv_status sv_batch_set_stream(sv_batch *b, void *cuda_stream);
/* Concatenated parameters (sum of tapes[i].n_params doubles), host or device. */
sv_status sv_batch_set_params(sv_batch *b, const double *params, int params_on_device);
/* Run every circuit: expvals_out[i] = <H_i> of circuit i.  Host outputs
 * synchronise and report SV_ERR_TIMEOUT if a bounded inter-CTA wait gave up;
 * device outputs are asynchronous (then check with sv_batch_status). */
sv_status sv_batch_run(sv_batch *b, double *expvals_out, int outputs_on_device);
/* SV_ERR_TIMEOUT if the last run's bounded waits gave up, else SV_OK (synchronises). */
sv_status sv_batch_status(sv_batch *b);
/* Time candidate tile widths and circuit-wave sizes on this device and keep the
 * fastest (the batch's autotuner); *best_ms gets the chosen run time. */
sv_status sv_batch_autotune(sv_batch *b, double *best_ms);
/* Plan facts: work items, persistent CTAs, tile bits, wave bytes, graph in use (0/1). */
sv_status sv_batch_info(const sv_batch *b, int64_t *work_items, int *ctas, int *tile_bits, int64_t *wave_bytes,
                        int *graph);

/* ---- Hermitian observables ------------------------------------------------------ */

/* Host-only (no GPU needed): the Pauli words of a Hermitian 2^k x 2^k matrix A
 * on k wires (an observable given as a matrix, Sec. 2.2), so that sv_expval,
 * sv_var, sv_adjoint_jacobian and the program calls measure it as the
 * Hamiltonian sum_P c_P P.  matrix: host, row-major, interleaved re/im, its
 * index bit k-1-j belonging to wires[j] (wires[0] most significant).
 * c_P = Tr(P A) / 2^k over the 4^k words on the k wires; words with
 * |c_P| <= tol are left out.  coeffs, x_masks, z_masks: caller-owned host
 * arrays of 4^k entries, filled with *n_terms words in sv_pauli_sum form (bit w
 * of a mask is wire w).  SV_ERR_ARG for n outside 1..63, k outside
 * 1..SV_MAX_HERMITIAN_WIRES, wires out of range or repeated, non-finite
 * entries, tol < 0, or A not Hermitian within 1e-12 * max(1, max |A_rc|). */
#define SV_MAX_HERMITIAN_WIRES 5
sv_status sv_hermitian_to_pauli(int n, const int *wires, int k, const double *matrix, double tol, double *coeffs,
                                uint64_t *x_masks, uint64_t *z_masks, int *n_terms);

/* Host-only planner query (no GPU needed): number of fused forward passes and
 * adjoint passes the library would use for a tape on n qubits and dtype. */
sv_status sv_plan_query(int n, sv_dtype dtype, const sv_tape *tape,
                        int *n_forward_passes, int *n_adjoint_passes);

/* Host-only planner description: micro-op counts of the forward and adjoint
 * plans (either array may be NULL), indexed by
 *   0 pair blocks, 1 diagonals, 2 dense blocks in a tile, 3 phase runs
 *   (adjacent RZ / IsingZZ sharing an angle), 4 fused single-wire runs,
 *   5 multi-wire micro-ops (up to 3 single-wire gates per barrier),
 *   6 wide dense steps outside tiles, 7 tile passes.
 * Same argument errors as sv_plan_query. */
#define SV_PLAN_KINDS 8
sv_status sv_plan_describe(int n, sv_dtype dtype, const sv_tape *tape, int forward_counts[SV_PLAN_KINDS],
                           int adjoint_counts[SV_PLAN_KINDS]);

/* ---- expectation values without device allocation ------------------------------ */

/* The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory when they need a measurement (an application that
 * reserved all GPU memory up front, code where cudaMalloc / cudaFree and the
 * device synchronisation of cudaFree are not allowed, or a framework whose
 * allocator must not see foreign allocations).
 *
 * The values of sv_expval, equal within rounding (the same term kernel; the
 * grid, and so the order of the partial sums, may differ), computed for a
 * state given by its device pointer psi (2^n amplitudes of dtype, 16-byte
 * aligned, read only) on cuda_stream (NULL = legacy default stream); results go
 * to the host array out[n_obs] and the call synchronises the stream.  psi must
 * be device (or managed) memory of the current device whose allocation holds
 * 2^n amplitudes from psi on; anything else (a host pointer, another device's
 * memory, a short buffer) is rejected with SV_ERR_ARG before any launch.  Every
 * temporary lives in one array compiled into the library
 * (SV_STATIC_SCRATCH_BYTES on every GPU that loads it, until exit); the call
 * makes no cudaMalloc / cudaFree or other allocation.
 *
 * Limits, rejected with SV_ERR_ARG and a message in sv_last_error(): at most
 * SV_STATIC_MAX_OBSERVABLES observables and SV_STATIC_MAX_TERMS Pauli terms in
 * total per call.  A Pauli word that flips more wires than one tile holds
 * (11 for complex128, 12 for complex64, less 3 or 4 always-local low bits) is
 * rejected with SV_ERR_UNSUPPORTED.
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and keeps it.  The call copies host tables and
 * synchronises its stream, so it must not be called while that stream, or any
 * stream in global capture mode, is capturing.  All calls share the array;
 * calls whose GPU work overlaps race and must be serialised by the caller.
 * The per-term totals are cleared at the start of every call. */
#define SV_STATIC_SCRATCH_BYTES (2u << 20)
#define SV_STATIC_MAX_TERMS 4096
#define SV_STATIC_MAX_OBSERVABLES 1024
sv_status sv_expval_static(const void *psi, int n, sv_dtype dtype, const sv_pauli_sum *obs, int n_obs,
                           double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SV_H */

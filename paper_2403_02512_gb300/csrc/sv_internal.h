// Internal tables shared by the host runtime (sv_api.cu) and the kernel
// launchers (sv_kernels_*.cu).  Plain PODs uploaded to device memory once per
// planned program.  Index convention: "global bit" b is bit b of an amplitude
// index; wire w lives at global bit n-1-w (wire 0 = most significant, Alg. 1).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace sv {

constexpr int kMaxLocalBits = 13;   // tile of up to 2^13 amplitudes
constexpr int kMaxTargets = 6;      // dense ops inside a tile: k <= 4; dense_k kernel: k <= 6
constexpr int kMaxTileTargets = 4;
constexpr int kMaxQubits = 34;
constexpr int kBlock = 256;         // threads per CTA in the tile kernels
constexpr int kMaxLambdaPerCta = 8; // lambdas sharing one phi tile in the adjoint kernel (at most)
constexpr int kMaxTrainPerPass = 32;
constexpr int kNormBlocks = 304;    // partial sums of a renormalisation (fixed count: same order every call)

// Micro-op kinds.  Every structured gate is a set of independent 2x2 blocks on
// amplitude pairs (kPair: e.g. IsingXX = blocks on |00>,|11> and |01>,|10>;
// DoubleExcitation = one block on |0011>,|1100>), or a diagonal (kDiag), or,
// for a user matrix on 2-4 wires, a dense block (kDense).
enum OpKind : int8_t { kPair = 0, kDiag = 1, kDense = 2, kPhase = 3, kMulti = 4 };
// kMulti: k = 2..3 consecutive uncontrolled single-wire pair micro-ops on
// distinct local bits (forward and batch plans): a thread holds the 2^k
// amplitudes its group spans in registers and applies member j (code mcode[j],
// 2x2 entries at mmat[j], local bit tl[j]) in order; ts[] = the bits sorted.
// kPhase: a run of r adjacent Z-parity rotations sharing one angle (RZ,
// IsingZZ; e.g. a QAOA cost layer) as one diagonal.  Member j multiplies by
// exp(-i theta/2 (-1)^p_j) with p_j the parity of the index bits it acts on,
// so the run multiplies by E[k] = exp(-i theta/2 (r - 2k)), k = sum_j p_j.
// Fields: mat = E[0..r]; oa = first member record in the plan's aux table
// (two words each: parity mask over local bits, parity mask over tile bits;
// members with local bits come first); ob = r; zmask = members with local bits.
constexpr int kMaxPhaseMembers = 64;
// 2x2 block structure (of the stored, already adjoint-resolved block).
enum MatCode : int8_t {
  mGen = 0,    // general complex
  mReal = 1,   // real entries (RY, Hadamard, Givens rotations)
  mImOff = 2,  // real diagonal, imaginary off-diagonal (RX, IsingXX/YY/XY blocks)
  mSwap = 3,   // [[0,1],[1,0]] (PauliX, CNOT target, SWAP block)
  mY = 4       // [[0,-i],[i,0]]
};
enum DiagCode : int8_t { dGen = 0, dNeg = 1 /* -1 on the all-ones pattern (Z, CZ) */ };
// Generator block of a trainable op, restricted to the op's pair or diagonal.
enum GenCode : int8_t {
  gNone = 0,
  gX = 1,    // gs * [[0,1],[1,0]] on the pair
  gY = 2,    // gs * [[0,-i],[i,0]] on the pair
  gDiag = 3, // g = ga (even) / gb (odd) by the parity of pattern & zmask
  gHerm = 4  // fused run: ngen general Hermitian 2x2 generators (entries at gmat)
};
// A run of single-wire gates on one wire (no other gate touching the wire in
// between) is applied as one 2x2 block; its trainable members' generators are
// carried to the run's end by conjugation with the members that follow them.
constexpr int kMaxFuseGen = 3;      // trainable members per fused run
constexpr int kMaxFuseMembers = 8;  // members per fused run

// One micro-op of one pass.
struct OpDev {
  int8_t kind, code, gcode, k;
  int8_t ts[4];          // kPair / kDense: local target bits, ascending
  int8_t tl[4];          // kDense: local bit of target j (j = 0 is the op's local MSB)
  int8_t tg[kMaxTargets];// kDiag / dense_k: global bit of target j
  int8_t sync_prev;      // barrier needed between the previous micro-op and this one
  int8_t ngen;           // gHerm: generators (trainable indices train .. train + ngen - 1)
  int32_t oa, ob;        // kPair: local offsets of the two members within a group
  int32_t zmask;         // gDiag: target-pattern bits whose parity selects gb
  int32_t train;         // trainable index within the pass, or -1
  int32_t mat;           // matrix entries: kPair 4 (2x2 block), kDiag 2^k, kDense / dense_k 4^k
  int32_t slot;          // global trainable slot, or -1
  float gs, ga, gb;
  int32_t gmat;          // gHerm: first generator (4 entries each, row-major)
  uint64_t cmask, cval;  // control bits (global) and their required values
  // The same controls split by the pass's tiles: local bits (as local-index
  // bits) vary inside a tile; the others are fixed per tile.
  uint32_t lcmask, lcval;
  uint64_t hcmask, hcval;
  int8_t mcode[3];       // kMulti: member codes
  int8_t fused;          // kPair made from a fused run of single-wire gates (1), for plan descriptions
  int32_t mmat[3];       // kMulti: member 2x2 entries
};

// One fused pass: a tile is the set of 2^T amplitudes that share every index
// bit outside the local bits pos[0..T).
struct PassDev {
  int32_t T;                       // local bits
  int32_t nlow;                    // pos[i] == i for i < nlow (contiguous low bits)
  int32_t pos[kMaxLocalBits];      // global bit of local bit i (ascending)
  int32_t nhi;                     // n - T
  int32_t hi[kMaxQubits];          // global bits that index tiles (ascending)
  int32_t op_begin, op_end;        // ops [op_begin, op_end) of the program's op table
  int32_t n_train;                 // trainable ops in this pass
  int32_t train_base;              // row of the first trainable op in the pass's partial block
  int32_t max_k;                   // widest kDense op in the pass (selects the kernel variant)
  int32_t zonly;                   // expectation pass whose words all have x = 0 (Z letters only)
};

// One Pauli term placed in an expectation / lambda pass.
struct TermDev {
  uint64_t xg, zg;   // global-bit masks (X/Y flip bits; Y/Z sign bits)
  uint32_t xl;       // the flip mask in local bits of the pass
  int32_t ny;        // number of Y letters mod 4
  int32_t obs;       // observable (row) index
  uint32_t zl;       // the sign mask in local bits of the pass
  double coeff;
};

// Gate-matrix slot built on the device from the parameter vector: the op's
// matrix E = U, or U^dagger when `dagger` (op's own adjoint flag XOR the
// adjoint sweep), written whole (mode 0), as its diagonal (1) or as the 2x2
// block on members (a, b) (2).  A fused run (mode 3) takes its members from
// slots [a, a + b) (mode 4, forward order, `dagger` = the member's own adjoint
// flag) and writes the run's product (adjoint when `dagger`) plus, for each
// trainable member (a = generator code gX / gY / gDiag with g0, g1 = gs or
// ga, gb), the conjugated generator at the member's `out`.  A phase run
// (mode 5, b = r members sharing this slot's angle) writes E[0..r].
struct MatSlot {
  int32_t kind;        // sv_op_kind
  int32_t k;
  int32_t dagger;
  int32_t mode;
  int32_t a, b;
  int32_t out;         // offset (complex entries) in the matrix buffer
  int32_t pidx[3];
  double scale;
  double cangle[3];
  int64_t src;         // SV_MATRIX: offset (complex entries) of the user matrix
  double g0, g1;       // mode 4: generator parameters
};

// A pass that holds one pair or diagonal micro-op runs straight from HBM
// (Alg. 2's enumeration: the unit index gets a zero inserted at every fixed
// bit, then the fixed values are or-ed in).  Pair units are the op's amplitude
// pairs; diagonal units are the amplitudes it scales.
struct StreamDev {
  int32_t kind, code, k;  // kPair (code) or kDiag (code, k <= 2 targets)
  int32_t nfix;           // fixed index bits (targets of a pair, controls, dNeg targets), ascending
  int8_t fix[16];
  uint64_t fixval;        // required values of the fixed bits
  uint64_t oa, ob;        // kPair: global offsets of the two members
  int32_t tg0, tg1;       // kDiag: global bits of the targets (entry = bit(tg0) [, bit(tg1)])
  int32_t mat;            // entries in the matrix buffer
  int32_t vec2;           // complex64: bit 0 is free, two adjacent units per 16-byte access
  int32_t pair16;         // complex64 pair on bit 0 alone: both members in one 16-byte access
};

// A sparse observable in device memory (CSR, 2^n rows, complex FP64 values).
struct SparseDev {
  int32_t n;
  int32_t pad;
  double nnz_per_row;      // mean stored entries per row (selects the lanes per row)
  const int64_t *indptr;   // 2^n + 1
  const int64_t *indices;  // nnz
  const double2 *vals;     // nnz
};

// Marginal probabilities of k wires: enumeration index j = bin * 2^(n-k) + other,
// amplitude index = `other` with zeros inserted at the wires' bits (ascending
// pos) or-ed with bin's bits placed at bitpos[0..k) (bitpos[0] = most
// significant bin bit).
struct ProbsDev {
  int32_t n, k, chunk_log;
  int32_t pad;
  int8_t pos[kMaxQubits];     // the wires' global bits, ascending
  int8_t bitpos[kMaxQubits];  // global bit of bin bit k-1-j for j = 0..k-1 (wires order)
};
constexpr int kMaxProbWires = 24;   // 2^24 bins at most
constexpr int kProbsSmallLog = 6;   // bins of <= 64 amplitudes: one thread per bin

// Deterministic inclusive prefix sum of m doubles in place (three fixed levels,
// `scratch` >= ceil(m / 4096) doubles), and inverse-transform sampling.
cudaError_t inclusive_scan(double *x, int64_t m, double *scratch, cudaStream_t st);
cudaError_t probs_combine(const double *partials, int64_t bins, int per_bin, double *out, cudaStream_t st);
cudaError_t sample_cdf(const double *cdf, int64_t m, const double *u, int64_t shots, uint64_t *out, cudaStream_t st);

// ---- batched circuits -------------------------------------------------------
// One circuit of a batch: its passes, its Z-only observable and its state slice.
struct BatchCircuit {
  int32_t n;
  int32_t pass_begin, n_pass;   // passes [pass_begin, pass_begin + n_pass) of the batch pass table
  int32_t term_begin, n_terms;  // Z words of its observable in the batch term table
  int32_t out;                  // index of its expectation value
  int32_t tiles;                // tiles per pass (2^(n - T); the same T for all its passes)
  int32_t pad;
  int64_t part_begin;           // partials [part_begin, + n_terms * tiles): one per (term, tile)
  uint64_t state_off;           // amplitude offset of its state in the state pool
  uint64_t basis;               // initial basis state
};

// A run of consecutive work items: every tile of pass `pass` of circuit `circ`.
struct BatchSeg {
  int64_t first_item;
  int32_t circ, pass;
  int32_t ntiles, pad;
};

struct ZTerm {
  uint64_t z;     // amplitude-index bits of the Z word
  double coeff;
};

// Launchers (defined once per precision in sv_kernels_{f32,f64,df}.cu, the adjoint
// launcher in sv_kernels_{f32,f64,df}_adjoint.cu).
// R = float (complex64) or double (complex128).  Every launcher returns the
// cudaError_t of its launch.
template <typename R>
struct Launch {
  static cudaError_t build_matrices(const MatSlot *slots, int n_slots, const double *params,
                                    const double *user_mats, void *mats, cudaStream_t st);
  static cudaError_t tile_forward(void *psi, int n, const PassDev &pass, const OpDev *ops,
                                  const void *mats, const uint64_t *aux, int grid, cudaStream_t st);
  // m lambdas, b of them per CTA (grid.x = ceil(m / b) lambda groups).
  static cudaError_t tile_adjoint(const void *phi_in, void *phi_out, void *lam, int n, int m, int b,
                                  const PassDev &pass, const OpDev *ops, const void *mats, const uint64_t *aux,
                                  double *partials, int grid, cudaStream_t st);
  static cudaError_t expval_pass(const void *psi, int n, const PassDev &pass, const TermDev *terms,
                                 int n_terms, double *partials, int grid, cudaStream_t st);
  // Expectation values of n_obs observables over the words placed in one pass,
  // words grouped by observable ([obs_term_begin[o], obs_term_begin[o + 1]) of
  // terms): FP64 partials[block * n_obs + o].
  static cudaError_t expval_obs_pass(const void *psi, int n, const PassDev &pass, const TermDev *terms,
                                     const int32_t *obs_term_begin, int n_obs, double *partials, int grid,
                                     cudaStream_t st);
  static cudaError_t lambda_pass(const void *phi, void *lam, int n, const PassDev &pass,
                                 const TermDev *terms, const int32_t *obs_term_begin, int n_obs,
                                 int first, int grid, cudaStream_t st);
  static cudaError_t dense_k(void *psi, int n, const OpDev &op, const void *mats, int adjoint,
                             cudaStream_t st);
  static cudaError_t set_basis(void *psi, int n, uint64_t index, cudaStream_t st);
  static cudaError_t stream_op(void *psi, int n, const StreamDev &sd, const void *mats, cudaStream_t st);
  // psi <- psi / ||psi|| (||psi||^2 in FP64 over kNormBlocks fixed partials in `scratch`).
  static cudaError_t renormalize(void *psi, int n, double *scratch, cudaStream_t st);
  // kNormBlocks FP64 partials of ||psi||^2 (fixed order).
  static cudaError_t norm_partials(const void *psi, int n, double *partials, cudaStream_t st);
  // Marginal-probability partials: partials[c] = sum of |psi_i|^2 over chunk c of 2^chunk_log
  // consecutive (bin, other) indices, bin = the bits at the wires (see ProbsDev).
  static cudaError_t probs_partials(const void *psi, const ProbsDev &pd, double *partials, cudaStream_t st);
  // Tangent pass (forward-mode JVP): psi and dpsi through one pass; coefs[slot] complex.
  static cudaError_t tile_tangent(void *psi, void *dpsi, int n, const PassDev &pass, const OpDev *ops,
                                  const void *mats, const double2 *coefs, int grid, cudaStream_t st);
  // kNormBlocks FP64 partials of Re <a|b> (fixed order).
  static cudaError_t dot_partials(const void *a, const void *b, int n, double *partials, cudaStream_t st);
  // Sparse (CSR) observable, 2^n rows: lambda = H psi, or kNormBlocks partials of Re <psi|H psi>.
  static cudaError_t csr_spmv(const void *psi, const SparseDev &h, void *out, cudaStream_t st);
  static cudaError_t csr_expval_partials(const void *psi, const SparseDev &h, double *partials, cudaStream_t st);
  // Bins of <= 2^kProbsSmallLog amplitudes: out[bin] directly, one thread per bin.
  static cudaError_t probs_small(const void *psi, const ProbsDev &pd, double *out, cudaStream_t st);
  // Persistent batch launch: `grid` CTAs drain the work items of all segments.
  static cudaError_t batch(void *states, const BatchCircuit *circs, const PassDev *passes, const OpDev *ops,
                           const void *mats, const uint64_t *aux, const BatchSeg *segs, int n_segs, int64_t total_items,
                           const ZTerm *terms, double *partials, int *done, unsigned long long *head, int *err,
                           int store_final, unsigned long long timeout_ns, int max_T, int max_terms, int max_k,
                           int no_publish, int grid, cudaStream_t st);
  static int batch_blocks_per_sm(int max_T, int max_terms, int max_k);
  static cudaError_t copy(void *dst, const void *src, int n, cudaStream_t st);
  static int max_T_forward();
  static int max_T_adjoint();
  // lambdas per adjoint CTA (largest compiled variant) and resident adjoint CTAs per SM
  static int adj_lambdas_max();
  static int adj_ctas_per_sm();
};

// Batch: out[c.out] = sum_term coeff * sum_tile partials (fixed order), one thread per circuit.
// Tensor-core application of a dense 5-qubit block to a complex64 state (sv_tc.cu).
cudaError_t dense5_tc(void *psi, int n, const OpDev &op, const void *mats, int adjoint, cudaStream_t st);
int dense5_tc_take_error();  // 1 if a tensor-core wait ran out since the last call (clears it)
void dense5_tc_enable(bool on);
bool dense5_tc_enabled();

// out[j0 + j] = 2 sum_b partials[j * nb + b], j < m (Jacobian-vector products).
// out[j0 + j] = scale * sum over b < nb of partials[j * nb + b] (fixed order).
cudaError_t jvp_combine(const double *partials, int nb, int m, int j0, double *out, cudaStream_t st,
                        double scale = 2.0);
// out[j0 + j] = sum_b partials[j * nb + b] - E[j0 + j]^2, j < m (variances).
cudaError_t var_combine(const double *partials, int nb, int m, const double *E, int j0, double *out, cudaStream_t st);
cudaError_t batch_reduce(const BatchCircuit *circs, int n_circ, const ZTerm *terms, const double *partials,
                         double *out, cudaStream_t st);

// Message returned by sv_last_error() on the calling thread (defined in sv_api.cu).
void set_error_message(const char *msg);

// Deterministic reductions (precision independent, sv_kernels_f64.cu).
// out[r] = sum_{b < nb} partials[b * stride + r] for r < rows, fixed order.
cudaError_t reduce_rows(const double *partials, int nb, int rows, int stride, double *out,
                        cudaStream_t st);
// out[(row0 + t) * ldo + col0 + j] = sum_b partials[b * (m * n_rows) + j * n_rows + t].
cudaError_t reduce_partials(const double *partials, int nb, int m, int n_rows, double *out, int ldo,
                            int row0, int col0, cudaStream_t st);
// expvals[o] = sum_t coeff_t * sums[t] over terms t of observable o (fixed order).
cudaError_t combine_terms(const double *term_sums, const TermDev *terms, const int32_t *obs_begin,
                          int n_obs, const int32_t *term_order, double *expvals, cudaStream_t st);
// J[j * n_params + p] = sum_{s in slots_of(p)} coef[s] * contrib[s * m + j]  (CSR over p).
cudaError_t assemble_jacobian(const double *contrib, const double *coef, const int32_t *p_begin,
                              const int32_t *p_slots, int n_params, int m, int row0, int ldj,
                              double *J, cudaStream_t st);

}  // namespace sv

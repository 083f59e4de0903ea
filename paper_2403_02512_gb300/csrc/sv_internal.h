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

// Op classes inside a pass.
enum OpClass : int32_t {
  kDense = 0,  // 2^k x 2^k matrix on k local target bits
  kDiag = 1,   // 2^k diagonal on k target bits anywhere in the index
};

// One op of one pass.  Matrices live in the program's matrix buffer, indexed in
// complex entries of the state's precision.
struct OpDev {
  int32_t cls;
  int32_t k;
  int32_t tl[kMaxTargets];  // kDense: local bit of target j (j = 0 is the op's local MSB)
  int32_t tg[kMaxTargets];  // kDiag:  global bit of target j
  uint64_t cmask;           // control bits (global)
  uint64_t cval;            // required values of the control bits
  int32_t mat;              // U: 4^k (dense) or 2^k (diag) entries
  int32_t gen;              // generator G (same shape as U) or -1
  int32_t train;            // index among the pass's trainable ops, or -1
  int32_t slot;             // contribution slot (expanded-op index), or -1
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
  int32_t max_k;                   // widest dense op in the pass (selects the kernel variant)
};

// One Pauli term placed in an expectation / lambda pass.
struct TermDev {
  uint64_t xg, zg;   // global-bit masks (X/Y flip bits; Y/Z sign bits)
  uint32_t xl;       // the flip mask in local bits of the pass
  int32_t ny;        // number of Y letters mod 4
  int32_t obs;       // observable (row) index
  int32_t pad;
  double coeff;
};

// Gate-matrix slot built on the device from the parameter vector.
struct MatSlot {
  int32_t kind;        // sv_op_kind
  int32_t k;
  int32_t adjoint;
  int32_t diag;        // write the 2^k diagonal only
  int32_t what;        // 0 = U, 1 = generator G
  int32_t out;         // offset (complex entries) in the matrix buffer
  int32_t pidx[3];
  int32_t pad;
  double scale;
  double cangle[3];
  int64_t src;         // SV_MATRIX: offset (complex entries) of the user matrix
};

// Launchers (defined once per precision in sv_kernels_f32.cu / sv_kernels_f64.cu).
// R = float (complex64) or double (complex128).  Every launcher returns the
// cudaError_t of its launch.
template <typename R>
struct Launch {
  static cudaError_t build_matrices(const MatSlot *slots, int n_slots, const double *params,
                                    const double *user_mats, void *mats, cudaStream_t st);
  static cudaError_t tile_forward(void *psi, int n, const PassDev &pass, const OpDev *ops,
                                  const void *mats, int grid, cudaStream_t st);
  static cudaError_t tile_adjoint(const void *phi_in, void *phi_out, void *lam, int n, int m,
                                  const PassDev &pass, const OpDev *ops, const void *mats,
                                  double *partials, int grid, cudaStream_t st);
  static cudaError_t expval_pass(const void *psi, int n, const PassDev &pass, const TermDev *terms,
                                 int n_terms, double *partials, int grid, cudaStream_t st);
  static cudaError_t lambda_pass(const void *phi, void *lam, int n, const PassDev &pass,
                                 const TermDev *terms, const int32_t *obs_term_begin, int n_obs,
                                 int first, int grid, cudaStream_t st);
  static cudaError_t dense_k(void *psi, int n, const OpDev &op, const void *mats, int adjoint,
                             cudaStream_t st);
  static cudaError_t set_basis(void *psi, int n, uint64_t index, cudaStream_t st);
  static cudaError_t copy(void *dst, const void *src, int n, cudaStream_t st);
  static int forward_smem(int T);
  static int adjoint_smem(int T);
  static int expval_smem(int T, int n_terms);
  static int max_T_forward();
  static int max_T_adjoint();
};

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

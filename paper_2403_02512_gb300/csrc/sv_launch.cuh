// Launcher definitions of Launch<R>; included once per precision.
//
// SV_LAUNCH_PART selects which launchers a translation unit defines, so that
// one precision compiles as two units in parallel (an explicit instantiation
// of Launch<R> instantiates only the members defined before it):
//   0 (default)  every launcher;
//   1            every launcher but tile_adjoint;
//   2            tile_adjoint alone (the adjoint kernel's variants).
#pragma once

#ifndef SV_LAUNCH_PART
#define SV_LAUNCH_PART 0
#endif

#include "sv_kernels.cuh"

namespace sv {

namespace detail {
inline int tile_bytes(int elem, int T) { return elem << T; }
inline int lut_bytes(const PassDev &p) { return 8 << (p.T - p.nlow); }
constexpr int kWarps = kBlock / 32;
constexpr int kMaxDynSmem = 227 * 1024;

// Opt in to large dynamic shared memory: the per-block limit minus the
// kernel's own static shared memory.
template <typename Kern>
inline void allow_big_smem(Kern k, bool &done) {
  if (!done) {
    cudaFuncAttributes fa;
    int stat = 0;
    if (cudaFuncGetAttributes(&fa, k) == cudaSuccess) stat = (int)fa.sharedSizeBytes;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem - stat);
    cudaGetLastError();
    done = true;
  }
}
}  // namespace detail

#if SV_LAUNCH_PART != 2
template <typename R>
cudaError_t Launch<R>::build_matrices(const MatSlot *slots, int n_slots, const double *params,
                                      const double *user_mats, void *mats, cudaStream_t st) {
  if (n_slots <= 0) return cudaSuccess;
  const int tpb = 64;
  k_build_matrices<R><<<(n_slots + tpb - 1) / tpb, tpb, 0, st>>>(slots, n_slots, params, user_mats,
                                                                   reinterpret_cast<c_t<R> *>(mats));
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::tile_forward(void *psi, int n, const PassDev &pass, const OpDev *ops,
                                    const void *mats, const uint64_t *aux, int grid, cudaStream_t st) {
  static bool attr2 = false, attr4 = false;
  const int smem = detail::tile_bytes(sizeof(c_t<R>), pass.T) + detail::lut_bytes(pass);
  if (pass.max_k <= 2) {
    detail::allow_big_smem(k_tile_forward<R, 2>, attr2);
    k_tile_forward<R, 2><<<grid, kBlock, smem, st>>>(reinterpret_cast<g_t<R> *>(psi), n, pass, ops,
                                                      reinterpret_cast<const c_t<R> *>(mats), aux);
  } else {
    detail::allow_big_smem(k_tile_forward<R, 4>, attr4);
    k_tile_forward<R, 4><<<grid, kBlock, smem, st>>>(reinterpret_cast<g_t<R> *>(psi), n, pass, ops,
                                                      reinterpret_cast<const c_t<R> *>(mats), aux);
  }
  return cudaGetLastError();
}

#endif  // SV_LAUNCH_PART != 2

#if SV_LAUNCH_PART != 1
namespace detail {
template <typename R, int MAXK, int B>
cudaError_t adjoint_b(const void *phi_in, void *phi_out, void *lam, int n, int m, const PassDev &pass,
                      const OpDev *ops, const void *mats, const uint64_t *aux, double *partials, int grid,
                      cudaStream_t st) {
  static bool attr = false;
  const int smem = (1 + B) * tile_bytes(sizeof(c_t<R>), pass.T) + lut_bytes(pass) + pass.n_train * B * kWarps * 8;
  allow_big_smem(k_tile_adjoint<R, MAXK, B>, attr);
  dim3 g((m + B - 1) / B, grid);
  k_tile_adjoint<R, MAXK, B><<<g, kBlock, smem, st>>>(
      reinterpret_cast<const g_t<R> *>(phi_in), reinterpret_cast<g_t<R> *>(phi_out), reinterpret_cast<g_t<R> *>(lam),
      n, m, pass, ops, reinterpret_cast<const c_t<R> *>(mats), aux, partials);
  return cudaGetLastError();
}

template <typename R, int MAXK>
cudaError_t adjoint_k(const void *phi_in, void *phi_out, void *lam, int n, int m, int b, const PassDev &pass,
                      const OpDev *ops, const void *mats, const uint64_t *aux, double *partials, int grid,
                      cudaStream_t st) {
  switch (b) {
    case 1: return adjoint_b<R, MAXK, 1>(phi_in, phi_out, lam, n, m, pass, ops, mats, aux, partials, grid, st);
    case 2: return adjoint_b<R, MAXK, 2>(phi_in, phi_out, lam, n, m, pass, ops, mats, aux, partials, grid, st);
    case 4: return adjoint_b<R, MAXK, 4>(phi_in, phi_out, lam, n, m, pass, ops, mats, aux, partials, grid, st);
    case 8:
      if constexpr (std::is_same<R, double>::value)
        return adjoint_b<R, MAXK, 8>(phi_in, phi_out, lam, n, m, pass, ops, mats, aux, partials, grid, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;  // lambdas per CTA: 1, 2, 4 (8: complex128)
  }
}
}  // namespace detail

template <typename R>
cudaError_t Launch<R>::tile_adjoint(const void *phi_in, void *phi_out, void *lam, int n, int m, int b,
                                    const PassDev &pass, const OpDev *ops, const void *mats, const uint64_t *aux,
                                    double *partials, int grid, cudaStream_t st) {
  if (pass.max_k <= 2)
    return detail::adjoint_k<R, 2>(phi_in, phi_out, lam, n, m, b, pass, ops, mats, aux, partials, grid, st);
  return detail::adjoint_k<R, 4>(phi_in, phi_out, lam, n, m, b, pass, ops, mats, aux, partials, grid, st);
}

#endif  // SV_LAUNCH_PART != 1

#if SV_LAUNCH_PART != 2
template <typename R>
cudaError_t Launch<R>::stream_op(void *psi, int n, const StreamDev &sd, const void *mats, cudaStream_t st) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const uint64_t units = 1ull << (n - sd.nfix);
  const uint64_t per_thread = (sd.vec2 ? 2 : 1) * kStreamUnroll;
  const uint64_t want = (units + per_thread * kBlock - 1) / (per_thread * kBlock);
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * (2048 / kBlock)));
  g_t<R> *p = reinterpret_cast<g_t<R> *>(psi);
  const c_t<R> *m = reinterpret_cast<const c_t<R> *>(mats);
  if (sd.kind == kPair) {
    switch (sd.code) {
      case mSwap: k_stream_pair<R, mSwap><<<grid, kBlock, 0, st>>>(p, units, sd, m); break;
      case mY: k_stream_pair<R, mY><<<grid, kBlock, 0, st>>>(p, units, sd, m); break;
      case mReal: k_stream_pair<R, mReal><<<grid, kBlock, 0, st>>>(p, units, sd, m); break;
      case mImOff: k_stream_pair<R, mImOff><<<grid, kBlock, 0, st>>>(p, units, sd, m); break;
      default: k_stream_pair<R, mGen><<<grid, kBlock, 0, st>>>(p, units, sd, m); break;
    }
  } else if (sd.code == dNeg) {
    k_stream_diag<R, 1, true><<<grid, kBlock, 0, st>>>(p, units, sd, m);
  } else if (sd.k == 1) {
    k_stream_diag<R, 1, false><<<grid, kBlock, 0, st>>>(p, units, sd, m);
  } else {
    k_stream_diag<R, 2, false><<<grid, kBlock, 0, st>>>(p, units, sd, m);
  }
  return cudaGetLastError();
}

namespace detail {
template <typename R, int NB>
cudaError_t expval_z(const void *psi, int n, const PassDev &pass, const TermDev *terms, int n_terms,
                     double *partials, int grid, cudaStream_t st) {
  static bool attr = false;
  allow_big_smem(k_expval_z<R, NB>, attr);
  const int smem = lut_bytes(pass) + (int)sizeof(R) * (kBlock << NB) + kZChunk * (8 + 4) + n_terms * kWarps * 8;
  k_expval_z<R, NB><<<grid, kBlock, smem, st>>>(reinterpret_cast<const g_t<R> *>(psi), n, pass, terms, n_terms,
                                                 partials);
  return cudaGetLastError();
}
}  // namespace detail

template <typename R>
cudaError_t Launch<R>::expval_pass(const void *psi, int n, const PassDev &pass, const TermDev *terms,
                                   int n_terms, double *partials, int grid, cudaStream_t st) {
  if (pass.zonly) {  // words with Z letters only: one transform of |psi|^2 per thread and tile
    switch (pass.T) {
      case 8: return detail::expval_z<R, 0>(psi, n, pass, terms, n_terms, partials, grid, st);
      case 9: return detail::expval_z<R, 1>(psi, n, pass, terms, n_terms, partials, grid, st);
      case 10: return detail::expval_z<R, 2>(psi, n, pass, terms, n_terms, partials, grid, st);
      case 11: return detail::expval_z<R, 3>(psi, n, pass, terms, n_terms, partials, grid, st);
      case 12: return detail::expval_z<R, 4>(psi, n, pass, terms, n_terms, partials, grid, st);
      default: break;  // tiles of fewer than 256 amplitudes: the general kernel
    }
  }
  static bool attr = false;
  detail::allow_big_smem(k_expval<R>, attr);
  const int smem = detail::tile_bytes(sizeof(c_t<R>), pass.T) + detail::lut_bytes(pass) +
                   n_terms * detail::kWarps * 8;
  k_expval<R><<<grid, kBlock, smem, st>>>(reinterpret_cast<const g_t<R> *>(psi), n, pass, terms, n_terms,
                                           partials);
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::expval_obs_pass(const void *psi, int n, const PassDev &pass, const TermDev *terms,
                                       const int32_t *obs_term_begin, int n_obs, double *partials, int grid,
                                       cudaStream_t st) {
  static bool attr[5] = {false, false, false, false, false};
  const int smem = detail::tile_bytes(sizeof(c_t<R>), pass.T) + detail::lut_bytes(pass) + n_obs * detail::kWarps * 8;
  const int na = pass.T > 8 ? 1 << (pass.T - 8) : 1;  // amplitudes per thread (kBlock = 256)
  auto go = [&](auto kern, bool &done) {
    detail::allow_big_smem(kern, done);
    kern<<<grid, kBlock, smem, st>>>(reinterpret_cast<const g_t<R> *>(psi), n, pass, terms, obs_term_begin, n_obs,
                                     partials);
    return cudaGetLastError();
  };
  switch (na) {
    case 1: return go(k_expval_obs<R, 1>, attr[0]);
    case 2: return go(k_expval_obs<R, 2>, attr[1]);
    case 4: return go(k_expval_obs<R, 4>, attr[2]);
    case 8: return go(k_expval_obs<R, 8>, attr[3]);
    case 16: return go(k_expval_obs<R, 16>, attr[4]);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t Launch<R>::lambda_pass(const void *phi, void *lam, int n, const PassDev &pass,
                                   const TermDev *terms, const int32_t *obs_term_begin, int n_obs,
                                   int first, int grid, cudaStream_t st) {
  static bool attr[5] = {false, false, false, false, false};
  const int smem = detail::tile_bytes(sizeof(c_t<R>), pass.T) + detail::lut_bytes(pass);
  const int na = pass.T > 8 ? 1 << (pass.T - 8) : 1;  // amplitudes per thread (kBlock = 256)
  dim3 g(grid, n_obs);
  auto go = [&](auto kern, bool &done) {
    detail::allow_big_smem(kern, done);
    kern<<<g, kBlock, smem, st>>>(reinterpret_cast<const g_t<R> *>(phi), reinterpret_cast<g_t<R> *>(lam), n, pass,
                                  terms, obs_term_begin, first);
    return cudaGetLastError();
  };
  switch (na) {
    case 1: return go(k_lambda<R, 1>, attr[0]);
    case 2: return go(k_lambda<R, 2>, attr[1]);
    case 4: return go(k_lambda<R, 4>, attr[2]);
    case 8: return go(k_lambda<R, 8>, attr[3]);
    case 16: return go(k_lambda<R, 16>, attr[4]);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t Launch<R>::dense_k(void *psi, int n, const OpDev &op, const void *mats, int adjoint,
                               cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value) {
    if (op.k == 5 && n >= 5 && dense5_tc_enabled()) return dense5_tc(psi, n, op, mats, adjoint, st);
  }
  const uint64_t groups = 1ull << (n - op.k);
  const int gpb = kBlock >> op.k;
  uint64_t blocks = (groups + gpb - 1) / gpb;
  if (blocks > 65535ull * 16) blocks = 65535ull * 16;
  k_dense_k<R><<<(unsigned)blocks, kBlock, 0, st>>>(reinterpret_cast<g_t<R> *>(psi), n, op,
                                                     reinterpret_cast<const c_t<R> *>(mats) + op.mat, adjoint);
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::set_basis(void *psi, int n, uint64_t index, cudaStream_t st) {
  const uint64_t N = 1ull << n;
  uint64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_set_basis<R><<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<g_t<R> *>(psi), N, index);
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::renormalize(void *psi, int n, double *scratch, cudaStream_t st) {
  const uint64_t N = 1ull << n;
  g_t<R> *p = reinterpret_cast<g_t<R> *>(psi);
  k_norm_partials<R><<<kNormBlocks, kBlock, 0, st>>>(p, N, scratch);
  k_norm_scale<R><<<kNormBlocks, kBlock, 0, st>>>(p, N, scratch, kNormBlocks);
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::norm_partials(const void *psi, int n, double *partials, cudaStream_t st) {
  k_norm_partials<R><<<kNormBlocks, kBlock, 0, st>>>(reinterpret_cast<const g_t<R> *>(psi), 1ull << n, partials);
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::probs_partials(const void *psi, const ProbsDev &pd, double *partials, cudaStream_t st) {
  const uint64_t blocks = 1ull << (pd.n - pd.chunk_log);
  k_probs_partials<R><<<(unsigned)blocks, kBlock, 0, st>>>(reinterpret_cast<const g_t<R> *>(psi), pd, partials);
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::tile_tangent(void *psi, void *dpsi, int n, const PassDev &pass, const OpDev *ops,
                                    const void *mats, const double2 *coefs, int grid, cudaStream_t st) {
  static bool attr2 = false, attr4 = false;
  const int smem = 2 * detail::tile_bytes(sizeof(c_t<R>), pass.T) + detail::lut_bytes(pass);
  g_t<R> *p = reinterpret_cast<g_t<R> *>(psi), *d = reinterpret_cast<g_t<R> *>(dpsi);
  const c_t<R> *m = reinterpret_cast<const c_t<R> *>(mats);
  if (pass.max_k <= 2) {
    detail::allow_big_smem(k_tile_tangent<R, 2>, attr2);
    k_tile_tangent<R, 2><<<grid, kBlock, smem, st>>>(p, d, n, pass, ops, m, coefs);
  } else {
    detail::allow_big_smem(k_tile_tangent<R, 4>, attr4);
    k_tile_tangent<R, 4><<<grid, kBlock, smem, st>>>(p, d, n, pass, ops, m, coefs);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::dot_partials(const void *a, const void *b, int n, double *partials, cudaStream_t st) {
  k_dot_partials<R><<<kNormBlocks, kBlock, 0, st>>>(reinterpret_cast<const g_t<R> *>(a),
                                                    reinterpret_cast<const g_t<R> *>(b), 1ull << n, partials);
  return cudaGetLastError();
}

namespace detail {
// Lanes per sparse row: the power of two >= the mean row length, 1..32.
inline int csr_group(const SparseDev &h) {
  const double mean = h.nnz_per_row;
  int g = 1;
  while (g < 32 && g < mean) g <<= 1;
  return g;
}
}  // namespace detail

template <typename R>
cudaError_t Launch<R>::csr_spmv(const void *psi, const SparseDev &h, void *out, cudaStream_t st) {
  const g_t<R> *p = reinterpret_cast<const g_t<R> *>(psi);
  g_t<R> *o = reinterpret_cast<g_t<R> *>(out);
  switch (detail::csr_group(h)) {
    case 1: k_csr_spmv<R, 1><<<kNormBlocks, kBlock, 0, st>>>(p, h, o); break;
    case 2: k_csr_spmv<R, 2><<<kNormBlocks, kBlock, 0, st>>>(p, h, o); break;
    case 4: k_csr_spmv<R, 4><<<kNormBlocks, kBlock, 0, st>>>(p, h, o); break;
    case 8: k_csr_spmv<R, 8><<<kNormBlocks, kBlock, 0, st>>>(p, h, o); break;
    case 16: k_csr_spmv<R, 16><<<kNormBlocks, kBlock, 0, st>>>(p, h, o); break;
    default: k_csr_spmv<R, 32><<<kNormBlocks, kBlock, 0, st>>>(p, h, o); break;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::csr_expval_partials(const void *psi, const SparseDev &h, double *partials, cudaStream_t st) {
  const g_t<R> *p = reinterpret_cast<const g_t<R> *>(psi);
  switch (detail::csr_group(h)) {
    case 1: k_csr_expval_partials<R, 1><<<kNormBlocks, kBlock, 0, st>>>(p, h, partials); break;
    case 2: k_csr_expval_partials<R, 2><<<kNormBlocks, kBlock, 0, st>>>(p, h, partials); break;
    case 4: k_csr_expval_partials<R, 4><<<kNormBlocks, kBlock, 0, st>>>(p, h, partials); break;
    case 8: k_csr_expval_partials<R, 8><<<kNormBlocks, kBlock, 0, st>>>(p, h, partials); break;
    case 16: k_csr_expval_partials<R, 16><<<kNormBlocks, kBlock, 0, st>>>(p, h, partials); break;
    default: k_csr_expval_partials<R, 32><<<kNormBlocks, kBlock, 0, st>>>(p, h, partials); break;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::probs_small(const void *psi, const ProbsDev &pd, double *out, cudaStream_t st) {
  const uint64_t bins = 1ull << pd.k;
  k_probs_small<R><<<(unsigned)((bins + kBlock - 1) / kBlock), kBlock, 0, st>>>(reinterpret_cast<const g_t<R> *>(psi),
                                                                               pd, out);
  return cudaGetLastError();
}

template <typename R>
int Launch<R>::batch_blocks_per_sm(int max_T, int max_terms, int max_k) {
  const int smem = (int)((sizeof(c_t<R>) + 8) << max_T) + max_terms * (detail::kWarps + 1) * 8;
  // the occupancy query honours the dynamic shared-memory opt-in: set it first
  static bool attr2 = false, attr4 = false;
  if (max_k <= 2)
    detail::allow_big_smem(k_batch<R, 2>, attr2);
  else
    detail::allow_big_smem(k_batch<R, 4>, attr4);
  int nb = 0;
  cudaError_t e = max_k <= 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<R, 2>, kBlock, smem)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<R, 4>, kBlock, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

template <typename R>
cudaError_t Launch<R>::batch(void *states, const BatchCircuit *circs, const PassDev *passes, const OpDev *ops,
                             const void *mats, const uint64_t *aux, const BatchSeg *segs, int n_segs, int64_t total_items,
                             const ZTerm *terms, double *partials, int *done, unsigned long long *head, int *err,
                             int store_final, unsigned long long timeout_ns, int max_T, int max_terms, int max_k,
                             int no_publish, int grid, cudaStream_t st) {
  static bool attr2 = false, attr4 = false;
  const int smem = (int)((sizeof(c_t<R>) + 8) << max_T) + max_terms * (detail::kWarps + 1) * 8;
  if (max_k <= 2) {
    detail::allow_big_smem(k_batch<R, 2>, attr2);
    k_batch<R, 2><<<grid, kBlock, smem, st>>>(reinterpret_cast<g_t<R> *>(states), circs, passes, ops,
                                               reinterpret_cast<const c_t<R> *>(mats), aux, segs, n_segs,
                                               (long long)total_items, terms, partials, done, head, err, store_final,
                                               timeout_ns, max_T, max_terms, no_publish);
  } else {
    detail::allow_big_smem(k_batch<R, 4>, attr4);
    k_batch<R, 4><<<grid, kBlock, smem, st>>>(reinterpret_cast<g_t<R> *>(states), circs, passes, ops,
                                               reinterpret_cast<const c_t<R> *>(mats), aux, segs, n_segs,
                                               (long long)total_items, terms, partials, done, head, err, store_final,
                                               timeout_ns, max_T, max_terms, no_publish);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t Launch<R>::copy(void *dst, const void *src, int n, cudaStream_t st) {
  return cudaMemcpyAsync(dst, src, sizeof(g_t<R>) << n, cudaMemcpyDeviceToDevice, st);
}

// Tile sizes: 32 KiB of amplitudes per tile in the forward / expval kernels,
// 2 x 16 KiB (phi + lambda) in the adjoint kernel.
template <typename R>
int Launch<R>::max_T_forward() {
  return sizeof(c_t<R>) == 8 ? 12 : 11;
}

template <typename R>
int Launch<R>::max_T_adjoint() {
  return sizeof(c_t<R>) == 8 ? 11 : 10;
}

// FP64 arithmetic runs at a small fraction of the FP32 rate, so eight warps
// per SM keep its pipe busy: the complex128 adjoint kernel runs one CTA per SM
// with up to 255 registers and 8 lambdas per phi tile (less phi work per lambda).
template <typename R>
int Launch<R>::adj_lambdas_max() {
  return std::is_same<R, double>::value ? 8 : 4;
}

template <typename R>
int Launch<R>::adj_ctas_per_sm() {
  return std::is_same<R, double>::value ? 1 : 2;
}
#endif  // SV_LAUNCH_PART != 2

}  // namespace sv

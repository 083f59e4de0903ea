// complex128 instantiation of the state-vector kernels, plus the
// precision-independent deterministic reductions.
#define SV_LAUNCH_PART 1  // tile_adjoint: sv_kernels_f64_adjoint.cu
#include "sv_launch.cuh"

namespace sv {
template struct Launch<double>;

// Fixed-order sum over b of partials[b * (m * n_rows) + j * n_rows + t] into
// out[(row0 + t) * ldo + col0 + j]: one thread per (j, t), b ascending.  The
// same inputs always give bitwise-equal outputs.
__global__ void k_reduce_partials(const double *__restrict__ partials, int nb, int m, int n_rows,
                                  double *__restrict__ out, int ldo, int row0, int col0) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m * n_rows) return;
  const int j = r / n_rows, t = r % n_rows;
  const size_t stride = (size_t)m * n_rows;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partials[(size_t)b * stride + r];
  out[(size_t)(row0 + t) * ldo + col0 + j] = s;
}

cudaError_t reduce_rows(const double *partials, int nb, int rows, int stride, double *out,
                        cudaStream_t st) {
  (void)stride;
  if (rows <= 0) return cudaSuccess;
  k_reduce_partials<<<(rows + 127) / 128, 128, 0, st>>>(partials, nb, 1, rows, out, 1, 0, 0);
  return cudaGetLastError();
}

cudaError_t reduce_partials(const double *partials, int nb, int m, int n_rows, double *out, int ldo,
                            int row0, int col0, cudaStream_t st) {
  const int total = m * n_rows;
  if (total <= 0) return cudaSuccess;
  k_reduce_partials<<<(total + 127) / 128, 128, 0, st>>>(partials, nb, m, n_rows, out, ldo, row0, col0);
  return cudaGetLastError();
}

// expvals[o] = sum_{i in [obs_begin[o], obs_begin[o+1])} coeff(term_order[i]) * sums[term_order[i]]
__global__ void k_combine_terms(const double *__restrict__ sums, const TermDev *__restrict__ terms,
                                const int32_t *__restrict__ obs_begin, int n_obs,
                                const int32_t *__restrict__ order, double *__restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_obs) return;
  double e = 0.0;
  for (int i = obs_begin[o]; i < obs_begin[o + 1]; ++i) {
    const int t = order[i];
    e += terms[t].coeff * sums[t];
  }
  out[o] = e;
}

cudaError_t combine_terms(const double *term_sums, const TermDev *terms, const int32_t *obs_begin,
                          int n_obs, const int32_t *term_order, double *expvals, cudaStream_t st) {
  if (n_obs <= 0) return cudaSuccess;
  k_combine_terms<<<(n_obs + 127) / 128, 128, 0, st>>>(term_sums, terms, obs_begin, n_obs, term_order,
                                                        expvals);
  return cudaGetLastError();
}

// J[(row0 + j) * ldj + p] = sum over slots s of parameter p (CSR, sweep order) of
// coef[s] * contrib[s * m + j].
__global__ void k_assemble_jacobian(const double *__restrict__ contrib, const double *__restrict__ coef,
                                    const int32_t *__restrict__ p_begin, const int32_t *__restrict__ p_slots,
                                    int n_params, int m, int row0, int ldj, double *__restrict__ J) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_params * m) return;
  const int j = i / n_params, p = i % n_params;
  double v = 0.0;
  for (int q = p_begin[p]; q < p_begin[p + 1]; ++q) {
    const int s = p_slots[q];
    v += coef[s] * contrib[(size_t)s * m + j];
  }
  J[(size_t)(row0 + j) * ldj + p] = v;
}

cudaError_t assemble_jacobian(const double *contrib, const double *coef, const int32_t *p_begin,
                              const int32_t *p_slots, int n_params, int m, int row0, int ldj,
                              double *J, cudaStream_t st) {
  const int total = n_params * m;
  if (total <= 0) return cudaSuccess;
  k_assemble_jacobian<<<(total + 127) / 128, 128, 0, st>>>(contrib, coef, p_begin, p_slots, n_params, m,
                                                            row0, ldj, J);
  return cudaGetLastError();
}

// Jacobian-vector products: out = 2 Re <lambda_j | dpsi>, partials ascending.
__global__ void k_jvp_combine(const double *__restrict__ partials, int nb, int m, int j0, double scale,
                              double *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += partials[(size_t)j * nb + b];
  out[j0 + j] = scale * t;
}

cudaError_t jvp_combine(const double *partials, int nb, int m, int j0, double *out, cudaStream_t st, double scale) {
  if (m <= 0) return cudaSuccess;
  k_jvp_combine<<<(m + 127) / 128, 128, 0, st>>>(partials, nb, m, j0, scale, out);
  return cudaGetLastError();
}

// Variances: one thread per observable, partials summed in ascending order.
__global__ void k_var_combine(const double *__restrict__ partials, int nb, int m, const double *__restrict__ E, int j0,
                              double *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += partials[(size_t)j * nb + b];
  const double e = E[j0 + j];
  out[j0 + j] = t - e * e;
}

cudaError_t var_combine(const double *partials, int nb, int m, const double *E, int j0, double *out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  k_var_combine<<<(m + 127) / 128, 128, 0, st>>>(partials, nb, m, E, j0, out);
  return cudaGetLastError();
}

// Probabilities: out[bin] = its per_bin consecutive partials, ascending.
__global__ void k_probs_combine(const double *__restrict__ partials, int64_t bins, int per_bin, double *__restrict__ out) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= bins) return;
  double t = 0.0;
  for (int c = 0; c < per_bin; ++c) t += partials[b * per_bin + c];
  out[b] = t;
}

cudaError_t probs_combine(const double *partials, int64_t bins, int per_bin, double *out, cudaStream_t st) {
  if (bins <= 0) return cudaSuccess;
  k_probs_combine<<<(unsigned)((bins + 255) / 256), 256, 0, st>>>(partials, bins, per_bin, out);
  return cudaGetLastError();
}

// Inclusive scan of one 4096-element segment per 1024-thread block: each
// thread sums its 4 elements in order, a Hillis-Steele scan over the 1024
// thread sums (fixed steps), then each thread writes its 4 running sums.
// totals[block] = the segment's sum.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanSeg = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) k_scan_segments(double *__restrict__ x, int64_t m,
                                                                double *__restrict__ totals) {
  __shared__ double sh[2][kScanThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanSeg + (int64_t)threadIdx.x * kScanPer;
  double v[kScanPer];
  double run = 0.0;
  for (int e = 0; e < kScanPer; ++e) {
    v[e] = base + e < m ? x[base + e] : 0.0;
    run += v[e];
  }
  int cur = 0;
  sh[0][threadIdx.x] = run;
  __syncthreads();
  for (int d = 1; d < kScanThreads; d <<= 1) {
    const double a = sh[cur][threadIdx.x];
    const double b = threadIdx.x >= (unsigned)d ? sh[cur][threadIdx.x - d] : 0.0;
    sh[cur ^ 1][threadIdx.x] = threadIdx.x >= (unsigned)d ? b + a : a;
    cur ^= 1;
    __syncthreads();
  }
  double pre = threadIdx.x > 0 ? sh[cur][threadIdx.x - 1] : 0.0;  // exclusive prefix of this thread
  for (int e = 0; e < kScanPer; ++e) {
    pre += v[e];
    if (base + e < m) x[base + e] = pre;
  }
  if (threadIdx.x == kScanThreads - 1 && totals) totals[blockIdx.x] = sh[cur][threadIdx.x];
}

__global__ void k_scan_add(double *__restrict__ x, int64_t m, const double *__restrict__ offsets) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t seg = i / kScanSeg;
  if (seg > 0) x[i] += offsets[seg - 1];
}

// Three fixed levels: segments of 4096, their totals (<= 4096 segments, one
// block), offsets added back.  m <= 2^24.
cudaError_t inclusive_scan(double *x, int64_t m, double *scratch, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int64_t segs = (m + kScanSeg - 1) / kScanSeg;
  if (segs > kScanSeg) return cudaErrorInvalidValue;
  k_scan_segments<<<(unsigned)segs, kScanThreads, 0, st>>>(x, m, segs > 1 ? scratch : nullptr);
  if (segs > 1) {
    k_scan_segments<<<1, kScanThreads, 0, st>>>(scratch, segs, nullptr);
    k_scan_add<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(x, m, scratch);
  }
  return cudaGetLastError();
}

// out[t] = first b with cdf[b] > u[t] * cdf[m - 1] (clamped to m - 1).
__global__ void k_sample_cdf(const double *__restrict__ cdf, int64_t m, const double *__restrict__ u, int64_t shots,
                             uint64_t *__restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= shots) return;
  const double target = u[t] * cdf[m - 1];
  int64_t lo = 0, hi = m - 1;  // answer in [lo, hi]
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (cdf[mid] > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  out[t] = (uint64_t)lo;
}

cudaError_t sample_cdf(const double *cdf, int64_t m, const double *u, int64_t shots, uint64_t *out, cudaStream_t st) {
  if (shots <= 0) return cudaSuccess;
  k_sample_cdf<<<(unsigned)((shots + 255) / 256), 256, 0, st>>>(cdf, m, u, shots, out);
  return cudaGetLastError();
}

// Batch: out[c.out] = sum_t coeff_t * sum_tile partials[part_begin + t * tiles + tile].
// One warp per circuit: lane l sums tiles l, l + 32, ... in ascending order,
// a fixed shuffle tree combines the lanes, terms are added in ascending order.
__global__ void k_batch_reduce(const BatchCircuit *__restrict__ circs, int n_circ, const ZTerm *__restrict__ terms,
                               const double *__restrict__ partials, double *__restrict__ out) {
  const int c = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= n_circ) return;
  const BatchCircuit cc = circs[c];
  double e = 0.0;
  for (int t = 0; t < cc.n_terms; ++t) {
    double v = 0.0;
    const double *p = partials + cc.part_begin + (int64_t)t * cc.tiles;
    for (int i = lane; i < cc.tiles; i += 32) v += p[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    e += terms[cc.term_begin + t].coeff * v;  // lane 0 holds the tile sum
  }
  if (lane == 0) out[cc.out] = e;
}

cudaError_t batch_reduce(const BatchCircuit *circs, int n_circ, const ZTerm *terms, const double *partials,
                         double *out, cudaStream_t st) {
  if (n_circ <= 0) return cudaSuccess;
  k_batch_reduce<<<(n_circ + 3) / 4, 128, 0, st>>>(circs, n_circ, terms, partials, out);
  return cudaGetLastError();
}

}  // namespace sv

// Pauli-sum expectation values with no device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// measurement: an application that reserved the whole GPU up front and hands
// memory to nobody, code running where cudaMalloc / cudaFree would stall the
// device (cudaFree synchronises it), or a framework whose allocator must not
// see foreign allocations.  For them sv_expval_static computes the values of
// sv_expval (the same term kernel; equal within rounding, since the grid and
// so the order of the partial sums may differ) with every temporary (the term
// table, the per-block partial sums and the per-term totals) in one fixed
// array compiled into the library.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its SV_STATIC_SCRATCH_BYTES until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device
// current) and keeps it.  The call copies its term tables from host memory and
// synchronises its stream, so it must not be called while that stream, or any
// stream in global capture mode, is capturing.  All calls share the array, so
// calls whose GPU work overlaps (on different streams, or from several
// threads) race; serialise them.
//
// Before any launch the call checks that psi is device memory of the current
// device and that its allocation holds 2^n amplitudes from psi on
// (cudaPointerGetAttributes, and the driver's cuMemGetAddressRange looked up
// through the runtime so that the library does not link libcuda); neither
// check allocates.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "sv.h"
#include "sv_internal.h"

using namespace sv;

namespace {

constexpr size_t kTermBytes = sizeof(TermDev) * SV_STATIC_MAX_TERMS;
constexpr int kPassTerms = 512;       // terms per expectation pass (shared-memory accumulators)
constexpr int kMaxGrid = 304;         // CTAs per expectation pass (2 per SM on a GB300)
constexpr size_t kPartialBytes = sizeof(double) * (size_t)kMaxGrid * kPassTerms;
constexpr size_t kSumBytes = sizeof(double) * SV_STATIC_MAX_TERMS;
constexpr size_t kObsBytes = sizeof(double) * SV_STATIC_MAX_OBSERVABLES;
constexpr size_t kIndexBytes = sizeof(int32_t) * (SV_STATIC_MAX_OBSERVABLES + 1 + SV_STATIC_MAX_TERMS);

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffTerms = 0;
constexpr size_t kOffPartials = kOffTerms + align256(kTermBytes);
constexpr size_t kOffSums = kOffPartials + align256(kPartialBytes);
constexpr size_t kOffObs = kOffSums + align256(kSumBytes);
constexpr size_t kOffIndex = kOffObs + align256(kObsBytes);
constexpr size_t kUsed = kOffIndex + align256(kIndexBytes);
static_assert(kUsed <= SV_STATIC_SCRATCH_BYTES, "static scratch layout exceeds SV_STATIC_SCRATCH_BYTES");

// The scratch itself: one per device, for the life of the process.
static __device__ __align__(256) unsigned char g_static_scratch[SV_STATIC_SCRATCH_BYTES];

sv_status fail(sv_status st, const char *msg) {
  set_error_message(msg);
  return st;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Once per device, with that device current: the device address of the array.
sv_status scratch_address(char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(SV_ERR_CUDA, "sv_expval_static: no current CUDA device");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(SV_ERR_CUDA, "sv_expval_static: cudaGetSymbolAddress of the scratch array failed");
    }
    g_scratch_ptr[dev] = p;
  }
  *out = (char *)g_scratch_ptr[dev];
  return SV_OK;
}

// The driver's cuMemGetAddressRange (base and size of the allocation holding an
// address), through the runtime's entry-point lookup: no link-time libcuda.
typedef CUresult (*AddressRangeFn)(CUdeviceptr *base, size_t *size, CUdeviceptr dptr);
std::once_flag g_range_once;
AddressRangeFn g_range_fn = nullptr;

// psi must be device (or managed) memory of the current device, with
// `bytes` bytes of its allocation from psi on.
sv_status check_state_memory(const void *psi, size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(SV_ERR_CUDA, "sv_expval_static: no current CUDA device");
  }
  cudaPointerAttributes a;
  memset(&a, 0, sizeof(a));
  if (cudaPointerGetAttributes(&a, psi) != cudaSuccess) {
    cudaGetLastError();
    return fail(SV_ERR_ARG, "sv_expval_static: psi is not an address CUDA knows");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(SV_ERR_ARG, "sv_expval_static: psi is not device memory");
  if (a.type == cudaMemoryTypeDevice && a.device != dev)
    return fail(SV_ERR_ARG, "sv_expval_static: psi is memory of another device than the current one");
  std::call_once(g_range_once, [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_range_fn = (AddressRangeFn)fn;
    cudaGetLastError();
  });
  if (!g_range_fn) return fail(SV_ERR_CUDA, "sv_expval_static: cuMemGetAddressRange is unavailable");
  CUdeviceptr base = 0;
  size_t size = 0;
  if (g_range_fn(&base, &size, (CUdeviceptr)(uintptr_t)psi) != CUDA_SUCCESS)
    return fail(SV_ERR_ARG, "sv_expval_static: psi lies in no device allocation");
  const uint64_t p = (uint64_t)(uintptr_t)psi;
  if (p < base || bytes > size || p - base > size - bytes)
    return fail(SV_ERR_ARG, "sv_expval_static: psi's allocation holds fewer than 2^n amplitudes from psi on");
  return SV_OK;
}

struct Term {
  int obs;
  double coeff;
  uint64_t x, z;  // amplitude-index bits
  int ny;
};

uint64_t to_index_bits(uint64_t wire_mask, int n) {
  uint64_t g = 0;
  for (int w = 0; w < n; ++w)
    if (wire_mask >> w & 1) g |= 1ull << (n - 1 - w);
  return g;
}

int popc(uint64_t v) { return __builtin_popcountll(v); }

PassDev make_pass(int n, uint64_t bits) {
  PassDev p;
  memset(&p, 0, sizeof(p));
  for (int b = 0; b < n; ++b) {
    if (bits >> b & 1)
      p.pos[p.T++] = b;
    else
      p.hi[p.nhi++] = b;
  }
  while (p.nlow < p.T && p.pos[p.nlow] == p.nlow) ++p.nlow;
  p.max_k = 1;
  return p;
}

uint64_t fill_low(uint64_t bits, int n, int T) {
  for (int b = 0; b < n && popc(bits) < T; ++b) bits |= 1ull << b;
  return bits;
}

}  // namespace

extern "C" {

sv_status sv_expval_static(const void *psi, int n, sv_dtype dtype, const sv_pauli_sum *obs, int n_obs,
                           double *out, void *cuda_stream) {
  if (!psi || !out || (n_obs > 0 && !obs)) return fail(SV_ERR_ARG, "sv_expval_static: NULL argument");
  if (((uintptr_t)psi) & 15) return fail(SV_ERR_ARG, "sv_expval_static: psi must be 16-byte aligned");
  if (n < 1 || n > SV_MAX_QUBITS) return fail(SV_ERR_ARG, "sv_expval_static: n out of range");
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "sv_expval_static: unknown dtype");
  if (n_obs < 0 || n_obs > SV_STATIC_MAX_OBSERVABLES)
    return fail(SV_ERR_ARG, "sv_expval_static: more observables than SV_STATIC_MAX_OBSERVABLES");
  if (n_obs == 0) return SV_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (sv_status s = check_state_memory(psi, (size_t)(dtype == SV_C64 ? 8 : 16) << n)) return s;

  // terms in index-bit form
  std::vector<Term> terms;
  const uint64_t valid = (1ull << n) - 1;
  for (int o = 0; o < n_obs; ++o) {
    const sv_pauli_sum &H = obs[o];
    if (H.n_terms < 0 || (H.n_terms > 0 && (!H.coeffs || !H.x_mask || !H.z_mask)))
      return fail(SV_ERR_ARG, "sv_expval_static: bad observable arrays");
    if ((long)terms.size() + H.n_terms > SV_STATIC_MAX_TERMS)
      return fail(SV_ERR_ARG, "sv_expval_static: more Pauli terms in total than SV_STATIC_MAX_TERMS");
    for (int t = 0; t < H.n_terms; ++t) {
      if ((H.x_mask[t] | H.z_mask[t]) & ~valid) return fail(SV_ERR_ARG, "sv_expval_static: term acts on a wire >= n");
      if (!std::isfinite(H.coeffs[t])) return fail(SV_ERR_ARG, "sv_expval_static: coefficient not finite");
      terms.push_back({o, H.coeffs[t], to_index_bits(H.x_mask[t], n), to_index_bits(H.z_mask[t], n),
                       popc(H.x_mask[t] & H.z_mask[t]) & 3});
    }
  }

  // passes: each term's flip bits must be local bits of its pass (the lowest
  // index bits are always local for coalesced, 16-byte aligned tile rows)
  const int Tmax = dtype == SV_C64 ? Launch<float>::max_T_forward() : Launch<double>::max_T_forward();
  const int nlow = dtype == SV_C64 ? 4 : 3;
  const int T = std::min(Tmax, n);
  std::vector<PassDev> passes;
  std::vector<int> begin(1, 0), placed;
  std::vector<char> done(terms.size(), 0);
  size_t left = terms.size();
  while (left > 0) {
    uint64_t bits = 0;
    for (int b = 0; b < nlow && b < n && b < T; ++b) bits |= 1ull << b;
    int cnt = 0;
    for (size_t t = 0; t < terms.size() && cnt < kPassTerms; ++t) {
      if (done[t]) continue;
      if (popc(bits | terms[t].x) <= T) {
        bits |= terms[t].x;
        done[t] = 1;
        placed.push_back((int)t);
        ++cnt;
        --left;
      }
    }
    if (cnt == 0) return fail(SV_ERR_UNSUPPORTED, "sv_expval_static: a Pauli word flips too many wires");
    passes.push_back(make_pass(n, fill_low(bits, n, T)));
    begin.push_back((int)placed.size());
  }

  std::vector<TermDev> tdev(placed.size());
  std::vector<int> dev_index(terms.size(), 0);
  for (size_t q = 0; q + 1 < begin.size(); ++q)
    for (int i = begin[q]; i < begin[q + 1]; ++i) {
      const Term &h = terms[placed[i]];
      TermDev &t = tdev[i];
      memset(&t, 0, sizeof(t));
      t.xg = h.x;
      t.zg = h.z;
      for (int b = 0; b < passes[q].T; ++b) {
        if (h.x >> passes[q].pos[b] & 1) t.xl |= 1u << b;
        if (h.z >> passes[q].pos[b] & 1) t.zl |= 1u << b;
      }
      t.ny = h.ny;
      t.obs = h.obs;
      t.coeff = h.coeff;
      dev_index[placed[i]] = i;
    }
  std::vector<int32_t> index(n_obs + 1 + terms.size(), 0);  // obs_begin, then term order
  for (const Term &h : terms) index[h.obs + 1]++;
  for (int o = 0; o < n_obs; ++o) index[o + 1] += index[o];
  {
    std::vector<int32_t> fill(index.begin(), index.begin() + n_obs);
    for (size_t t = 0; t < terms.size(); ++t) index[n_obs + 1 + fill[terms[t].obs]++] = dev_index[t];
  }

  char *base = nullptr;
  if (sv_status s = scratch_address(&base)) return s;
  TermDev *d_terms = (TermDev *)(base + kOffTerms);
  double *d_partials = (double *)(base + kOffPartials);
  double *d_sums = (double *)(base + kOffSums);
  double *d_obs = (double *)(base + kOffObs);
  int32_t *d_index = (int32_t *)(base + kOffIndex);

  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t tiles = 1ull << (n - T);
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, std::min(kMaxGrid, 2 * sms)));

  cudaError_t e = cudaSuccess;
  if (!tdev.empty()) e = cudaMemcpyAsync(d_terms, tdev.data(), tdev.size() * sizeof(TermDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_index, index.data(), index.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_sums, 0, kSumBytes, st);  // per-term totals start at zero
  for (size_t q = 0; q + 1 < begin.size() && e == cudaSuccess; ++q) {
    const int b0 = begin[q], cnt = begin[q + 1] - b0;
    e = dtype == SV_C64
            ? Launch<float>::expval_pass(psi, n, passes[q], d_terms + b0, cnt, d_partials, grid, st)
            : Launch<double>::expval_pass(psi, n, passes[q], d_terms + b0, cnt, d_partials, grid, st);
    if (e == cudaSuccess) e = reduce_partials(d_partials, grid, 1, cnt, d_sums, 1, b0, 0, st);
  }
  if (e == cudaSuccess) e = combine_terms(d_sums, d_terms, d_index, n_obs, d_index + n_obs + 1, d_obs, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_obs, sizeof(double) * n_obs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error_message((std::string("sv_expval_static: ") + cudaGetErrorString(e)).c_str());
    return SV_ERR_CUDA;
  }
  return SV_OK;
}

}  // extern "C"

// Tensor-core path for a dense 5-qubit block on a complex64 state (a user
// matrix on 5 wires, 32 x 32 complex, applied to every group of 32 amplitudes
// that share the other index bits; Sec. 2.1.2's generic many-qubit gate).
//
// As a real GEMM per tile of 128 groups:  D (128 x 64) = X (128 x 64) * Ur^T,
// where row g of X holds group g's 32 amplitudes (real and imaginary parts)
// and Ur (64 x 64), built from Re U and Im U, maps them to the outputs' real
// and imaginary parts.  Inputs are ordered along K as (member pair s, member
// of the pair, re / im): k = 4 s + 2 h + c, with the pair bit pb the member bit
// of the target on global index bit 0 when there is one.  Then each 16-byte
// segment of a row is two amplitudes adjacent in memory, and the operand is
// gathered with cp.async (all copies in flight) before one pass splits it
// into TF32 halves; other target sets gather element by element.  Outputs
// along N are (member, re / im) in member order.  One tcgen05.mma (kind::tf32, M = 128, N = 64, K = 8)
// per 8 columns of K; FP32 accuracy from three products of TF32 halves,
// hi*hi + hi*lo + lo*hi (x = hi + lo, each rounded to TF32), accumulated in
// FP32 in tensor memory.  Operands sit in shared memory in the no-swizzle
// K-major layout of 8-row x 16-byte core matrices; the accumulator (128
// lanes x 64 FP32 columns) is read back by each warp's 32 lanes with
// tcgen05.ld.  The wait for the MMAs is bounded: past the limit the kernel
// sets an error flag and stops.
#include "sv_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

namespace sv {
namespace {

constexpr int kTcRows = 128;              // groups per tile (MMA M)
constexpr int kTcK = 64;                  // 32 real + 32 imaginary inputs
constexpr int kTcN = 64;                  // 32 real + 32 imaginary outputs
constexpr int kTcThreads = 256;           // eight warps; warps w and w + 4 read TMEM lanes 32(w % 4) ..
constexpr int kOpBytesA = kTcRows * kTcK * 4;  // 32 KB per TF32 operand half
constexpr int kOpBytesB = kTcN * kTcK * 4;     // 16 KB
constexpr int kSBO = (kTcK / 4) * 128;         // bytes between 8-row core-matrix blocks
constexpr int kLBO = 128;                      // bytes between core matrices along K
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s bound on the MMA wait

__device__ int g_tc_error;  // set when a wait ran out; read and cleared by the host

// Byte offset of element (row, k) in the K-major core-matrix layout.
__device__ __forceinline__ int kmajor_off(int row, int k) {
  return (row >> 3) * kSBO + (k >> 2) * kLBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x = hi + lo, both TF32.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - hi);
}

// K position of member m's real part (imaginary part: + 1).
__device__ __forceinline__ int kpos(int m, int pb) {
  const int s = ((m >> (pb + 1)) << pb) | (m & ((1 << pb) - 1));
  return 4 * s + 2 * ((m >> pb) & 1);
}

__device__ __forceinline__ void cp_async16_zfill(uint32_t saddr, const void *gaddr, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(gaddr), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void st_shared_f32(uint32_t addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns_tc() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 16 FP32 columns of this warp's 32 TMEM lanes; the wait takes the registers
// as operands, so no use of them can be scheduled before the load completes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Group base index of group g: g's bits dealt, in order, to the index bits that
// are not targets (zeros inserted at the ascending target bits).  Linear over
// disjoint bit sets, so the base of tile * 128 + row is D(tile << 7) | D(row).
__device__ __forceinline__ uint64_t deposit(uint64_t x, const int (&sorted)[5]) {
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int b = sorted[j];
    x = ((x >> b) << (b + 1)) | (x & ((1ull << b) - 1));
  }
  return x;
}

__device__ __forceinline__ void cp_async8_zfill(uint32_t saddr, const void *gaddr, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(saddr), "l"(gaddr), "r"(src_bytes) : "memory");
}

// Shared memory of the kernel (bytes from the 1024-aligned base).
constexpr int kOffRaw = 0;                          // two raw operand buffers (cp.async targets)
constexpr int kOffAhi = kOffRaw + 2 * kOpBytesA;    // TF32 halves of the operand
constexpr int kOffAlo = kOffAhi + kOpBytesA;
constexpr int kOffBhi = kOffAlo + kOpBytesA;        // TF32 halves of the matrix
constexpr int kOffBlo = kOffBhi + kOpBytesB;
constexpr int kOffStage = kOffBlo + kOpBytesB;      // outputs [group][member], float2 (SEG layout)
constexpr int kOffOffs = kOffStage + kTcRows * 32 * 8;   // member offsets (global index bits), 32 x u64
constexpr int kOffDrow = kOffOffs + 32 * 8;              // group-base deposits of the tile's rows, 128 x u64
constexpr int kOffMbar = kOffDrow + kTcRows * 8;
constexpr int kSmemBytes = kOffMbar + 16;

// Pipelined over the CTA's tiles (one CTA per SM, persistent): while tile i is
// split into TF32 halves and its MMAs run, tile i + 1 is in flight to the
// other raw buffer (cp.async) and tile i - 1 is read back from the other
// accumulator (two 64-column TMEM buffers) and stored.  SEG: a target is on
// global index bit 0, so members pair up in 16-byte segments (gathered in
// 16-byte copies, outputs staged and stored with lane = member); otherwise
// consecutive groups are adjacent in memory and gather and store run with
// lane = group (the store straight from registers).
template <bool SEG>
__global__ void __launch_bounds__(kTcThreads, 1) k_dense5_tc(float2 *__restrict__ psi, int n, const OpDev op,
                                                             const float2 *__restrict__ M, int dagger, int pb) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t sbase = smem_u32(smem);
  const uint32_t raw[2] = {sbase + kOffRaw, sbase + kOffRaw + kOpBytesA};
  const uint32_t a_hi = sbase + kOffAhi, a_lo = sbase + kOffAlo, b_hi = sbase + kOffBhi, b_lo = sbase + kOffBlo;
  float2 *stage = reinterpret_cast<float2 *>(smem + kOffStage);
  uint64_t *offs = reinterpret_cast<uint64_t *>(smem + kOffOffs);
  uint64_t *drow = reinterpret_cast<uint64_t *>(smem + kOffDrow);
  const uint32_t mbar = sbase + kOffMbar;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffMbar + 8);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  int sorted[5];
  for (int j = 0; j < 5; ++j) sorted[j] = op.tg[j];
  for (int i = 1; i < 5; ++i)
    for (int j = i; j > 0 && sorted[j - 1] > sorted[j]; --j) {
      const int t = sorted[j];
      sorted[j] = sorted[j - 1];
      sorted[j - 1] = t;
    }
  if (threadIdx.x < 32) {  // member m (wire order: bit 4 - j of m is target j)
    uint64_t o = 0;
    for (int j = 0; j < 5; ++j)
      if ((threadIdx.x >> (4 - j)) & 1) o |= 1ull << op.tg[j];
    offs[threadIdx.x] = o;
  }
  if (threadIdx.x < kTcRows) drow[threadIdx.x] = deposit((uint64_t)threadIdx.x, sorted);

  // B halves: row nn = 2 o + c' (output member o, re / im), column k(i, c), K-major.
  for (int e = threadIdx.x; e < kTcN * 32; e += blockDim.x) {
    const int nn = e >> 5, i = e & 31;
    const int o = nn >> 1, co = nn & 1;
    const float2 u = dagger ? make_float2(M[i * 32 + o].x, -M[i * 32 + o].y) : M[o * 32 + i];
    const int k = kpos(i, pb);
    const float vr = co == 0 ? u.x : u.y;   // coefficient of the input's real part
    const float vi = co == 0 ? -u.y : u.x;  // ... of its imaginary part
    float hi, lo;
    split_tf32(vr, hi, lo);
    st_shared_f32(b_hi + kmajor_off(nn, k), hi);
    st_shared_f32(b_lo + kmajor_off(nn, k), lo);
    split_tf32(vi, hi, lo);
    st_shared_f32(b_hi + kmajor_off(nn, k + 1), hi);
    st_shared_f32(b_lo + kmajor_off(nn, k + 1), lo);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const uint64_t ngroups = 1ull << (n - 5);
  const uint64_t ntiles = (ngroups + kTcRows - 1) / kTcRows;
  const int niter = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;

  // Issue the copies of tile `tile` into raw buffer `dst` (all asynchronous).
  auto gather = [&](uint64_t tile, uint32_t dst) {
    const uint64_t dt = deposit(tile << 7, sorted);
    if constexpr (SEG) {
      // 16-byte segment seg (members m, m + 2^pb) of rows c * 8 + (lane % 8), c in this warp half's 8
      const int seg = (warp & 3) * 4 + (lane >> 3);
      const int m = ((seg >> pb) << (pb + 1)) | (seg & ((1 << pb) - 1));
      const uint64_t om = offs[m];
#pragma unroll 4
      for (int c = (warp >> 2) * 8; c < (warp >> 2) * 8 + 8; ++c) {
        const int row = c * 8 + (lane & 7);
        const bool ok = tile * kTcRows + row < ngroups;
        cp_async16_zfill(dst + kmajor_off(row, 4 * seg), psi + (ok ? (dt | drow[row] | om) : 0), ok ? 16 : 0);
      }
    } else {
      // lane = group (row (warp % 4) * 32 + lane): member m of 32 consecutive groups per
      // instruction, members split between the two warps of a row quarter
      const int row = (warp & 3) * 32 + lane;
      const bool ok = tile * kTcRows + row < ngroups;
      const uint64_t base = dt | drow[row];
#pragma unroll 4
      for (int m = (warp >> 2) * 16; m < (warp >> 2) * 16 + 16; ++m)
        cp_async8_zfill(dst + kmajor_off(row, 2 * m), psi + (ok ? (base | offs[m]) : 0), ok ? 8 : 0);
    }
  };

  if (niter > 0) gather(blockIdx.x, raw[0]);
  asm volatile("cp.async.commit_group;" ::: "memory");
  uint32_t phase = 0;
  bool failed = false;
  for (int it = 0; it <= niter; ++it) {
    const bool cur = it < niter, prev = it > 0;
    if (it + 1 < niter) gather(blockIdx.x + (uint64_t)(it + 1) * gridDim.x, raw[(it + 1) & 1]);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // tile it has landed
    __syncthreads();
    if (prev) {  // tile it - 1's MMAs: A may be overwritten, its accumulator read
      const unsigned long long t0 = global_ns_tc();
      while (!mbar_try_wait(mbar, phase)) {
        if (global_ns_tc() - t0 > kWaitNs) {
          failed = true;
          break;
        }
      }
      phase ^= 1;
      if (__syncthreads_or(failed)) {
        if (threadIdx.x == 0) atomicExch(&g_tc_error, 1);
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (cur) {
      // split: a_hi <- TF32(x), a_lo <- TF32(x - hi), element by element in the K-major layout
      const float4 *src = reinterpret_cast<const float4 *>(smem + kOffRaw + (it & 1) * kOpBytesA);
      float4 *hi4 = reinterpret_cast<float4 *>(smem + kOffAhi), *lo4 = reinterpret_cast<float4 *>(smem + kOffAlo);
#pragma unroll 4
      for (int c = threadIdx.x; c < kOpBytesA / 16; c += blockDim.x) {
        float4 x = src[c], lo;
        split_tf32(x.x, x.x, lo.x);
        split_tf32(x.y, x.y, lo.y);
        split_tf32(x.z, x.z, lo.z);
        split_tf32(x.w, x.w, lo.w);
        hi4[c] = x;
        lo4[c] = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t as[3] = {a_hi, a_hi, a_lo}, bs[3] = {b_hi, b_lo, b_hi};
        const uint32_t dcol = tmem + (uint32_t)((it & 1) * kTcN);
        for (int pr = 0; pr < 3; ++pr)
          for (int ks = 0; ks < kTcK / 8; ++ks)  // K = 8 per MMA: two core matrices along K
            mma_tf32(dcol, mat_desc(as[pr] + ks * 2 * kLBO), mat_desc(bs[pr] + ks * 2 * kLBO), (pr | ks) != 0);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                     : "memory");
      }
    }
    if (prev) {
      // epilogue of tile it - 1: warp w reads rows 32(w % 4) .. (its TMEM lane quarter),
      // columns 32(w / 4) .. + 31 (outputs 16(w / 4) .. + 15)
      const uint64_t tile = blockIdx.x + (uint64_t)(it - 1) * gridDim.x;
      const int half = warp >> 2;
      const uint32_t scol = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(((it - 1) & 1) * kTcN + half * 32);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float d[kTcN / 2];
#pragma unroll
      for (int c = 0; c < kTcN / 32; ++c) {
        float v[16];
        tmem_ld16(scol + (uint32_t)(c * 16), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) d[c * 16 + i] = v[i];
      }
      const int row = (warp & 3) * 32 + lane;
      const uint64_t dt = deposit(tile << 7, sorted);
      if constexpr (SEG) {
        // members adjacent in memory: staged (index row * 32 + (member ^ (row % 32)),
        // conflict-free both ways), then stored lane = member, one group per step
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int mi = half * 16 + i;
          stage[row * 32 + (mi ^ lane)] = make_float2(d[2 * i], d[2 * i + 1]);
        }
        __syncthreads();  // a row's outputs come from two warps
        const uint64_t om = offs[lane];
        for (int q = half * 16; q < half * 16 + 16; ++q) {
          const int rr = (warp & 3) * 32 + q;
          if (tile * kTcRows + rr >= ngroups) break;
          const uint64_t i0 = dt | drow[rr];
          if ((i0 & op.cmask) == op.cval) __stcs(psi + (i0 | om), stage[rr * 32 + (lane ^ q)]);
        }
      } else {
        // consecutive groups adjacent in memory: stored straight from registers,
        // lane = group, each member's store coalesced across the warp
        const uint64_t i0 = dt | drow[row];
        if (tile * kTcRows + row < ngroups && (i0 & op.cmask) == op.cval) {
#pragma unroll
          for (int i = 0; i < 16; ++i) __stcs(psi + (i0 | offs[half * 16 + i]), make_float2(d[2 * i], d[2 * i + 1]));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // buffers of this iteration are free for the next
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the kernel, on every path
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcN) : "memory");
}

}  // namespace

int dense5_tc_smem() { return kSmemBytes; }

namespace {
std::atomic<bool> g_tc_launched{false};
std::atomic<bool> g_tc_enabled{true};
}  // namespace

void dense5_tc_enable(bool on) { g_tc_enabled = on; }
bool dense5_tc_enabled() { return g_tc_enabled; }

// Host side: read and clear the wait-timeout flag (0: no timeout since the last call).
int dense5_tc_take_error() {
  if (!g_tc_launched) return 0;
  int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return 0;
  if (v) cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
  return v;
}

cudaError_t dense5_tc(void *psi, int n, const OpDev &op, const void *mats, int adjoint, cudaStream_t st) {
  static bool attr = false;
  const int smem = dense5_tc_smem();
  if (!attr) {
    cudaFuncSetAttribute(k_dense5_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_dense5_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  // pair bit: the member bit of the target on global index bit 0 (segments of two adjacent amplitudes)
  int pb = 0;
  bool seg = false;
  for (int j = 0; j < 5; ++j)
    if (op.tg[j] == 0) {
      pb = 4 - j;
      seg = true;
    }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t ntiles = ((1ull << (n - 5)) + kTcRows - 1) / kTcRows;
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)sms);  // one persistent CTA per SM
  g_tc_launched = true;
  if (seg)
    k_dense5_tc<true><<<grid, kTcThreads, smem, st>>>(reinterpret_cast<float2 *>(psi), n, op,
                                                     reinterpret_cast<const float2 *>(mats) + op.mat, adjoint, pb);
  else
    k_dense5_tc<false><<<grid, kTcThreads, smem, st>>>(reinterpret_cast<float2 *>(psi), n, op,
                                                      reinterpret_cast<const float2 *>(mats) + op.mat, adjoint, pb);
  return cudaGetLastError();
}

}  // namespace sv

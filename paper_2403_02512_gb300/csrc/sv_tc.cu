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
constexpr int kTcThreads = 128;           // four warps: TMEM lanes 32w .. 32w + 31
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

template <bool SEG>
__global__ void __launch_bounds__(kTcThreads) k_dense5_tc(float2 *__restrict__ psi, int n, const OpDev op,
                                                          const float2 *__restrict__ M, int dagger, int pb) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *a_hi = smem, *a_lo = smem + kOpBytesA;
  unsigned char *b_hi = smem + 2 * kOpBytesA, *b_lo = b_hi + kOpBytesB;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(b_lo + kOpBytesB);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
  float2 *stage = reinterpret_cast<float2 *>(a_hi);  // outputs [group][32], after the MMAs read A
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

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
    st_shared_f32(smem_u32(b_hi) + kmajor_off(nn, k), hi);
    st_shared_f32(smem_u32(b_lo) + kmajor_off(nn, k), lo);
    split_tf32(vi, hi, lo);
    st_shared_f32(smem_u32(b_hi) + kmajor_off(nn, k + 1), hi);
    st_shared_f32(smem_u32(b_lo) + kmajor_off(nn, k + 1), lo);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  int sorted[5];
  for (int j = 0; j < 5; ++j) sorted[j] = op.tg[j];
  for (int i = 1; i < 5; ++i)
    for (int j = i; j > 0 && sorted[j - 1] > sorted[j]; --j) {
      const int t = sorted[j];
      sorted[j] = sorted[j - 1];
      sorted[j - 1] = t;
    }
  uint64_t roff = 0;  // this lane's member of a group (row index r = lane, wire order)
  for (int j = 0; j < 5; ++j)
    if ((lane >> (4 - j)) & 1) roff |= 1ull << op.tg[j];

  const uint64_t ngroups = 1ull << (n - 5);
  const uint64_t ntiles = (ngroups + kTcRows - 1) / kTcRows;
  uint32_t phase = 0;
  bool failed = false;
  for (uint64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    if constexpr (SEG) {
      // 512-byte chunks of the operand: 8 rows x 4 segments; lane -> (row l % 8, segment l / 8)
      for (int chunk = warp; chunk < (kTcRows / 8) * (kTcK / 16); chunk += kTcThreads / 32) {
        const int row = (chunk >> 2) * 8 + (lane & 7);
        const int seg = (chunk & 3) * 4 + (lane >> 3);  // pair index s
        const uint64_t g = tile * kTcRows + row;
        uint64_t i0 = 0;
        if (g < ngroups) {
          i0 = g;
          for (int j = 0; j < 5; ++j) {
            const int b = sorted[j];
            i0 = ((i0 >> b) << (b + 1)) | (i0 & ((1ull << b) - 1));
          }
        }
        // member of pair s with the pair bit clear
        const int m = ((seg >> pb) << (pb + 1)) | (seg & ((1 << pb) - 1));
        uint64_t off = 0;
        for (int j = 0; j < 5; ++j)
          if ((m >> (4 - j)) & 1) off |= 1ull << op.tg[j];
        cp_async16_zfill(smem_u32(a_hi) + kmajor_off(row, 4 * seg), psi + (i0 | off), g < ngroups ? 16 : 0);
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      // split in place: a_hi <- TF32(x), a_lo <- TF32(x - hi); consecutive 16-byte chunks per lane
      for (int c = threadIdx.x; c < kOpBytesA / 16; c += blockDim.x) {
        float4 x = reinterpret_cast<const float4 *>(a_hi)[c], lo;
        split_tf32(x.x, x.x, lo.x);
        split_tf32(x.y, x.y, lo.y);
        split_tf32(x.z, x.z, lo.z);
        split_tf32(x.w, x.w, lo.w);
        reinterpret_cast<float4 *>(a_hi)[c] = x;
        reinterpret_cast<float4 *>(a_lo)[c] = lo;
      }
    } else {
      // gather: warp w loads groups 32w .. 32w + 31 of the tile, lane = member
      const int kl = kpos(lane, pb);
      for (int q = 0; q < 32; ++q) {
        const int row = warp * 32 + q;
        const uint64_t g = tile * kTcRows + row;
        float2 a = make_float2(0.f, 0.f);
        if (g < ngroups) {
          uint64_t i0 = g;
          for (int j = 0; j < 5; ++j) {
            const int b = sorted[j];
            i0 = ((i0 >> b) << (b + 1)) | (i0 & ((1ull << b) - 1));
          }
          a = __ldcs(psi + (i0 | roff));
        }
        float hi, lo;
        split_tf32(a.x, hi, lo);
        st_shared_f32(smem_u32(a_hi) + kmajor_off(row, kl), hi);
        st_shared_f32(smem_u32(a_lo) + kmajor_off(row, kl), lo);
        split_tf32(a.y, hi, lo);
        st_shared_f32(smem_u32(a_hi) + kmajor_off(row, kl + 1), hi);
        st_shared_f32(smem_u32(a_lo) + kmajor_off(row, kl + 1), lo);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      const uint32_t as[3] = {ah, ah, al}, bs[3] = {bh, bl, bh};
      for (int pr = 0; pr < 3; ++pr)
        for (int ks = 0; ks < kTcK / 8; ++ks)  // K = 8 per MMA: two core matrices along K
          mma_tf32(tmem, mat_desc(as[pr] + ks * 2 * kLBO), mat_desc(bs[pr] + ks * 2 * kLBO), (pr | ks) != 0);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(mbar))
                   : "memory");
    }
    const unsigned long long t0 = global_ns_tc();
    while (!mbar_try_wait(smem_u32(mbar), phase)) {
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
    // each warp reads its 32 rows (TMEM lanes 32w ..) x 64 columns
    float d[kTcN];
#pragma unroll
    for (int c = 0; c < kTcN / 16; ++c) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
#pragma unroll
      for (int i = 0; i < 16; ++i) d[c * 16 + i] = v[i];
    }
    const int row = warp * 32 + lane;
    // staging index row * 32 + (member ^ (row % 32)): conflict-free for these per-row
    // writes and for the per-group reads below
#pragma unroll
    for (int i = 0; i < 32; ++i) stage[row * 32 + (i ^ lane)] = make_float2(d[2 * i], d[2 * i + 1]);
    __syncwarp();
    // store: warp w writes its 32 groups, lane = member (coalesced for low target bits)
    for (int q = 0; q < 32; ++q) {
      const int rr = warp * 32 + q;
      const uint64_t g = tile * kTcRows + rr;
      if (g >= ngroups) break;
      uint64_t i0 = g;
      for (int j = 0; j < 5; ++j) {
        const int b = sorted[j];
        i0 = ((i0 >> b) << (b + 1)) | (i0 & ((1ull << b) - 1));
      }
      if ((i0 & op.cmask) == op.cval) __stcs(psi + (i0 | roff), stage[rr * 32 + (lane ^ (rr & 31))]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the stage and A are rewritten by the next tile
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN) : "memory");
}

}  // namespace

int dense5_tc_smem() { return 2 * kOpBytesA + 2 * kOpBytesB + 64; }

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
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)sms * 2);
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

// Device kernels of the state-vector hot path, templated on the real type R
// (float = complex64 states, double = complex128 states).
//
// Layout: a state is 2^n amplitudes of c_t<R> (float2 / double2), interleaved
// (re, im).  Wire w is global index bit n-1-w (Alg. 1).
//
// Tile model (the GPU counterpart of Alg. 1 / Alg. 2's pair enumeration):
// a pass fixes T "local" index bits pos[0..T).  A tile is the 2^T amplitudes
// that share all other bits; tiles are disjoint and cover the state, the same
// disjointness that lets Alg. 1 update pairs concurrently (Sec. 2.1.1).  The
// lowest nlow local bits are the contiguous low index bits, so a tile is read
// as 2^(T-nlow) runs of 2^nlow consecutive amplitudes (>= 128 bytes: full
// 128-bit coalesced accesses).  Every op whose non-diagonal target wires are
// local bits is applied in shared memory; diagonal ops (RZ, PhaseShift,
// IsingZZ, CZ, ...) may act on any bits because they only need each
// amplitude's own global index.  Controls (Alg. 2) may be any bits: a group is
// updated only when its global index holds the control values.
#pragma once

#include <cstdint>
#include <type_traits>

#include "df64.cuh"
#include "sv_internal.h"
#include "sv.h"

namespace sv {

// Compute type R -> complex type in registers / shared memory (c_t) and the
// amplitude type in global memory (g_t).  R = df computes complex128 states in
// double-float arithmetic: global double2, converted on tile load / store.
template <typename R>
struct Types;
template <>
struct Types<float> {
  using C = float2;
  using G = float2;
};
template <>
struct Types<double> {
  using C = double2;
  using G = double2;
};
template <>
struct Types<df> {
  using C = dfc;
  using G = double2;
};
template <typename R>
using c_t = typename Types<R>::C;
template <typename R>
using g_t = typename Types<R>::G;

template <typename R>
__device__ __forceinline__ c_t<R> to_c(g_t<R> v) {
  if constexpr (std::is_same<R, df>::value) {
    dfc r;
    r.x = df(v.x);
    r.y = df(v.y);
    return r;
  } else {
    return v;
  }
}

template <typename R>
__device__ __forceinline__ g_t<R> to_g(c_t<R> v) {
  if constexpr (std::is_same<R, df>::value) {
    return make_double2((double)v.x, (double)v.y);
  } else {
    return v;
  }
}

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// acc + a * b
template <typename C>
__device__ __forceinline__ C cmac(C acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}

template <typename C>
__device__ __forceinline__ C cconj(C a) {
  a.y = -a.y;
  return a;
}

__device__ __forceinline__ int insert_zero(int x, int b) {
  return ((x >> b) << (b + 1)) | (x & ((1 << b) - 1));
}

// Error-free sum (Knuth TwoSum): s + e == a + b exactly.
template <typename R>
__device__ __forceinline__ void two_sum(R a, R b, R &s, R &e) {
  s = a + b;
  R bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Per-thread partial sum inside one tile: FP32 for complex64 states (a
// handful of terms), FP64 for complex128.  Tile partials are combined across
// warps and tiles in compensated form (see WarpAcc).
template <typename R>
struct Acc {
  R s = R(0);
  __device__ __forceinline__ void add(R v) { s += v; }
  __device__ __forceinline__ R value() const { return s; }
};

__device__ __forceinline__ float to_r(float v, float) { return v; }
__device__ __forceinline__ double to_r(float v, double) { return (double)v; }

// Per-warp accumulator slot in shared memory, summed over tiles: a
// double-float pair (hi, lo) updated with TwoSum for complex64 (no FP64
// instruction in the hot loop), a plain double for complex128.
template <typename R>
struct WarpAcc;
template <>
struct WarpAcc<float> {
  static __device__ __forceinline__ void add(double *slot, float v) {
    float2 *p = reinterpret_cast<float2 *>(slot);
    float2 a = *p;
    float s, e;
    two_sum(a.x, v, s, e);
    a.y += e;
    a.x = s;
    *p = a;
  }
  static __device__ __forceinline__ double read(const double *slot) {
    const float2 a = *reinterpret_cast<const float2 *>(slot);
    return (double)a.x + (double)a.y;
  }
};
template <>
struct WarpAcc<double> {
  static __device__ __forceinline__ void add(double *slot, double v) { *slot += v; }
  static __device__ __forceinline__ double read(const double *slot) { return *slot; }
};

__device__ __forceinline__ df warp_sum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = v + df_make(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
  return v;
}

template <>
struct WarpAcc<df> {
  static __device__ __forceinline__ void add(double *slot, df v) {
    df *p = reinterpret_cast<df *>(slot);
    *p = *p + v;
  }
  static __device__ __forceinline__ double read(const double *slot) { return (double)*reinterpret_cast<const df *>(slot); }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float shfl_x(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_x(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df shfl_x(df v, int o) {
  return df_make(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}

// Warp sums of P per-lane values of W components each (P a power of two up
// to 32), by reduce-scatter.  At exchange offset o = 16 >> K a lane holding
// c > 1 values keeps one half (the upper half when bit o of its lane is set),
// sends the other half to lane ^ o and adds what that lane sends for its kept
// half; once one value is left, plain exchanges over the remaining offsets
// finish the sum.  On return v[0] is the warp total of value `slot`, held by
// the 32 / P lanes that differ only in their low log2(32 / P) bits.  The cost
// is W (P - 1 + 5 - log2 P) additions, against 5 W P for P separate warp sums.
template <typename R, int P, int W, int K>
__device__ __forceinline__ void reduce_scatter_step(R (&v)[P][W], int lane, int &slot) {
  if constexpr (K < 5) {
    constexpr int o = 16 >> K;
    constexpr int c = P >> K;
    if constexpr (c > 1) {
      constexpr int h = c / 2;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i)
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const R send = up ? v[i][w] : v[i + h][w];
          const R keep = up ? v[i + h][w] : v[i][w];
          v[i][w] = keep + shfl_x(send, o);
        }
      if (up) slot += h;
    } else {
#pragma unroll
      for (int w = 0; w < W; ++w) v[0][w] = v[0][w] + shfl_x(v[0][w], o);
    }
    reduce_scatter_step<R, P, W, K + 1>(v, lane, slot);
  }
}

template <typename R, int P, int W>
__device__ __forceinline__ bool warp_reduce_scatter(R (&v)[P][W], int lane, int &slot) {
  static_assert(P >= 1 && P <= 32 && (P & (P - 1)) == 0, "P must be a power of two up to 32");
  slot = 0;
  reduce_scatter_step<R, P, W, 0>(v, lane, slot);
  return (lane & (32 / P - 1)) == 0;  // this lane writes slot's total
}

__host__ __device__ constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2); }

// ---------------------------------------------------------------------------
// Tile geometry
// ---------------------------------------------------------------------------
struct TileGeom {
  int T, nlow, A;
  uint32_t lowmask;
  const uint64_t *lut;  // shared: global offset of chunk c (local bits >= nlow)
  uint64_t base;        // global bits of the current tile

  __device__ __forceinline__ uint64_t gidx(int l) const {
    return base | lut[l >> nlow] | (uint64_t)(l & lowmask);
  }
};

__device__ __forceinline__ void build_lut(uint64_t *lut, const PassDev &p) {
  const int nch = 1 << (p.T - p.nlow);
  for (int c = threadIdx.x; c < nch; c += blockDim.x) {
    uint64_t o = 0;
    for (int i = p.nlow; i < p.T; ++i)
      if ((c >> (i - p.nlow)) & 1) o |= 1ull << p.pos[i];
    lut[c] = o;
  }
}

__device__ __forceinline__ uint64_t tile_base(const PassDev &p, uint64_t tile) {
  uint64_t b = 0;
  for (int i = 0; i < p.nhi; ++i)
    if ((tile >> i) & 1) b |= 1ull << p.hi[i];
  return b;
}

// 128-bit coalesced tile load / store (c64: two amplitudes per access).
template <typename R>
__device__ __forceinline__ void load_tile(const g_t<R> *__restrict__ g, c_t<R> *s, const TileGeom &tg) {
  if constexpr (std::is_same<R, float>::value) {
    const int nv = tg.A >> 1;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      const int l = v << 1;
      const float4 x = __ldg(reinterpret_cast<const float4 *>(g + tg.gidx(l)));
      reinterpret_cast<float4 *>(s)[v] = x;
    }
  } else {
    for (int l = threadIdx.x; l < tg.A; l += blockDim.x) s[l] = to_c<R>(__ldg(g + tg.gidx(l)));
  }
}


// Asynchronous tile load: every thread issues all of its 16-byte copies
// global -> shared (cp.async, L2 only) before waiting, so a whole tile is in
// flight at once.  Complete with tile_async_wait; double-float tiles then need
// tile_async_convert (the copies land as IEEE doubles in the same bytes).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <typename R>
__device__ __forceinline__ void load_tile_async(const g_t<R> *g, c_t<R> *s, const TileGeom &tg) {
  static_assert(sizeof(c_t<R>) == sizeof(g_t<R>), "tile bytes land unchanged");
  if constexpr (std::is_same<R, float>::value) {
    const int nv = tg.A >> 1;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) cp_async16(s + 2 * v, g + tg.gidx(v << 1));
  } else {
    for (int l = threadIdx.x; l < tg.A; l += blockDim.x) cp_async16(s + l, g + tg.gidx(l));
  }
}

__device__ __forceinline__ void tile_async_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
}

// In-place IEEE double -> double-float conversion of n amplitudes (after the wait).
template <typename R>
__device__ __forceinline__ void tile_async_convert(c_t<R> *s, int n) {
  if constexpr (std::is_same<R, df>::value) {
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      const double2 v = *reinterpret_cast<const double2 *>(s + l);
      s[l] = to_c<R>(v);
    }
    __syncthreads();
  }
}

template <typename R>
__device__ __forceinline__ void store_tile(g_t<R> *g, const c_t<R> *s, const TileGeom &tg) {
  if constexpr (std::is_same<R, float>::value) {
    const int nv = tg.A >> 1;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      const int l = v << 1;
      *reinterpret_cast<float4 *>(g + tg.gidx(l)) = reinterpret_cast<const float4 *>(s)[v];
    }
  } else {
    for (int l = threadIdx.x; l < tg.A; l += blockDim.x) g[tg.gidx(l)] = to_g<R>(s[l]);
  }
}

// ---------------------------------------------------------------------------
// Micro-op application inside a tile
// ---------------------------------------------------------------------------
// First member of group g of a k-target micro-op: g with a zero inserted at
// every target bit (Alg. 1 / Alg. 2 enumeration, on local bits).
__device__ __forceinline__ int group_base(const OpDev &op, int g) {
  int l = g;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (j < op.k) l = insert_zero(l, op.ts[j]);
  return l;
}

// The fields of a micro-op that the per-amplitude loops use, copied into
// registers once per op: reading them through the descriptor pointer inside a
// loop that stores to shared memory forces a reload on every iteration.
struct OpRegs {
  int k, ts0, ts1, ts2, ts3, oa, ob;
  uint64_t cmask, cval;
  __device__ __forceinline__ explicit OpRegs(const OpDev &op)
      : k(op.k), ts0(op.ts[0]), ts1(op.ts[1]), ts2(op.ts[2]), ts3(op.ts[3]), oa(op.oa), ob(op.ob),
        cmask(op.cmask), cval(op.cval) {}
  __device__ __forceinline__ int base(int g) const {
    int l = insert_zero(g, ts0);
    if (k > 1) l = insert_zero(l, ts1);
    if (k > 2) l = insert_zero(l, ts2);
    if (k > 3) l = insert_zero(l, ts3);
    return l;
  }
};

// Diagonal micro-op fields in registers (targets anywhere, entries up to 2^2
// held directly; wider diagonals read their entries from the matrix buffer).
template <typename R>
struct DiagRegs {
  int k, b0, b1, mat, code;
  uint64_t cmask, cval;
  c_t<R> d[4];
  bool small;
  __device__ __forceinline__ DiagRegs(const OpDev &op, const c_t<R> *__restrict__ mats)
      : k(op.k), b0(op.tg[0]), b1(op.k > 1 ? op.tg[1] : 0), mat(op.mat), code(op.code), cmask(op.cmask),
        cval(op.cval) {
    small = k <= 2 && code == dGen;
    if (small)
#pragma unroll
      for (int e = 0; e < 4; ++e) d[e] = e < (1 << k) ? mats[mat + e] : c_t<R>();
  }
  __device__ __forceinline__ int index(const OpDev &op, uint64_t g) const {
    if (k == 1) return (int)((g >> b0) & 1);
    if (k == 2) return (int)(((g >> b0) & 1) << 1 | ((g >> b1) & 1));
    int idx = 0;
    for (int j = 0; j < op.k; ++j) idx = (idx << 1) | (int)((g >> op.tg[j]) & 1);
    return idx;
  }
  __device__ __forceinline__ c_t<R> mul(const c_t<R> *__restrict__ mats, int idx, c_t<R> v) const {
    if (code == dNeg) {
      if (idx == (1 << k) - 1) {
        v.x = -v.x;
        v.y = -v.y;
      }
      return v;
    }
    if (small) {
      c_t<R> dv = d[0];
#pragma unroll
      for (int e = 1; e < 4; ++e)
        if (idx == e) dv = d[e];
      return cmul(v, dv);
    }
    return cmul(v, mats[mat + idx]);
  }
};

// Packed FP32 arithmetic for complex64 (the sm_100 family's two-lane FMA:
// one instruction for both components of a float2).  A complex product is
// formed from the vector's components: m v = vx (mr, mi) + vy (-mi, mr).
// (The other split, (mr, mr) v + (-mi, mi) (vy, vx), measured slower: its
// swapped copies cost extra moves.)
__device__ __forceinline__ float2 pk_swap(float2 v) { return make_float2(v.y, v.x); }
__device__ __forceinline__ float2 pk_re(float2 m) { return make_float2(m.x, m.x); }

// m0 a + m1 b for complex m0, m1, a, b (four packed instructions).
__device__ __forceinline__ float2 pk_cmv2(float2 m0, float2 a, float2 m1, float2 b) {
  return __ffma2_rn(make_float2(a.x, a.x), m0,
                    __ffma2_rn(make_float2(a.y, a.y), make_float2(-m0.y, m0.x),
                               __ffma2_rn(make_float2(b.x, b.x), m1, __fmul2_rn(make_float2(b.y, b.y), make_float2(-m1.y, m1.x)))));
}

// (va, vb) <- E (va, vb) for a 2x2 block E stored row-major in M.
// PK: complex64 general and real blocks in packed FP32 (where the kernel has
// registers to spare for the packed coefficients).
template <typename R, bool PK = false>
__device__ __forceinline__ void pair_apply(int code, const c_t<R> *M, c_t<R> &va, c_t<R> &vb) {
  using C = c_t<R>;
  C na, nb;
  if constexpr (PK && std::is_same<R, float>::value) {
    if (code == mReal) {
      na = __ffma2_rn(pk_re(M[0]), va, __fmul2_rn(pk_re(M[1]), vb));
      nb = __ffma2_rn(pk_re(M[2]), va, __fmul2_rn(pk_re(M[3]), vb));
      va = na;
      vb = nb;
      return;
    }
    if (code == mGen) {
      na = pk_cmv2(M[0], va, M[1], vb);
      nb = pk_cmv2(M[2], va, M[3], vb);
      va = na;
      vb = nb;
      return;
    }
  }
  switch (code) {
    case mSwap:
      na = vb;
      nb = va;
      break;
    case mY:
      na.x = vb.y;
      na.y = -vb.x;
      nb.x = -va.y;
      nb.y = va.x;
      break;
    case mReal: {
      const R m00 = M[0].x, m01 = M[1].x, m10 = M[2].x, m11 = M[3].x;
      na.x = fma(m00, va.x, m01 * vb.x);
      na.y = fma(m00, va.y, m01 * vb.y);
      nb.x = fma(m10, va.x, m11 * vb.x);
      nb.y = fma(m10, va.y, m11 * vb.y);
      break;
    }
    case mImOff: {
      const R d0 = M[0].x, o01 = M[1].y, o10 = M[2].y, d1 = M[3].x;
      na.x = fma(d0, va.x, -o01 * vb.y);
      na.y = fma(d0, va.y, o01 * vb.x);
      nb.x = fma(d1, vb.x, -o10 * va.y);
      nb.y = fma(d1, vb.y, o10 * va.x);
      break;
    }
    default: {
      na.x = R(0);
      na.y = R(0);
      nb = na;
      na = cmac(cmac(na, M[0], va), M[1], vb);
      nb = cmac(cmac(nb, M[2], va), M[3], vb);
      break;
    }
  }
  va = na;
  vb = nb;
}

// Im(conj(x) y) and Re(conj(x) y)
template <typename C>
__device__ __forceinline__ auto im_cx(C x, C y) -> decltype(x.x) { return x.x * y.y - x.y * y.x; }
template <typename C>
__device__ __forceinline__ auto re_cx(C x, C y) -> decltype(x.x) { return x.x * y.x + x.y * y.y; }

// acc += Im <l | G p> / gs over one pair for the generator codes gX / gY (the
// block scale gs is applied once per tile when the partial is flushed).
//   gX: Im(conj(la) pb) + Im(conj(lb) pa)
//   gY: (G p)_a = -i pb, (G p)_b = i pa  ->  Re(conj(lb) pa) - Re(conj(la) pb)
template <typename R, int GCODE>
__device__ __forceinline__ R pair_ip_acc(R acc, c_t<R> pa, c_t<R> pb, c_t<R> la, c_t<R> lb) {
  if (GCODE == gX) {
    acc = fma(la.x, pb.y, acc);
    acc = fma(-la.y, pb.x, acc);
    acc = fma(lb.x, pa.y, acc);
    acc = fma(-lb.y, pa.x, acc);
  } else {
    acc = fma(lb.x, pa.x, acc);
    acc = fma(lb.y, pa.y, acc);
    acc = fma(-la.x, pb.x, acc);
    acc = fma(-la.y, pb.y, acc);
  }
  return acc;
}


// Controls on bits outside the tile decide per tile whether an op acts at all.
__device__ __forceinline__ bool op_active(const OpDev &op, uint64_t base) {
  return (base & op.hcmask) == op.hcval;
}

template <typename R, int CODE, bool CTL>
__device__ void fwd_pair_t(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats) {
  using C = c_t<R>;
  C Mr[4];
  if (CODE == mGen || CODE == mReal || CODE == mImOff)
#pragma unroll
    for (int q = 0; q < 4; ++q) Mr[q] = mats[op.mat + q];
  const OpRegs o(op);
  const uint32_t lcm = op.lcmask, lcv = op.lcval;
  const int ng = tg.A >> o.k;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    const int l0 = o.base(g);
    if (CTL && (((uint32_t)l0 & lcm) != lcv)) continue;
    C va = s[l0 + o.oa], vb = s[l0 + o.ob];
    pair_apply<R, true>(CODE, Mr, va, vb);
    s[l0 + o.oa] = va;
    s[l0 + o.ob] = vb;
  }
}

template <typename R, int CODE>
__device__ __forceinline__ void fwd_pair_c(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *mats) {
  if (op.lcmask)
    fwd_pair_t<R, CODE, true>(s, tg, op, mats);
  else
    fwd_pair_t<R, CODE, false>(s, tg, op, mats);
}

template <typename R>
__device__ __forceinline__ void fwd_pair(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *mats) {
  switch (op.code) {
    case mSwap: fwd_pair_c<R, mSwap>(s, tg, op, mats); break;
    case mY: fwd_pair_c<R, mY>(s, tg, op, mats); break;
    case mReal: fwd_pair_c<R, mReal>(s, tg, op, mats); break;
    case mImOff: fwd_pair_c<R, mImOff>(s, tg, op, mats); break;
    default: fwd_pair_c<R, mGen>(s, tg, op, mats); break;
  }
}

// Diagonal index of local element l for a 1- or 2-target diagonal: targets in
// the tile come from l, the others are fixed for the tile.
struct DiagIdx {
  int fixed, sh0, sh1;
  __device__ __forceinline__ DiagIdx(const OpDev &op, uint64_t base, int kd) {
    fixed = 0;
    sh0 = op.tl[0] >= 0 ? op.tl[0] : 31;  // l < 2^13: (l >> 31) == 0
    if (op.tl[0] < 0) fixed |= (int)((base >> op.tg[0]) & 1) << (kd - 1);
    sh1 = 31;
    if (kd == 2) {
      sh1 = op.tl[1] >= 0 ? op.tl[1] : 31;
      if (op.tl[1] < 0) fixed |= (int)((base >> op.tg[1]) & 1);
    }
  }
  template <int KD>
  __device__ __forceinline__ int of(int l) const {
    if (KD == 1) return fixed | ((l >> sh0) & 1);
    return fixed | (((l >> sh0) & 1) << 1) | ((l >> sh1) & 1);
  }
};

template <typename C, int KD>
__device__ __forceinline__ C pick(const C (&d)[4], int idx) {
  if (KD == 1) return idx ? d[1] : d[0];
  C v = d[0];
  v = idx == 1 ? d[1] : v;
  v = idx == 2 ? d[2] : v;
  v = idx == 3 ? d[3] : v;
  return v;
}

template <typename C>
__device__ __forceinline__ C negate_if(C v, bool neg) {
  if (neg) {
    v.x = -v.x;
    v.y = -v.y;
  }
  return v;
}

template <typename R, int KD, bool NEG, bool CTL>
__device__ void fwd_diag_t(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats) {
  using C = c_t<R>;
  C d[4];
  if (!NEG)
#pragma unroll
    for (int e = 0; e < 4; ++e) d[e] = e < (1 << KD) ? mats[op.mat + e] : C();
  const DiagIdx di(op, tg.base, KD);
  const uint32_t lcm = op.lcmask, lcv = op.lcval;
  constexpr int full = (1 << KD) - 1;
  for (int l = threadIdx.x; l < tg.A; l += blockDim.x) {
    if (CTL && (((uint32_t)l & lcm) != lcv)) continue;
    const int idx = di.of<KD>(l);
    s[l] = NEG ? negate_if(s[l], idx == full) : cmul(s[l], pick<C, KD>(d, idx));
  }
}

template <typename R, int KD, bool NEG>
__device__ __forceinline__ void fwd_diag_c(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *mats) {
  if (op.lcmask)
    fwd_diag_t<R, KD, NEG, true>(s, tg, op, mats);
  else
    fwd_diag_t<R, KD, NEG, false>(s, tg, op, mats);
}

template <typename R>
__device__ void fwd_diag(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats) {
  if (op.k == 1) {
    if (op.code == dNeg)
      fwd_diag_c<R, 1, true>(s, tg, op, mats);
    else
      fwd_diag_c<R, 1, false>(s, tg, op, mats);
    return;
  }
  if (op.k == 2) {
    if (op.code == dNeg)
      fwd_diag_c<R, 2, true>(s, tg, op, mats);
    else
      fwd_diag_c<R, 2, false>(s, tg, op, mats);
    return;
  }
  const DiagRegs<R> dr(op, mats);  // wider diagonals: entries from the matrix buffer
  for (int l = threadIdx.x; l < tg.A; l += blockDim.x) {
    const uint64_t g = tg.gidx(l);
    if ((g & dr.cmask) != dr.cval) continue;
    s[l] = dr.mul(mats, dr.index(op, g), s[l]);
  }
}

// Dense 2^K x 2^K block of a user matrix (not trainable), inputs in registers.
template <int K>
struct GroupIdx {
  int offs[1 << K];
  __device__ __forceinline__ void init(const OpDev &op) {
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) {
      int o = 0;
#pragma unroll
      for (int j = 0; j < K; ++j)
        if ((r >> (K - 1 - j)) & 1) o |= 1 << op.tl[j];
      offs[r] = o;
    }
  }
};

template <typename R, int K>
__device__ __forceinline__ c_t<R> matrow(const c_t<R> (&v)[1 << K], const c_t<R> *__restrict__ M, int r) {
  using C = c_t<R>;
  constexpr int D = 1 << K;
  C acc;
  acc.x = R(0);
  acc.y = R(0);
#pragma unroll
  for (int c = 0; c < D; ++c) acc = cmac(acc, M[r * D + c], v[c]);
  return acc;
}

template <typename R, int K>
__device__ void dense_vec(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats) {
  using C = c_t<R>;
  constexpr int D = 1 << K;
  GroupIdx<K> gi;
  gi.init(op);
  const C *M = mats + op.mat;
  const int ng = tg.A >> K;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    const int l0 = group_base(op, g);
    if (op.cmask && ((tg.gidx(l0) & op.cmask) != op.cval)) continue;
    C v[D];
#pragma unroll
    for (int r = 0; r < D; ++r) v[r] = s[l0 + gi.offs[r]];
#pragma unroll
    for (int r = 0; r < D; ++r) s[l0 + gi.offs[r]] = matrow<R, K>(v, M, r);
  }
}

template <typename R, int MAXK>
__device__ __forceinline__ void dense_any(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *mats) {
  if (MAXK <= 2 || op.k == 2) {
    dense_vec<R, 2>(s, tg, op, mats);
  } else if (op.k == 3) {
    dense_vec<R, (MAXK >= 3 ? 3 : 2)>(s, tg, op, mats);
  } else {
    dense_vec<R, (MAXK >= 4 ? 4 : 2)>(s, tg, op, mats);
  }
}

// Parity count of a phase run at the local indices l = threadIdx.x + kBlock i:
// bit j of the word is member j's parity over l's local bits and the tile bits
// (the XOR of the transposed-mask words of l's set bits and the tile's flip
// word), so k = k0 + popcount(word): one popcount per amplitude for all members.
struct PhaseCount {
  const uint64_t *xw;  // transposed local masks, one word per local bit
  uint64_t pu;         // flip word XOR the words of the thread's bits (l's low 8 bits)
  int k0, T;
  __device__ __forceinline__ PhaseCount(const OpDev &op, const TileGeom &tg, const uint64_t *__restrict__ aux) {
    const uint64_t *m = aux + 2 * op.oa;
    const int r = op.ob, rl = op.zmask;
    xw = m + 2 * r;
    T = tg.T;
    uint64_t flip = 0;  // member j's parity over the tile bits (j < rl)
    k0 = 0;             // members without local bits: constant for the tile
    for (int j = 0; j < r; ++j) {
      const int f = __popcll(tg.base & __ldg(m + 2 * j + 1)) & 1;
      if (j < rl)
        flip |= (uint64_t)f << j;
      else
        k0 += f;
    }
    pu = flip;
    for (int b = 0; b < 8 && b < T; ++b)
      if ((threadIdx.x >> b) & 1) pu ^= __ldg(xw + b);
  }
  // k for l = threadIdx.x + kBlock * i
  __device__ __forceinline__ int at(int i) const {
    uint64_t w = pu;
    for (int b = 8; b < T; ++b)
      if ((i >> (b - 8)) & 1) w ^= __ldg(xw + b);
    return k0 + __popcll(w);
  }
};

// Phase run: k(l) = parities of the members over the tile's fixed bits (once
// per tile) plus their parities over the local bits of l; then one table entry.
template <typename R>
__device__ void fwd_phase(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats,
                          const uint64_t *__restrict__ aux) {
  const PhaseCount pc(op, tg, aux);
  for (int l = threadIdx.x, i = 0; l < tg.A; l += kBlock, ++i) s[l] = cmul(s[l], mats[op.mat + pc.at(i)]);
}

// Multi-wire micro-op: each thread takes groups of 2^W amplitudes (zeros
// inserted at the W sorted bits), applies the members' 2x2 blocks in order in
// registers, and stores the group back: one barrier for W gates.
template <typename R, int W>
__device__ void fwd_multi_t(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats) {
  using C = c_t<R>;
  constexpr int G = 1 << W;
  C M[W][4];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    const int c = op.mcode[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) M[j][q] = (c == mGen || c == mReal || c == mImOff) ? mats[op.mmat[j] + q] : C();
  }
  int off[G];
#pragma unroll
  for (int i = 0; i < G; ++i) {
    int o = 0;
#pragma unroll
    for (int j = 0; j < W; ++j)
      if ((i >> j) & 1) o += 1 << op.tl[j];
    off[i] = o;
  }
  const int ts0 = op.ts[0], ts1 = op.ts[1], ts2 = op.ts[2];
  const int ng = tg.A >> W;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    int l0 = insert_zero(insert_zero(g, ts0), ts1);
    if (W > 2) l0 = insert_zero(l0, ts2);
    C v[G];
#pragma unroll
    for (int i = 0; i < G; ++i) v[i] = s[l0 + off[i]];
#pragma unroll
    for (int j = 0; j < W; ++j)
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (!((i >> j) & 1)) pair_apply<R>(op.mcode[j], M[j], v[i], v[i | (1 << j)]);
#pragma unroll
    for (int i = 0; i < G; ++i) s[l0 + off[i]] = v[i];
  }
}

template <typename R, int MAXK>
__device__ __forceinline__ void apply_op(c_t<R> *s, const TileGeom &tg, const OpDev &op, const c_t<R> *mats,
                                         const uint64_t *aux) {
  if (op.kind == kMulti) {
    if (op.k == 2)
      fwd_multi_t<R, 2>(s, tg, op, mats);
    else
      fwd_multi_t<R, 3>(s, tg, op, mats);
    return;
  }
  if (op.kind != kDense && !op_active(op, tg.base)) return;
  if (op.kind == kPair)
    fwd_pair<R>(s, tg, op, mats);
  else if (op.kind == kDiag)
    fwd_diag<R>(s, tg, op, mats);
  else if (op.kind == kPhase)
    fwd_phase<R>(s, tg, op, mats, aux);
  else
    dense_any<R, MAXK>(s, tg, op, mats);
}

// ---------------------------------------------------------------------------
// Forward pass kernel: load tile, apply the pass's micro-ops, store.
// A barrier separates micro-ops whose thread-to-amplitude maps differ; runs of
// diagonal micro-ops and the blocks of one gate need none (each thread keeps
// the same amplitudes, or the blocks are disjoint).
// ---------------------------------------------------------------------------
template <typename R, int MAXK>
__global__ void __launch_bounds__(kBlock) k_tile_forward(g_t<R> *__restrict__ psi, int n, const PassDev pass,
                                                          const OpDev *__restrict__ ops,
                                                          const c_t<R> *__restrict__ mats,
                                                          const uint64_t *__restrict__ aux) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  C *s = reinterpret_cast<C *>(smem);
  uint64_t *lut = reinterpret_cast<uint64_t *>(smem + (sizeof(C) << pass.T));
  build_lut(lut, pass);
  TileGeom tg;
  tg.T = pass.T;
  tg.nlow = pass.nlow;
  tg.A = 1 << pass.T;
  tg.lowmask = (1u << pass.nlow) - 1u;
  tg.lut = lut;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pass.T);
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    tg.base = tile_base(pass, tile);
    load_tile_async<R>(psi, s, tg);
    tile_async_wait();
    tile_async_convert<R>(s, tg.A);
    for (int o = pass.op_begin; o < pass.op_end; ++o) {
      const OpDev &op = ops[o];
      if (op.sync_prev && o > pass.op_begin) __syncthreads();
      apply_op<R, MAXK>(s, tg, op, mats, aux);
    }
    __syncthreads();
    store_tile<R>(psi, s, tg);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Tangent pass (forward-mode Jacobian-vector product): psi and dpsi tiles go
// through the pass's micro-ops together; a trainable micro-op (generator G on
// its pair or diagonal) then adds coef[slot] * G psi_new to dpsi, with
// coef = i s scale tangent[p] for U = exp(i s theta G).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ c_t<R> tan_coef(const double2 *coefs, int slot) {
  const double2 c = coefs[slot];
  c_t<R> r;
  r.x = (R)c.x;
  r.y = (R)c.y;
  return r;
}

template <typename R>
__device__ void tan_pair(c_t<R> *sp, c_t<R> *sd, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats,
                         const double2 *__restrict__ coefs) {
  using C = c_t<R>;
  C Mr[4];
  if (op.code == mGen || op.code == mReal || op.code == mImOff)
#pragma unroll
    for (int q = 0; q < 4; ++q) Mr[q] = mats[op.mat + q];
  const bool tr = op.train >= 0 && op.slot >= 0 && (op.gcode == gX || op.gcode == gY);
  C c;
  c.x = R(0);
  c.y = R(0);
  if (tr) {
    c = tan_coef<R>(coefs, op.slot);
    const R gs = (R)op.gs;
    c.x = c.x * gs;
    c.y = c.y * gs;
  }
  const OpRegs o(op);
  const uint32_t lcm = op.lcmask, lcv = op.lcval;
  const int ng = tg.A >> o.k;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    const int l0 = o.base(g);
    if (((uint32_t)l0 & lcm) != lcv) continue;
    const int ia = l0 + o.oa, ib = l0 + o.ob;
    C va = sp[ia], vb = sp[ib];
    pair_apply<R>(op.code, Mr, va, vb);
    sp[ia] = va;
    sp[ib] = vb;
    C da = sd[ia], db = sd[ib];
    pair_apply<R>(op.code, Mr, da, db);
    if (tr) {
      C ga, gb;  // G psi on the pair: X -> (b, a), Y -> (-i b, i a)
      if (op.gcode == gX) {
        ga = vb;
        gb = va;
      } else {
        ga.x = vb.y;
        ga.y = -vb.x;
        gb.x = -va.y;
        gb.y = va.x;
      }
      const C ca = cmul(c, ga), cb = cmul(c, gb);
      da.x = da.x + ca.x;
      da.y = da.y + ca.y;
      db.x = db.x + cb.x;
      db.y = db.y + cb.y;
    }
    sd[ia] = da;
    sd[ib] = db;
  }
}

template <typename R>
__device__ void tan_diag(c_t<R> *sp, c_t<R> *sd, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats,
                         const double2 *__restrict__ coefs) {
  using C = c_t<R>;
  const DiagRegs<R> dr(op, mats);
  const bool tr = op.train >= 0 && op.slot >= 0 && op.gcode == gDiag;
  const C c = tr ? tan_coef<R>(coefs, op.slot) : C();
  const R ga = (R)op.ga, gb = (R)op.gb;
  for (int l = threadIdx.x; l < tg.A; l += blockDim.x) {
    const uint64_t g = tg.gidx(l);
    if ((g & dr.cmask) != dr.cval) continue;
    const int idx = dr.index(op, g);
    const C v = dr.mul(mats, idx, sp[l]);
    sp[l] = v;
    C d = dr.mul(mats, idx, sd[l]);
    if (tr) {
      const R gd = (__popc(idx & op.zmask) & 1) ? gb : ga;
      const C cv = cmul(c, v);
      d.x = d.x + gd * cv.x;
      d.y = d.y + gd * cv.y;
    }
    sd[l] = d;
  }
}

template <typename R, int MAXK>
__global__ void __launch_bounds__(kBlock) k_tile_tangent(g_t<R> *__restrict__ psi, g_t<R> *__restrict__ dpsi, int n,
                                                          const PassDev pass, const OpDev *__restrict__ ops,
                                                          const c_t<R> *__restrict__ mats,
                                                          const double2 *__restrict__ coefs) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int A = 1 << pass.T;
  C *sp = reinterpret_cast<C *>(smem);
  C *sd = sp + A;
  uint64_t *lut = reinterpret_cast<uint64_t *>(sd + A);
  build_lut(lut, pass);
  TileGeom tg;
  tg.T = pass.T;
  tg.nlow = pass.nlow;
  tg.A = A;
  tg.lowmask = (1u << pass.nlow) - 1u;
  tg.lut = lut;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pass.T);
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    tg.base = tile_base(pass, tile);
    load_tile_async<R>(psi, sp, tg);
    load_tile_async<R>(dpsi, sd, tg);
    tile_async_wait();
    tile_async_convert<R>(sp, 2 * A);
    for (int o = pass.op_begin; o < pass.op_end; ++o) {
      const OpDev &op = ops[o];
      if (op.sync_prev && o > pass.op_begin) __syncthreads();
      if (op.kind == kDense) {
        dense_any<R, MAXK>(sp, tg, op, mats);
        dense_any<R, MAXK>(sd, tg, op, mats);
      } else if (op_active(op, tg.base)) {
        if (op.kind == kPair)
          tan_pair<R>(sp, sd, tg, op, mats, coefs);
        else
          tan_diag<R>(sp, sd, tg, op, mats, coefs);
      }
    }
    __syncthreads();
    store_tile<R>(psi, sp, tg);
    store_tile<R>(dpsi, sd, tg);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Adjoint pass kernel.  For the pass's micro-ops in reverse order:
//   acc[op, j] += Im <lambda_j | G phi>   (before the op is un-applied),
//   phi <- E phi, lambda_j <- E lambda_j   (E = U^dagger, stored by the builder).
// One CTA holds a phi tile and b lambda tiles in shared memory, so phi is
// un-applied once per b lambdas.  blockIdx.x = lambda group (fastest, so the
// CTAs sharing a phi tile run together and re-read it from L2), blockIdx.y =
// tile group.  phi_out is written by lambda group 0 only: with several groups
// phi_in / phi_out are distinct buffers; with one group each phi tile is read
// and written by one CTA and phi_out may equal phi_in.
// Partial layout: partials[(blockIdx.y * m + j) * n_train + t].
// ---------------------------------------------------------------------------
// The warp's partial sums of NG x B accumulators (generator g, lambda jj)
// go to their per-warp slots accs[((train + g) * B + jj) * nwarps + warp],
// summed over the warp by one reduce-scatter.
template <typename R, int NG, int B>
__device__ __forceinline__ void flush_acc(const R (&acc)[NG][B], int bb, int train, double *accs, int nwarps,
                                          int warp, int lane, R scale) {
  constexpr int P = pow2_at_least(NG * B);
  R v[P][1];
#pragma unroll
  for (int i = 0; i < P; ++i) v[i][0] = i < NG * B ? acc[i / B][i % B] : R(0);
  int slot;
  const bool writer = warp_reduce_scatter<R, P, 1>(v, lane, slot);
  const int g = slot / B, jj = slot % B;
  if (writer && g < NG && jj < bb) WarpAcc<R>::add(&accs[((train + g) * B + jj) * nwarps + warp], scale * v[0][0]);
}

template <typename R, int B>
__device__ __forceinline__ void flush_acc(const R (&acc)[B], int bb, int train, double *accs, int nwarps, int warp,
                                          int lane, R scale) {
  flush_acc<R, 1, B>(reinterpret_cast<const R(&)[1][B]>(acc), bb, train, accs, nwarps, warp, lane, scale);
}

// Adjoint pair micro-op on phi and B lambda tiles (slots past the CTA's last
// lambda are zero and never stored).  acc[j] += Im <lambda_j | G phi> / gs.
template <typename R, int B, int CODE, int GCODE, bool CTL>
__device__ void adj_pair_t(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                           const c_t<R> *__restrict__ mats, R (&acc)[B]) {
  using C = c_t<R>;
  C Mr[4];
  if (CODE == mGen || CODE == mReal || CODE == mImOff)
#pragma unroll
    for (int q = 0; q < 4; ++q) Mr[q] = mats[op.mat + q];
  const OpRegs o(op);
  const uint32_t lcm = op.lcmask, lcv = op.lcval;
  const int ng = tg.A >> o.k;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    const int l0 = o.base(g);
    if (CTL && (((uint32_t)l0 & lcm) != lcv)) continue;
    const int ia = l0 + o.oa, ib = l0 + o.ob;
    C pa = sp[ia], pb = sp[ib];
    const C qa = pa, qb = pb;  // phi before the un-apply
    pair_apply<R, true>(CODE, Mr, pa, pb);
    sp[ia] = pa;
    sp[ib] = pb;
#pragma unroll
    for (int jj = 0; jj < B; ++jj) {
      C la = sl[jj * tg.A + ia], lb = sl[jj * tg.A + ib];
      if (GCODE != gNone) acc[jj] = pair_ip_acc<R, GCODE>(acc[jj], qa, qb, la, lb);
      pair_apply<R, true>(CODE, Mr, la, lb);
      sl[jj * tg.A + ia] = la;
      sl[jj * tg.A + ib] = lb;
    }
  }
}

template <typename R, int B, int CODE, int GCODE>
__device__ __forceinline__ void adj_pair_c(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                                           const c_t<R> *mats, R (&acc)[B]) {
  if (op.lcmask)
    adj_pair_t<R, B, CODE, GCODE, true>(sp, sl, tg, op, mats, acc);
  else
    adj_pair_t<R, B, CODE, GCODE, false>(sp, sl, tg, op, mats, acc);
}

template <typename R, int B, int CODE>
__device__ __forceinline__ void adj_pair_g(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                                           const c_t<R> *mats, R (&acc)[B]) {
  const int gcode = op.train >= 0 ? op.gcode : gNone;
  if (gcode == gX)
    adj_pair_c<R, B, CODE, gX>(sp, sl, tg, op, mats, acc);
  else if (gcode == gY)
    adj_pair_c<R, B, CODE, gY>(sp, sl, tg, op, mats, acc);
  else
    adj_pair_c<R, B, CODE, gNone>(sp, sl, tg, op, mats, acc);
}

template <typename R, int B>
__device__ __forceinline__ void adj_pair(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                                         const c_t<R> *mats, R (&acc)[B]) {
  switch (op.code) {
    case mSwap: adj_pair_g<R, B, mSwap>(sp, sl, tg, op, mats, acc); break;
    case mY: adj_pair_g<R, B, mY>(sp, sl, tg, op, mats, acc); break;
    case mReal: adj_pair_g<R, B, mReal>(sp, sl, tg, op, mats, acc); break;
    case mImOff: adj_pair_g<R, B, mImOff>(sp, sl, tg, op, mats, acc); break;
    default: adj_pair_g<R, B, mGen>(sp, sl, tg, op, mats, acc); break;
  }
}

// Fused run in the adjoint sweep: phi and B lambdas on pairs (a, b); for each
// of NG generators G' (Hermitian: G00, G11 real, G10 = conj(G01)) the
// contribution Im <lambda | G' phi> is taken before the run's U^dagger is
// applied.  Two ways to form it:
//  * products: w = G' phi once per pair, then every lambda adds
//    Im(conj(l_a) w_a + conj(l_b) w_b) (4 FMA per generator and lambda);
//  * moments (MOM): every lambda accumulates four real bilinear moments of
//    (lambda, phi) over its pairs,
//      D0 = Im(conj(l_a) p_a), D1 = Im(conj(l_b) p_b),
//      SY = Im(conj(l_a) p_b) + Im(conj(l_b) p_a),
//      SX = Re(conj(l_a) p_b) - Re(conj(l_b) p_a)   (12 FMA per lambda),
//    and after the warp reduction each generator's contribution is
//      G00 D0 + G11 D1 + Re(G01) SY + Im(G01) SX,
//    which equals the sum over pairs of Im(conj(l_a)(G' p)_a + conj(l_b)(G' p)_b).
//    No w = G' phi products are formed.
template <typename R, int B, int NG, bool CTL, bool MOM, bool SWZ = false>
__device__ void adj_fused_t(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                            const c_t<R> *__restrict__ mats, int bb, double *accs, int nwarps, int warp, int lane) {
  using C = c_t<R>;
  C Mr[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) Mr[q] = mats[op.mat + q];
  R g00[NG], g11[NG];
  C g01[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    g00[g] = mats[op.gmat + 4 * g].x;
    g01[g] = mats[op.gmat + 4 * g + 1];
    g11[g] = mats[op.gmat + 4 * g + 3].x;
  }
  constexpr int NA = MOM ? 4 : NG;  // accumulators per lambda
  constexpr bool PK = MOM && std::is_same<R, float>::value;
  R acc[NA][B];
  float2 pm[PK ? 4 : 1][PK ? B : 1];  // packed moment halves (complex64)
#pragma unroll
  for (int g = 0; g < NA; ++g)
#pragma unroll
    for (int jj = 0; jj < B; ++jj) acc[g][jj] = R(0);
  if constexpr (PK)
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int jj = 0; jj < B; ++jj) pm[g][jj] = make_float2(0.f, 0.f);
  const OpRegs o(op);
  const uint32_t lcm = op.lcmask, lcv = op.lcval;
  const int ng = tg.A >> 1;
  // SWZ (complex64 pair bit below 4): lanes 8..15 of each half-warp access their
  // pair's b member first.  A half-warp's a members then share no bank pair with
  // its b members (bit t of the index differs), so each access is conflict-free
  // instead of 2-way.  Such a thread holds (b, a): it applies P U P (P the
  // member swap, i.e. the block's entries mirrored) and its moments come out
  // as (D1, D0, SY, -SX), put back in order before the reduction.
  static_assert(!SWZ || MOM, "the swapped access order is written for the moment path");
  const bool sw = SWZ && ((threadIdx.x >> 3) & 1);
  const int oa = sw ? o.ob : o.oa, ob = sw ? o.oa : o.ob;
  if (SWZ && sw) {
    const C t0 = Mr[0], t1 = Mr[1];
    Mr[0] = Mr[3];
    Mr[1] = Mr[2];
    Mr[2] = t1;
    Mr[3] = t0;
  }
  for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
    const int l0 = o.base(gi);
    if (CTL && (((uint32_t)l0 & lcm) != lcv)) continue;
    const int ia = l0 + oa, ib = l0 + ob;  // first / second member in access order
    C pa = sp[ia], pb = sp[ib];
    if constexpr (MOM && std::is_same<R, float>::value) {
      // Packed moments: each float2 accumulator holds two partial products
      // whose sum (or difference) is one moment, resolved after the loop:
      //   pm[0] = (sum la.x qa.y, sum la.y qa.x)            D0 = x - y
      //   pm[1] = (sum lb.x qb.y, sum lb.y qb.x)            D1 = x - y
      //   pm[2] = la (qb.y, qb.x) + lb (qa.y, qa.x)         SY = x - y
      //   pm[3] = la (qb.x, qb.y) - lb (qa.x, qa.y)         SX = x + y
      const C qa = pa, qb = pb;
      const C qas = pk_swap(qa), qbs = pk_swap(qb), nqa = make_float2(-qa.x, -qa.y);
      pair_apply<R, true>(mGen, Mr, pa, pb);
      sp[ia] = pa;
      sp[ib] = pb;
#pragma unroll
      for (int jj = 0; jj < B; ++jj) {
        C la = sl[jj * tg.A + ia], lb = sl[jj * tg.A + ib];
        pm[0][jj] = __ffma2_rn(la, qas, pm[0][jj]);
        pm[1][jj] = __ffma2_rn(lb, qbs, pm[1][jj]);
        pm[2][jj] = __ffma2_rn(lb, qas, __ffma2_rn(la, qbs, pm[2][jj]));
        pm[3][jj] = __ffma2_rn(lb, nqa, __ffma2_rn(la, qb, pm[3][jj]));
        pair_apply<R, true>(mGen, Mr, la, lb);
        sl[jj * tg.A + ia] = la;
        sl[jj * tg.A + ib] = lb;
      }
    } else if constexpr (MOM) {
      const C qa = pa, qb = pb;  // phi before the un-apply
      pair_apply<R, true>(mGen, Mr, pa, pb);
      sp[ia] = pa;
      sp[ib] = pb;
#pragma unroll
      for (int jj = 0; jj < B; ++jj) {
        C la = sl[jj * tg.A + ia], lb = sl[jj * tg.A + ib];
        acc[0][jj] = fma(la.x, qa.y, fma(-la.y, qa.x, acc[0][jj]));
        acc[1][jj] = fma(lb.x, qb.y, fma(-lb.y, qb.x, acc[1][jj]));
        acc[2][jj] = fma(la.x, qb.y, fma(-la.y, qb.x, fma(lb.x, qa.y, fma(-lb.y, qa.x, acc[2][jj]))));
        acc[3][jj] = fma(la.x, qb.x, fma(la.y, qb.y, fma(-lb.x, qa.x, fma(-lb.y, qa.y, acc[3][jj]))));
        pair_apply<R, true>(mGen, Mr, la, lb);
        sl[jj * tg.A + ia] = la;
        sl[jj * tg.A + ib] = lb;
      }
    } else {
      C wa[NG], wb[NG];
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        // wa = g00 pa + g01 pb ; wb = conj(g01) pa + g11 pb
        wa[g].x = fma(g01[g].x, pb.x, fma(-g01[g].y, pb.y, g00[g] * pa.x));
        wa[g].y = fma(g01[g].x, pb.y, fma(g01[g].y, pb.x, g00[g] * pa.y));
        wb[g].x = fma(g01[g].x, pa.x, fma(g01[g].y, pa.y, g11[g] * pb.x));
        wb[g].y = fma(g01[g].x, pa.y, fma(-g01[g].y, pa.x, g11[g] * pb.y));
      }
      pair_apply<R, true>(mGen, Mr, pa, pb);
      sp[ia] = pa;
      sp[ib] = pb;
#pragma unroll
      for (int jj = 0; jj < B; ++jj) {
        C la = sl[jj * tg.A + ia], lb = sl[jj * tg.A + ib];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          R a = acc[g][jj];
          a = fma(la.x, wa[g].y, a);
          a = fma(-la.y, wa[g].x, a);
          a = fma(lb.x, wb[g].y, a);
          a = fma(-lb.y, wb[g].x, a);
          acc[g][jj] = a;
        }
        pair_apply<R, true>(mGen, Mr, la, lb);
        sl[jj * tg.A + ia] = la;
        sl[jj * tg.A + ib] = lb;
      }
    }
  }
  if constexpr (PK)
#pragma unroll
    for (int jj = 0; jj < B; ++jj) {
      acc[0][jj] = pm[0][jj].x - pm[0][jj].y;
      acc[1][jj] = pm[1][jj].x - pm[1][jj].y;
      acc[2][jj] = pm[2][jj].x - pm[2][jj].y;
      acc[3][jj] = pm[3][jj].x + pm[3][jj].y;
    }
  if constexpr (SWZ) {
    if (sw)
#pragma unroll
      for (int jj = 0; jj < B; ++jj) {
        const R d0 = acc[0][jj];
        acc[0][jj] = acc[1][jj];
        acc[1][jj] = d0;
        acc[3][jj] = -acc[3][jj];
      }
  }
  if constexpr (MOM) {
    // reduce-scatter over the lambdas with the four moments as one value
    R v[B][4];
#pragma unroll
    for (int jj = 0; jj < B; ++jj)
#pragma unroll
      for (int q = 0; q < 4; ++q) v[jj][q] = acc[q][jj];
    int jj;
    const bool writer = warp_reduce_scatter<R, B, 4>(v, lane, jj);
    if (writer && jj < bb)
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const R val = g00[g] * v[0][0] + g11[g] * v[0][1] + g01[g].x * v[0][2] + g01[g].y * v[0][3];
        WarpAcc<R>::add(&accs[((op.train + g) * B + jj) * nwarps + warp], val);
      }
  } else {
    flush_acc<R, NG, B>(acc, bb, op.train, accs, nwarps, warp, lane, R(1));
  }
}

template <typename R, int B, int NG>
__device__ __forceinline__ void adj_fused_c(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                                            const c_t<R> *mats, int bb, double *accs, int nwarps, int warp,
                                            int lane) {
  // moments when they cost fewer operations than the products (three
  // generators; two with at most two lambdas)
  constexpr bool MOM = NG == 3 || (NG == 2 && B <= 2);
  // complex64 pairs on the lowest four bits: access order that avoids bank conflicts
  if constexpr (MOM && std::is_same<R, float>::value) {
    if (op.ts[0] < 4) {
      if (op.lcmask)
        adj_fused_t<R, B, NG, true, MOM, true>(sp, sl, tg, op, mats, bb, accs, nwarps, warp, lane);
      else
        adj_fused_t<R, B, NG, false, MOM, true>(sp, sl, tg, op, mats, bb, accs, nwarps, warp, lane);
      return;
    }
  }
  if (op.lcmask)
    adj_fused_t<R, B, NG, true, MOM>(sp, sl, tg, op, mats, bb, accs, nwarps, warp, lane);
  else
    adj_fused_t<R, B, NG, false, MOM>(sp, sl, tg, op, mats, bb, accs, nwarps, warp, lane);
}

template <typename R, int B>
__device__ __forceinline__ void adj_fused(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                                          const c_t<R> *mats, int bb, double *accs, int nwarps, int warp, int lane) {
  if (op.ngen == 1)
    adj_fused_c<R, B, 1>(sp, sl, tg, op, mats, bb, accs, nwarps, warp, lane);
  else if (op.ngen == 2)
    adj_fused_c<R, B, 2>(sp, sl, tg, op, mats, bb, accs, nwarps, warp, lane);
  else
    adj_fused_c<R, B, 3>(sp, sl, tg, op, mats, bb, accs, nwarps, warp, lane);
}

// Phase run in the adjoint sweep: per amplitude k = parity count (as in the
// forward op); a trainable run adds (r - 2k) Im(conj(lambda_j) phi) for every
// lambda (the sum of its members' Z-parity generators) before phi and the
// lambdas are multiplied by the stored E[k] (adjoint entries).
template <typename R, int B>
__device__ void adj_phase(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op, const c_t<R> *__restrict__ mats,
                          const uint64_t *__restrict__ aux, int bb, double *accs, int nwarps, int warp, int lane) {
  using C = c_t<R>;
  const int r = op.ob;
  const bool tr = op.train >= 0;
  const PhaseCount pc(op, tg, aux);
  R acc[B];
#pragma unroll
  for (int jj = 0; jj < B; ++jj) acc[jj] = R(0);
  for (int l = threadIdx.x, i = 0; l < tg.A; l += kBlock, ++i) {
    const int k = pc.at(i);
    const C e = mats[op.mat + k];
    const C p = sp[l];
    const R g = R(r - 2 * k);
    const R gpy = g * p.y, gpx = g * p.x;
    sp[l] = cmul(p, e);
#pragma unroll
    for (int jj = 0; jj < B; ++jj) {
      const C q = sl[jj * tg.A + l];
      if (tr) acc[jj] = fma(q.x, gpy, fma(-q.y, gpx, acc[jj]));
      sl[jj * tg.A + l] = cmul(q, e);
    }
  }
  if (tr) flush_acc<R, B>(acc, bb, op.train, accs, nwarps, warp, lane, R(1));
}

// Adjoint diagonal micro-op: acc[j] += g(idx) Im(conj(lambda_j) phi) before
// multiplying phi and every lambda by the stored (adjoint) entry.
template <typename R, int B, int KD, bool NEG, bool CTL, bool TRAIN>
__device__ void adj_diag_t(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                           const c_t<R> *__restrict__ mats, R (&acc)[B]) {
  using C = c_t<R>;
  C d[4];
  if (!NEG)
#pragma unroll
    for (int e = 0; e < 4; ++e) d[e] = e < (1 << KD) ? mats[op.mat + e] : C();
  const DiagIdx di(op, tg.base, KD);
  const uint32_t lcm = op.lcmask, lcv = op.lcval;
  const R ga = (R)op.ga, gb = (R)op.gb;
  const int zmask = op.zmask;
  constexpr int full = (1 << KD) - 1;
  for (int l = threadIdx.x; l < tg.A; l += blockDim.x) {
    if (CTL && (((uint32_t)l & lcm) != lcv)) continue;
    const int idx = di.of<KD>(l);
    const C p = sp[l];
    R gpy = R(0), gpx = R(0);
    if (TRAIN) {
      const R gd = (__popc(idx & zmask) & 1) ? gb : ga;
      gpy = gd * p.y;
      gpx = gd * p.x;
    }
    C dv;
    if (!NEG) dv = pick<C, KD>(d, idx);
    const bool neg = idx == full;
    sp[l] = NEG ? negate_if(p, neg) : cmul(p, dv);
#pragma unroll
    for (int jj = 0; jj < B; ++jj) {
      const C q = sl[jj * tg.A + l];
      if (TRAIN) acc[jj] = fma(q.x, gpy, fma(-q.y, gpx, acc[jj]));
      sl[jj * tg.A + l] = NEG ? negate_if(q, neg) : cmul(q, dv);
    }
  }
}

template <typename R, int B, int KD, bool NEG>
__device__ __forceinline__ void adj_diag_c(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                                           const c_t<R> *mats, R (&acc)[B]) {
  const bool tr = op.train >= 0;
  if (op.lcmask) {
    if (tr)
      adj_diag_t<R, B, KD, NEG, true, true>(sp, sl, tg, op, mats, acc);
    else
      adj_diag_t<R, B, KD, NEG, true, false>(sp, sl, tg, op, mats, acc);
  } else {
    if (tr)
      adj_diag_t<R, B, KD, NEG, false, true>(sp, sl, tg, op, mats, acc);
    else
      adj_diag_t<R, B, KD, NEG, false, false>(sp, sl, tg, op, mats, acc);
  }
}

// Wider diagonals (user matrices on 3+ wires; never trainable).
template <typename R, int B>
__device__ void adj_diag_wide(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                              const c_t<R> *__restrict__ mats) {
  const DiagRegs<R> dr(op, mats);
  for (int l = threadIdx.x; l < tg.A; l += blockDim.x) {
    const uint64_t g = tg.gidx(l);
    if ((g & dr.cmask) != dr.cval) continue;
    const int idx = dr.index(op, g);
    sp[l] = dr.mul(mats, idx, sp[l]);
#pragma unroll
    for (int jj = 0; jj < B; ++jj) sl[jj * tg.A + l] = dr.mul(mats, idx, sl[jj * tg.A + l]);
  }
}

template <typename R, int B>
__device__ __forceinline__ void adj_diag(c_t<R> *sp, c_t<R> *sl, const TileGeom &tg, const OpDev &op,
                                         const c_t<R> *mats, R (&acc)[B]) {
  if (op.k == 1) {
    if (op.code == dNeg)
      adj_diag_c<R, B, 1, true>(sp, sl, tg, op, mats, acc);
    else
      adj_diag_c<R, B, 1, false>(sp, sl, tg, op, mats, acc);
  } else if (op.k == 2) {
    if (op.code == dNeg)
      adj_diag_c<R, B, 2, true>(sp, sl, tg, op, mats, acc);
    else
      adj_diag_c<R, B, 2, false>(sp, sl, tg, op, mats, acc);
  } else {
    adj_diag_wide<R, B>(sp, sl, tg, op, mats);
  }
}

template <typename R, int MAXK, int B>
__global__ void __launch_bounds__(kBlock, (std::is_same<R, double>::value && B >= 4) ? 1 : 2) k_tile_adjoint(const g_t<R> *phi_in, g_t<R> *phi_out,
                                                             g_t<R> *__restrict__ lam_base, int n, int m,
                                                             const PassDev pass, const OpDev *__restrict__ ops,
                                                             const c_t<R> *__restrict__ mats,
                                                             const uint64_t *__restrict__ aux,
                                                             double *__restrict__ partials) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int A = 1 << pass.T;
  const int j0 = blockIdx.x * B;
  const int bb = min(B, m - j0);
  C *sp = reinterpret_cast<C *>(smem);
  C *sl = sp + A;  // B lambda tiles; slots bb..B-1 stay zero
  uint64_t *lut = reinterpret_cast<uint64_t *>(sl + (size_t)B * A);
  const int nch = 1 << (pass.T - pass.nlow);
  double *accs = reinterpret_cast<double *>(lut + nch);  // [n_train][B][nwarps]
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  build_lut(lut, pass);
  for (int i = threadIdx.x; i < pass.n_train * B * nwarps; i += blockDim.x) accs[i] = 0.0;
  for (int i = threadIdx.x + bb * A; i < B * A; i += blockDim.x) {
    C z;
    z.x = R(0);
    z.y = R(0);
    sl[i] = z;
  }
  TileGeom tg;
  tg.T = pass.T;
  tg.nlow = pass.nlow;
  tg.A = A;
  tg.lowmask = (1u << pass.nlow) - 1u;
  tg.lut = lut;
  __syncthreads();

  const uint64_t ntiles = 1ull << (n - pass.T);
  for (uint64_t tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    tg.base = tile_base(pass, tile);
    load_tile_async<R>(phi_in, sp, tg);  // phi_in may equal phi_out (one lambda group, in place)
    for (int jj = 0; jj < bb; ++jj) load_tile_async<R>(lam_base + ((size_t)(j0 + jj) << n), sl + (size_t)jj * A, tg);
    tile_async_wait();
    tile_async_convert<R>(sp, A * (1 + bb));  // sp and the lambda tiles are contiguous
    for (int o = pass.op_end - 1; o >= pass.op_begin; --o) {
      const OpDev &op = ops[o];
      if (op.kind == kDense) {
        dense_any<R, MAXK>(sp, tg, op, mats);
        for (int jj = 0; jj < bb; ++jj) dense_any<R, MAXK>(sl + (size_t)jj * A, tg, op, mats);
      } else if (op.kind == kPhase) {
        adj_phase<R, B>(sp, sl, tg, op, mats, aux, bb, accs, nwarps, warp, lane);
      } else if (op.gcode == gHerm && op.train >= 0) {
        if (op_active(op, tg.base)) adj_fused<R, B>(sp, sl, tg, op, mats, bb, accs, nwarps, warp, lane);
      } else if (op_active(op, tg.base)) {
        R acc[B];
#pragma unroll
        for (int jj = 0; jj < B; ++jj) acc[jj] = R(0);
        if (op.kind == kPair)
          adj_pair<R, B>(sp, sl, tg, op, mats, acc);
        else
          adj_diag<R, B>(sp, sl, tg, op, mats, acc);
        if (op.train >= 0) flush_acc<R, B>(acc, bb, op.train, accs, nwarps, warp, lane, op.kind == kPair ? (R)op.gs : R(1));
      }
      if (op.sync_prev && o > pass.op_begin) __syncthreads();
    }
    __syncthreads();
    for (int jj = 0; jj < bb; ++jj) store_tile<R>(lam_base + ((size_t)(j0 + jj) << n), sl + (size_t)jj * A, tg);
    if (blockIdx.x == 0) store_tile<R>(phi_out, sp, tg);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < pass.n_train * bb; i += blockDim.x) {
    const int t = i / bb, jj = i % bb;
    double v = 0.0;
    for (int w = 0; w < nwarps; ++w) v += WarpAcc<R>::read(&accs[(t * B + jj) * nwarps + w]);
    partials[((size_t)blockIdx.y * m + j0 + jj) * pass.n_train + t] = v;
  }
}

// ---------------------------------------------------------------------------
// Expectation values: for every term t placed in this pass,
//   <P_t> partial = sum_l Re( i^{ny} (-1)^{popcount((g ^ x) & z)} conj(psi_g) psi_{g ^ x} )
// over the tile (P|i> = i^{ny} (-1)^{popcount(i & z)} |i ^ x>).  x lies inside
// the local bits, so both amplitudes are in the tile.  Term coefficients are
// applied later (combine_terms).  partials[b * n_terms + t].
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R pauli_re(c_t<R> a, c_t<R> b, int ny) {
  // Re(i^ny * conj(a) * b)
  const R re = a.x * b.x + a.y * b.y;
  const R im = a.x * b.y - a.y * b.x;
  switch (ny & 3) {
    case 0: return re;
    case 1: return -im;
    case 2: return -re;
    default: return im;
  }
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_expval(const g_t<R> *__restrict__ psi, int n, const PassDev pass,
                                                    const TermDev *__restrict__ terms, int n_terms,
                                                    double *__restrict__ partials) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int A = 1 << pass.T;
  C *s = reinterpret_cast<C *>(smem);
  uint64_t *lut = reinterpret_cast<uint64_t *>(s + A);
  const int nch = 1 << (pass.T - pass.nlow);
  double *accs = reinterpret_cast<double *>(lut + nch);  // [n_terms][nwarps]
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  build_lut(lut, pass);
  for (int i = threadIdx.x; i < n_terms * nwarps; i += blockDim.x) accs[i] = 0.0;
  TileGeom tg;
  tg.T = pass.T;
  tg.nlow = pass.nlow;
  tg.A = A;
  tg.lowmask = (1u << pass.nlow) - 1u;
  tg.lut = lut;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pass.T);
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    tg.base = tile_base(pass, tile);
    load_tile<R>(psi, s, tg);
    __syncthreads();
    for (int t = 0; t < n_terms; ++t) {
      const TermDev tm = terms[t];
      Acc<R> acc;
      // sign (-1)^popcount((g ^ x) & z) with g = tile base | local bits of l and
      // l = threadIdx.x + kBlock i: a per-thread part and the parity of i's bits
      const int s0 = (__popcll(tg.base & tm.zg) + __popcll(tm.xg & tm.zg) +
                      __popc((uint32_t)threadIdx.x & tm.zl & 0xFFu)) & 1;
      const uint32_t zh = tm.zl >> 8;
      for (int l = threadIdx.x, i = 0; l < A; l += kBlock, ++i) {
        const int par = s0 ^ (__popc((uint32_t)i & zh) & 1);
        R v = pauli_re<R>(s[l], s[l ^ tm.xl], tm.ny);
        acc.add(par ? -v : v);
      }
      const R part = warp_sum(acc.value());
      if (lane == 0) WarpAcc<R>::add(&accs[t * nwarps + warp], part);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n_terms; t += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nwarps; ++w) v += WarpAcc<R>::read(&accs[t * nwarps + w]);
    partials[(size_t)blockIdx.x * n_terms + t] = v;
  }
}

// ---------------------------------------------------------------------------
// Expectation pass for Pauli words with only Z letters (x = 0):
//   <P_t> = sum_g (-1)^{popcount(g & z_t)} |psi_g|^2.
// Thread u of the CTA owns the tile's local indices l = u + 256 i, i < NA =
// 2^NB (NB = T - 8).  Over those the sign factors: popcount(g & z) =
// popcount(tile base & z) + popcount(u & z_l) + popcount(i & (z_l >> 8)), with
// z_l the word's mask in local bits.  One Walsh-Hadamard transform of the
// thread's NA values p_i = |psi|^2, W[k] = sum_i (-1)^{popcount(i & k)} p_i,
// therefore gives every Z word's signed sum over the thread's amplitudes:
// (+-) W[z_l >> 8], the sign from the tile base and the thread bits.  Each
// thread accumulates its words over all its tiles in registers (words in
// chunks of 32, one read of the state per chunk), then one reduce-scatter per
// warp and fixed-order sums give partials[b * n_terms + t].
// ---------------------------------------------------------------------------
// v with its sign bit flipped when p is 1.
__device__ __forceinline__ float flip_sign(float v, uint32_t p) { return __int_as_float(__float_as_int(v) ^ (int)(p << 31)); }
__device__ __forceinline__ double flip_sign(double v, uint32_t p) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)p << 63));
}
__device__ __forceinline__ df flip_sign(df v, uint32_t p) { return df_make(flip_sign(v.h, p), flip_sign(v.l, p)); }

template <typename R>
struct ZSum;  // per-thread running sum of a word over tiles
template <>
struct ZSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct ZSum<float> {  // compensated (TwoSum): no FP64 instruction per tile
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float t, e;
    two_sum(s, v, t, e);
    s = t;
    c += e;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <>
struct ZSum<df> {
  df s = df(0.f);
  __device__ __forceinline__ void add(df v) { s = s + v; }
  __device__ __forceinline__ double value() const { return (double)s; }
};

constexpr int kZChunk = 32;

template <typename R, int NB>
__global__ void __launch_bounds__(kBlock) k_expval_z(const g_t<R> *__restrict__ psi, int n, const PassDev pass,
                                                      const TermDev *__restrict__ terms, int n_terms,
                                                      double *__restrict__ partials) {
  constexpr int NA = 1 << NB;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nch = 1 << (pass.T - pass.nlow);
  uint64_t *lut = reinterpret_cast<uint64_t *>(smem);
  R *sw = reinterpret_cast<R *>(lut + nch);                        // W[k] of thread u at sw[k * kBlock + u]
  uint64_t *zg = reinterpret_cast<uint64_t *>(sw + NA * kBlock);    // chunk words' global z masks
  int *zk = reinterpret_cast<int *>(zg + kZChunk);                  // ... their upper local z bits
  double *accs = reinterpret_cast<double *>(zk + kZChunk);          // [n_terms][nwarps]
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int u = threadIdx.x;
  build_lut(lut, pass);
  for (int i = threadIdx.x; i < n_terms * nwarps; i += blockDim.x) accs[i] = 0.0;
  TileGeom tg;
  tg.T = pass.T;
  tg.nlow = pass.nlow;
  tg.A = 1 << pass.T;
  tg.lowmask = (1u << pass.nlow) - 1u;
  tg.lut = lut;
  const uint64_t ntiles = 1ull << (n - pass.T);
  for (int t0 = 0; t0 < n_terms; t0 += kZChunk) {
    const int nt = min(kZChunk, n_terms - t0);
    __syncthreads();  // the previous chunk's words are no longer read
    uint32_t par_thread = 0;  // bit t: parity of the thread bits under word t
    for (int t = 0; t < nt; ++t) {
      const uint64_t z = terms[t0 + t].zg;
      uint32_t zl = 0;  // z in local bits
      for (int b = 0; b < pass.T; ++b)
        if (z >> pass.pos[b] & 1) zl |= 1u << b;
      par_thread |= (uint32_t)(__popc(zl & (uint32_t)u & 0xFFu) & 1) << t;
      if (threadIdx.x == 0) {
        zg[t] = z;
        zk[t] = (int)(zl >> 8);
      }
    }
    __syncthreads();  // zg / zk written (each thread reads only its own column of sw)
    ZSum<R> acc[kZChunk];
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      tg.base = tile_base(pass, tile);
      R w[NA];
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        const c_t<R> a = to_c<R>(__ldcs(psi + tg.gidx(u + i * kBlock)));
        w[i] = a.x * a.x + a.y * a.y;
      }
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int i = 0; i < NA; ++i)
          if (!(i >> b & 1)) {
            const R x = w[i], y = w[i | (1 << b)];
            w[i] = x + y;
            w[i | (1 << b)] = x - y;
          }
#pragma unroll
      for (int i = 0; i < NA; ++i) sw[i * kBlock + u] = w[i];
#pragma unroll
      for (int t = 0; t < kZChunk; ++t) {
        if (t < nt) {
          const uint32_t neg = ((par_thread >> t) & 1u) ^ (uint32_t)(__popcll(tg.base & zg[t]) & 1);
          acc[t].add(flip_sign(sw[zk[t] * kBlock + u], neg));
        }
      }
    }
    // per-warp sums of the chunk's words
    double v[kZChunk][1];
#pragma unroll
    for (int t = 0; t < kZChunk; ++t) v[t][0] = t < nt ? acc[t].value() : 0.0;
    int slot;
    const bool writer = warp_reduce_scatter<double, kZChunk, 1>(v, lane, slot);
    if (writer && slot < nt) accs[(t0 + slot) * nwarps + warp] += v[0][0];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n_terms; t += blockDim.x) {
    double s = 0.0;
    for (int wi = 0; wi < nwarps; ++wi) s += accs[t * nwarps + wi];
    partials[(size_t)blockIdx.x * n_terms + t] = s;
  }
}

// ---------------------------------------------------------------------------
// Lambda initialisation: lam_o += sum_{t in o} c_t P_t phi over the terms of
// this pass (output-stationary: each lambda amplitude written once per pass).
//   (P phi)_g = i^{ny} (-1)^{popcount((g ^ x) & z)} phi_{g ^ x}
// Words are the outer loop over NA register sums per thread (the word's masks
// and signed coefficients formed once per thread), as in k_expval_obs below.
// blockIdx.y = observable within the chunk; first != 0 overwrites lam.
// ---------------------------------------------------------------------------
// h[k] += i^{ny} c (-1)^{popcount((g[k] ^ x) & z)} s[l_k ^ x_l] for the words [t0, t1).
template <typename R, int NA>
__device__ __forceinline__ void pauli_rows(const c_t<R> *s, int A, const uint64_t (&g)[NA],
                                           const TermDev *__restrict__ terms, int t0, int t1, R (&hx)[NA],
                                           R (&hy)[NA]) {
  using C = c_t<R>;
  for (int t = t0; t < t1; ++t) {
    const TermDev tm = terms[t];
    // i^ny c b:  x += cx * (swap ? b.y : b.x),  y += cy * (swap ? b.x : b.y)
    const int ny = tm.ny & 3;
    const bool swap = (ny & 1) != 0;
    const R c = R(tm.coeff);
    const R cx = (ny == 1 || ny == 2) ? -c : c;
    const R cy = ny >= 2 ? -c : c;
    const uint32_t tpar = (uint32_t)__popcll(tm.xg & tm.zg) & 1u;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const int l = threadIdx.x + k * kBlock;
      if (l < A) {
        const C b = s[l ^ tm.xl];
        const uint32_t par = ((uint32_t)__popcll(g[k] & tm.zg) & 1u) ^ tpar;
        const R bx = flip_sign(b.x, par), by = flip_sign(b.y, par);
        hx[k] = fma(cx, swap ? by : bx, hx[k]);
        hy[k] = fma(cy, swap ? bx : by, hy[k]);
      }
    }
  }
}

template <typename R, int NA>
__global__ void __launch_bounds__(kBlock) k_lambda(const g_t<R> *__restrict__ phi, g_t<R> *__restrict__ lam_base,
                                                    int n, const PassDev pass, const TermDev *__restrict__ terms,
                                                    const int32_t *__restrict__ obs_term_begin, int first) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int A = 1 << pass.T;
  C *s = reinterpret_cast<C *>(smem);
  uint64_t *lut = reinterpret_cast<uint64_t *>(s + A);
  const int o = blockIdx.y;
  const int t0 = obs_term_begin[o], t1 = obs_term_begin[o + 1];
  g_t<R> *lam = lam_base + ((size_t)o << n);
  build_lut(lut, pass);
  TileGeom tg;
  tg.T = pass.T;
  tg.nlow = pass.nlow;
  tg.A = A;
  tg.lowmask = (1u << pass.nlow) - 1u;
  tg.lut = lut;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pass.T);
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    tg.base = tile_base(pass, tile);
    load_tile<R>(phi, s, tg);
    __syncthreads();
    uint64_t g[NA];
    R hx[NA], hy[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const int l = threadIdx.x + k * kBlock;
      g[k] = l < A ? tg.gidx(l) : 0;
      hx[k] = R(0);
      hy[k] = R(0);
    }
    pauli_rows<R, NA>(s, A, g, terms, t0, t1, hx, hy);
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const int l = threadIdx.x + k * kBlock;
      if (l < A) {
        C acc;
        if (first) {
          acc.x = hx[k];
          acc.y = hy[k];
        } else {
          acc = to_c<R>(lam[g[k]]);
          acc.x = acc.x + hx[k];
          acc.y = acc.y + hy[k];
        }
        lam[g[k]] = to_g<R>(acc);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Expectation values by observable (Hamiltonians of many words): for
// each amplitude g of the tile, (H_o psi)_g over the words of observable o
// placed in this pass is accumulated in registers, then Re(conj(psi_g)
// (H_o psi)_g) is summed: one reduction per observable and tile instead of one
// per word.  Words are the outer loop, so a word's masks and signed
// coefficients are formed once per thread for its NA amplitudes.  The sign
// (-1)^{popcount((g ^ x) & z)} = (-1)^{popcount(g & z)} (-1)^{popcount(x & z)}
// is applied by flipping the sign bits of the partner amplitude (pauli_rows).
// partials[block * n_obs + o].
// ---------------------------------------------------------------------------
template <typename R, int NA>
__global__ void __launch_bounds__(kBlock) k_expval_obs(const g_t<R> *__restrict__ psi, int n, const PassDev pass,
                                                        const TermDev *__restrict__ terms,
                                                        const int32_t *__restrict__ obs_term_begin, int n_obs,
                                                        double *__restrict__ partials) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int A = 1 << pass.T;
  C *s = reinterpret_cast<C *>(smem);
  uint64_t *lut = reinterpret_cast<uint64_t *>(s + A);
  const int nch = 1 << (pass.T - pass.nlow);
  double *accs = reinterpret_cast<double *>(lut + nch);  // [n_obs][nwarps]
  const int nwarps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  build_lut(lut, pass);
  for (int i = threadIdx.x; i < n_obs * nwarps; i += blockDim.x) accs[i] = 0.0;
  TileGeom tg;
  tg.T = pass.T;
  tg.nlow = pass.nlow;
  tg.A = A;
  tg.lowmask = (1u << pass.nlow) - 1u;
  tg.lut = lut;
  __syncthreads();
  const uint64_t ntiles = 1ull << (n - pass.T);
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    tg.base = tile_base(pass, tile);
    load_tile<R>(psi, s, tg);
    __syncthreads();
    uint64_t g[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      const int l = threadIdx.x + k * kBlock;
      g[k] = l < A ? tg.gidx(l) : 0;
    }
    for (int o = 0; o < n_obs; ++o) {
      const int t0 = obs_term_begin[o], t1 = obs_term_begin[o + 1];
      if (t0 == t1) continue;
      R hx[NA], hy[NA];
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        hx[k] = R(0);
        hy[k] = R(0);
      }
      pauli_rows<R, NA>(s, A, g, terms, t0, t1, hx, hy);
      Acc<R> acc;
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        const int l = threadIdx.x + k * kBlock;
        if (l < A) {
          const C a = s[l];
          acc.add(a.x * hx[k] + a.y * hy[k]);
        }
      }
      const R part = warp_sum(acc.value());
      if (lane == 0) WarpAcc<R>::add(&accs[o * nwarps + warp], part);
    }
    __syncthreads();
  }
  for (int o = threadIdx.x; o < n_obs; o += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nwarps; ++w) v += WarpAcc<R>::read(&accs[o * nwarps + w]);
    partials[(size_t)blockIdx.x * n_obs + o] = v;
  }
}

// ---------------------------------------------------------------------------
// Dense k-qubit block applied straight from global memory (k = 5, 6), one
// output amplitude per thread: CTA stages 256 / 2^k groups in shared memory.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBlock) k_dense_k(g_t<R> *__restrict__ psi, int n, const OpDev op,
                                                     const c_t<R> *__restrict__ M, int dagger) {
  using C = c_t<R>;
  __shared__ C sv[kBlock];
  const int K = op.k, D = 1 << K;
  const int gpb = kBlock / D;  // groups per CTA
  int sorted[kMaxTargets];
  for (int j = 0; j < K; ++j) sorted[j] = op.tg[j];
  for (int i = 1; i < K; ++i)
    for (int j = i; j > 0 && sorted[j - 1] > sorted[j]; --j) {
      int t = sorted[j];
      sorted[j] = sorted[j - 1];
      sorted[j - 1] = t;
    }
  const uint64_t ngroups = 1ull << (n - K);
  const int r = threadIdx.x % D, gl = threadIdx.x / D;
  uint64_t roff = 0;
  for (int j = 0; j < K; ++j)
    if ((r >> (K - 1 - j)) & 1) roff |= 1ull << op.tg[j];
  for (uint64_t g0 = (uint64_t)blockIdx.x * gpb; g0 < ngroups; g0 += (uint64_t)gridDim.x * gpb) {
    const uint64_t g = g0 + gl;
    uint64_t i0 = g;
    for (int j = 0; j < K; ++j) {
      const int b = sorted[j];
      i0 = ((i0 >> b) << (b + 1)) | (i0 & ((1ull << b) - 1));
    }
    const bool active = (g < ngroups) && ((i0 & op.cmask) == op.cval);
    if (active) sv[threadIdx.x] = to_c<R>(psi[i0 | roff]);
    __syncthreads();
    if (active) {
      C acc;
      acc.x = R(0);
      acc.y = R(0);
      for (int c = 0; c < D; ++c) {
        C m = dagger ? cconj(M[c * D + r]) : M[r * D + c];
        acc = cmac(acc, m, sv[gl * D + c]);
      }
      psi[i0 | roff] = to_g<R>(acc);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Gate matrices from parameters (one thread per slot, FP64 trigonometry).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 dc(double re, double im) { return make_double2(re, im); }

// Writes the 2^k x 2^k matrix of a base gate (not SV_MATRIX) into m (row-major).
__device__ inline void gate_matrix(int kind, const double *a, double2 *m) {
  double c = 0.0, s = 0.0;
  if (kind == SV_RX || kind == SV_RY || kind == SV_ISING_XX || kind == SV_ISING_YY ||
      kind == SV_ISING_XY || kind == SV_SINGLE_EXCITATION || kind == SV_DOUBLE_EXCITATION)
    sincos(0.5 * a[0], &s, &c);
  const double r2 = 0.70710678118654752440;
  switch (kind) {
    case SV_IDENTITY: m[0] = dc(1, 0); m[1] = dc(0, 0); m[2] = dc(0, 0); m[3] = dc(1, 0); break;
    case SV_PAULI_X: m[0] = dc(0, 0); m[1] = dc(1, 0); m[2] = dc(1, 0); m[3] = dc(0, 0); break;
    case SV_PAULI_Y: m[0] = dc(0, 0); m[1] = dc(0, -1); m[2] = dc(0, 1); m[3] = dc(0, 0); break;
    case SV_PAULI_Z: m[0] = dc(1, 0); m[1] = dc(0, 0); m[2] = dc(0, 0); m[3] = dc(-1, 0); break;
    case SV_HADAMARD: m[0] = dc(r2, 0); m[1] = dc(r2, 0); m[2] = dc(r2, 0); m[3] = dc(-r2, 0); break;
    case SV_S: m[0] = dc(1, 0); m[1] = dc(0, 0); m[2] = dc(0, 0); m[3] = dc(0, 1); break;
    case SV_T: m[0] = dc(1, 0); m[1] = dc(0, 0); m[2] = dc(0, 0); m[3] = dc(r2, r2); break;
    case SV_PHASE_SHIFT: {
      double ps, pc;
      sincos(a[0], &ps, &pc);
      m[0] = dc(1, 0); m[1] = dc(0, 0); m[2] = dc(0, 0); m[3] = dc(pc, ps);
      break;
    }
    case SV_RX: m[0] = dc(c, 0); m[1] = dc(0, -s); m[2] = dc(0, -s); m[3] = dc(c, 0); break;
    case SV_RY: m[0] = dc(c, 0); m[1] = dc(-s, 0); m[2] = dc(s, 0); m[3] = dc(c, 0); break;
    case SV_RZ: {
      double zs, zc;
      sincos(0.5 * a[0], &zs, &zc);
      m[0] = dc(zc, -zs); m[1] = dc(0, 0); m[2] = dc(0, 0); m[3] = dc(zc, zs);
      break;
    }
    case SV_ROT: {
      // RZ(w) RY(t) RZ(p): [[e^{-i(p+w)/2} c, -e^{i(p-w)/2} s], [e^{-i(p-w)/2} s, e^{i(p+w)/2} c]]
      double tc, ts, ac, as, bc, bs;
      sincos(0.5 * a[1], &ts, &tc);
      sincos(0.5 * (a[0] + a[2]), &as, &ac);
      sincos(0.5 * (a[0] - a[2]), &bs, &bc);
      m[0] = dc(ac * tc, -as * tc);
      m[1] = dc(-bc * ts, -bs * ts);
      m[2] = dc(bc * ts, -bs * ts);
      m[3] = dc(ac * tc, as * tc);
      break;
    }
    case SV_SWAP:
      for (int i = 0; i < 16; ++i) m[i] = dc(0, 0);
      m[0] = m[6] = m[9] = m[15] = dc(1, 0);
      break;
    case SV_ISING_XX:
      for (int i = 0; i < 16; ++i) m[i] = dc(0, 0);
      for (int i = 0; i < 4; ++i) {
        m[i * 4 + i] = dc(c, 0);
        m[i * 4 + (3 - i)] = dc(0, -s);
      }
      break;
    case SV_ISING_YY:
      for (int i = 0; i < 16; ++i) m[i] = dc(0, 0);
      for (int i = 0; i < 4; ++i) m[i * 4 + i] = dc(c, 0);
      m[3] = m[12] = dc(0, s);
      m[6] = m[9] = dc(0, -s);
      break;
    case SV_ISING_ZZ: {
      double zs, zc;
      sincos(0.5 * a[0], &zs, &zc);
      for (int i = 0; i < 16; ++i) m[i] = dc(0, 0);
      m[0] = m[15] = dc(zc, -zs);
      m[5] = m[10] = dc(zc, zs);
      break;
    }
    case SV_ISING_XY:
      for (int i = 0; i < 16; ++i) m[i] = dc(0, 0);
      m[0] = m[15] = dc(1, 0);
      m[5] = m[10] = dc(c, 0);
      m[6] = m[9] = dc(0, s);
      break;
    case SV_SINGLE_EXCITATION:
      for (int i = 0; i < 16; ++i) m[i] = dc(0, 0);
      m[0] = m[15] = dc(1, 0);
      m[5] = m[10] = dc(c, 0);
      m[6] = dc(-s, 0);
      m[9] = dc(s, 0);
      break;
    case SV_DOUBLE_EXCITATION:
      for (int i = 0; i < 256; ++i) m[i] = dc(0, 0);
      for (int i = 0; i < 16; ++i) m[i * 16 + i] = dc(1, 0);
      m[3 * 16 + 3] = m[12 * 16 + 12] = dc(c, 0);
      m[3 * 16 + 12] = dc(-s, 0);
      m[12 * 16 + 3] = dc(s, 0);
      break;
    default: break;
  }
}

template <typename R>
__device__ __forceinline__ void put_entry(const MatSlot &sl, c_t<R> *o, int r, int c, double re, double im) {
  c_t<R> v;
  v.x = (R)re;
  v.y = (R)im;
  const int D = 1 << sl.k;
  if (sl.mode == 0) {
    o[r * D + c] = v;
  } else if (sl.mode == 1) {
    if (r == c) o[r] = v;
  } else {
    const int rr = r == sl.a ? 0 : (r == sl.b ? 1 : -1);
    const int cc = c == sl.a ? 0 : (c == sl.b ? 1 : -1);
    if (rr >= 0 && cc >= 0) o[rr * 2 + cc] = v;
  }
}

// One thread per slot: E = U (or U^dagger) from FP64 trigonometry, written
// whole, as its diagonal, or as one 2x2 block.
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }

// 2x2 matrix of a single-wire member of a fused run (its own adjoint applied).
__device__ inline void member_matrix(const MatSlot &m, const double *__restrict__ params, const double *__restrict__ user,
                              double2 (&u)[4]) {
  if (m.kind == SV_MATRIX) {
    for (int e = 0; e < 4; ++e) u[e] = make_double2(user[2 * (m.src + e)], user[2 * (m.src + e) + 1]);
  } else {
    double a[3];
    for (int q = 0; q < 3; ++q) a[q] = m.pidx[q] >= 0 ? m.scale * params[m.pidx[q]] : m.cangle[q];
    double2 g[256];
    gate_matrix(m.kind, a, g);
    for (int e = 0; e < 4; ++e) u[e] = g[e];
  }
  if (m.dagger) {
    const double2 t = u[1];
    u[0] = zconj(u[0]);
    u[1] = zconj(u[2]);
    u[2] = zconj(t);
    u[3] = zconj(u[3]);
  }
}

// Fused run: V = U_r ... U_1 built from the last member backwards; a trainable
// member i gets G_i' = W G_i W^dagger with W = U_r ... U_{i+1}, the generator
// seen from the run's end (Im<lambda|G_i' phi> there equals Im<lambda|G_i phi>
// right after member i).
template <typename R>
__device__ void build_run(const MatSlot *__restrict__ slots, const MatSlot &head, const double *__restrict__ params,
                          const double *__restrict__ user, c_t<R> *__restrict__ out) {
  double2 V[4] = {make_double2(1, 0), make_double2(0, 0), make_double2(0, 0), make_double2(1, 0)};
  auto put = [&](int off, int e, double2 v) {
    c_t<R> c;
    c.x = (R)v.x;
    c.y = (R)v.y;
    out[off + e] = c;
  };
  for (int q = head.b - 1; q >= 0; --q) {
    const MatSlot m = slots[head.a + q];
    if (m.a != gNone) {
      double2 G[4];
      if (m.a == gX) {
        G[0] = make_double2(0, 0); G[1] = make_double2(m.g0, 0); G[2] = make_double2(m.g0, 0); G[3] = make_double2(0, 0);
      } else if (m.a == gY) {
        G[0] = make_double2(0, 0); G[1] = make_double2(0, -m.g0); G[2] = make_double2(0, m.g0); G[3] = make_double2(0, 0);
      } else {
        G[0] = make_double2(m.g0, 0); G[1] = make_double2(0, 0); G[2] = make_double2(0, 0); G[3] = make_double2(m.g1, 0);
      }
      double2 T[4];  // V G
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) T[r * 2 + c] = zadd(zmul(V[r * 2], G[c]), zmul(V[r * 2 + 1], G[2 + c]));
      for (int r = 0; r < 2; ++r)  // (V G) V^dagger
        for (int c = 0; c < 2; ++c)
          put(m.out, r * 2 + c, zadd(zmul(T[r * 2], zconj(V[c * 2])), zmul(T[r * 2 + 1], zconj(V[c * 2 + 1]))));
    }
    double2 U[4];
    member_matrix(m, params, user, U);
    double2 W[4];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) W[r * 2 + c] = zadd(zmul(V[r * 2], U[c]), zmul(V[r * 2 + 1], U[2 + c]));
    for (int e = 0; e < 4; ++e) V[e] = W[e];
  }
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) put(head.out, r * 2 + c, head.dagger ? zconj(V[c * 2 + r]) : V[r * 2 + c]);
}

template <typename R>
__global__ void k_build_matrices(const MatSlot *__restrict__ slots, int n_slots,
                                 const double *__restrict__ params, const double *__restrict__ user,
                                 c_t<R> *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slots) return;
  const MatSlot sl = slots[i];
  if (sl.mode == 4) return;  // member of a fused run: built by its head
  if (sl.mode == 3) {
    build_run<R>(slots, sl, params, user, out);
    return;
  }
  if (sl.mode == 5) {  // phase run: E[k] = exp(-i theta/2 (r - 2k)), conjugated when dagger
    const double th = sl.pidx[0] >= 0 ? sl.scale * params[sl.pidx[0]] : sl.cangle[0];
    for (int k = 0; k <= sl.b; ++k) {
      double sn, cs;
      sincos(-0.5 * th * (double)(sl.b - 2 * k), &sn, &cs);
      c_t<R> v;
      v.x = (R)cs;
      v.y = (R)(sl.dagger ? -sn : sn);
      out[sl.out + k] = v;
    }
    return;
  }
  const int D = 1 << sl.k;
  c_t<R> *o = out + sl.out;
  if (sl.kind == SV_MATRIX) {
    for (int r = 0; r < D; ++r)
      for (int c = 0; c < D; ++c) {
        if (sl.mode == 1 && r != c) continue;
        const int64_t e = sl.dagger ? (int64_t)c * D + r : (int64_t)r * D + c;
        const double re = user[2 * (sl.src + e)];
        const double im = sl.dagger ? -user[2 * (sl.src + e) + 1] : user[2 * (sl.src + e) + 1];
        put_entry<R>(sl, o, r, c, re, im);
      }
    return;
  }
  double a[3];
  for (int q = 0; q < 3; ++q) a[q] = sl.pidx[q] >= 0 ? sl.scale * params[sl.pidx[q]] : sl.cangle[q];
  double2 m[256];
  gate_matrix(sl.kind, a, m);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      if (sl.mode == 1 && r != c) continue;
      if (sl.mode == 2 && !((r == sl.a || r == sl.b) && (c == sl.a || c == sl.b))) continue;
      const double2 v = sl.dagger ? make_double2(m[c * D + r].x, -m[c * D + r].y) : m[r * D + c];
      put_entry<R>(sl, o, r, c, v.x, v.y);
    }
}

// ---------------------------------------------------------------------------
// Single-op passes straight from HBM: every thread takes kStreamUnroll units
// per step, issues all their loads before any store (several 128-bit accesses
// in flight per thread), and the grid strides over the units.
// ---------------------------------------------------------------------------
constexpr int kStreamUnroll = 4;

__device__ __forceinline__ uint64_t stream_index(const StreamDev &sd, uint64_t u) {
  for (int j = 0; j < sd.nfix; ++j) {
    const int b = sd.fix[j];
    u = ((u >> b) << (b + 1)) | (u & ((1ull << b) - 1));
  }
  return u | sd.fixval;
}

// Streams of a double-float state compute in double-float like its tile
// passes: the stored complex128 amplitudes are split into float pairs with
// integer operations, and the result costs one FP64 addition per real value
// on the way back (two per amplitude, where FP64 gate arithmetic takes four
// to eight).  Permutations and sign flips (swap, Y, the all-ones negation)
// move the stored doubles as they are.
template <typename R, bool PERM>
using stream_r = typename std::conditional<std::is_same<R, df>::value && PERM, double, R>::type;

template <typename R>
__device__ __forceinline__ c_t<R> stream_in(g_t<R> v) {
  if constexpr (std::is_same<R, df>::value) {
    dfc r;
    r.x = df_split_fast(v.x);
    r.y = df_split_fast(v.y);
    return r;
  } else {
    return v;
  }
}

template <typename R>
__device__ __forceinline__ g_t<R> stream_out(c_t<R> v) {
  if constexpr (std::is_same<R, df>::value)
    return make_double2(df_join_fast(v.x), df_join_fast(v.y));
  else
    return v;
}

template <typename R0, int CODE>
__global__ void __launch_bounds__(kBlock) k_stream_pair(g_t<R0> *__restrict__ psi, uint64_t units, const StreamDev sd,
                                                        const c_t<R0> *__restrict__ mats) {
  using R = stream_r<R0, CODE == mSwap || CODE == mY>;
  using C = c_t<R>;
  C M[4];
  if constexpr (std::is_same<R, R0>::value)
    if (CODE == mGen || CODE == mReal || CODE == mImOff)
#pragma unroll
      for (int q = 0; q < 4; ++q) M[q] = mats[sd.mat + q];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (std::is_same<R, float>::value) {
    if (sd.vec2) {  // units 2v, 2v + 1 are adjacent amplitudes in both members
      float4 *p4 = reinterpret_cast<float4 *>(psi);
      const uint64_t nv = units >> 1;
      for (uint64_t v0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v0 < nv; v0 += stride * kStreamUnroll) {
        uint64_t ia[kStreamUnroll];
        float4 a[kStreamUnroll], b[kStreamUnroll];
#pragma unroll
        for (int r = 0; r < kStreamUnroll; ++r) {
          const uint64_t v = v0 + r * stride;
          ia[r] = v < nv ? stream_index(sd, v << 1) : 0;
          if (v < nv) {
            a[r] = __ldcs(p4 + ((ia[r] + sd.oa) >> 1));
            b[r] = __ldcs(p4 + ((ia[r] + sd.ob) >> 1));
          }
        }
#pragma unroll
        for (int r = 0; r < kStreamUnroll; ++r) {
          if (v0 + r * stride >= nv) break;
          C a0 = make_float2(a[r].x, a[r].y), a1 = make_float2(a[r].z, a[r].w);
          C b0 = make_float2(b[r].x, b[r].y), b1 = make_float2(b[r].z, b[r].w);
          pair_apply<R>(CODE, M, a0, b0);
          pair_apply<R>(CODE, M, a1, b1);
          __stcs(p4 + ((ia[r] + sd.oa) >> 1), make_float4(a0.x, a0.y, a1.x, a1.y));
          __stcs(p4 + ((ia[r] + sd.ob) >> 1), make_float4(b0.x, b0.y, b1.x, b1.y));
        }
      }
      return;
    }
    if (sd.pair16) {  // members 2v, 2v + 1; twice the units per step (one access each)
      constexpr int U2 = 2 * kStreamUnroll;
      float4 *p4 = reinterpret_cast<float4 *>(psi);
      for (uint64_t u0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u0 < units; u0 += stride * U2) {
        uint64_t ia[U2];
        float4 a[U2];
#pragma unroll
        for (int r = 0; r < U2; ++r) {
          const uint64_t u = u0 + r * stride;
          ia[r] = u < units ? stream_index(sd, u) >> 1 : 0;
          if (u < units) a[r] = __ldcs(p4 + ia[r]);
        }
#pragma unroll
        for (int r = 0; r < U2; ++r) {
          if (u0 + r * stride >= units) break;
          C va = make_float2(a[r].x, a[r].y), vb = make_float2(a[r].z, a[r].w);
          pair_apply<R>(CODE, M, va, vb);
          __stcs(p4 + ia[r], make_float4(va.x, va.y, vb.x, vb.y));
        }
      }
      return;
    }
  }
  for (uint64_t u0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u0 < units; u0 += stride * kStreamUnroll) {
    uint64_t ia[kStreamUnroll];
    g_t<R> a[kStreamUnroll], b[kStreamUnroll];
#pragma unroll
    for (int r = 0; r < kStreamUnroll; ++r) {
      const uint64_t u = u0 + r * stride;
      ia[r] = u < units ? stream_index(sd, u) : 0;
      if (u < units) {
        a[r] = __ldcs(psi + ia[r] + sd.oa);
        b[r] = __ldcs(psi + ia[r] + sd.ob);
      }
    }
#pragma unroll
    for (int r = 0; r < kStreamUnroll; ++r) {
      if (u0 + r * stride >= units) break;
      C va = stream_in<R>(a[r]), vb = stream_in<R>(b[r]);
      pair_apply<R>(CODE, M, va, vb);
      __stcs(psi + ia[r] + sd.oa, stream_out<R>(va));
      __stcs(psi + ia[r] + sd.ob, stream_out<R>(vb));
    }
  }
}

template <typename R, int KD, bool NEG>
__device__ __forceinline__ c_t<R> stream_diag_mul(const StreamDev &sd, const c_t<R> (&d)[4], uint64_t i, c_t<R> v) {
  if (NEG) {
    v.x = -v.x;  // every unit is on the all-ones target pattern
    v.y = -v.y;
    return v;
  }
  int idx = (int)((i >> sd.tg0) & 1);
  if (KD == 2) idx = (idx << 1) | (int)((i >> sd.tg1) & 1);
  return cmul(v, pick<c_t<R>, KD>(d, idx));
}

template <typename R0, int KD, bool NEG>
__global__ void __launch_bounds__(kBlock) k_stream_diag(g_t<R0> *__restrict__ psi, uint64_t units, const StreamDev sd,
                                                        const c_t<R0> *__restrict__ mats) {
  using R = stream_r<R0, NEG>;
  using C = c_t<R>;
  C d[4];
  if constexpr (!NEG)
#pragma unroll
    for (int e = 0; e < 4; ++e) d[e] = e < (1 << KD) ? mats[sd.mat + e] : C();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (std::is_same<R, float>::value) {
    if (sd.vec2) {
      float4 *p4 = reinterpret_cast<float4 *>(psi);
      const uint64_t nv = units >> 1;
      for (uint64_t v0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v0 < nv; v0 += stride * kStreamUnroll) {
        uint64_t ia[kStreamUnroll];
        float4 a[kStreamUnroll];
#pragma unroll
        for (int r = 0; r < kStreamUnroll; ++r) {
          const uint64_t v = v0 + r * stride;
          ia[r] = v < nv ? stream_index(sd, v << 1) : 0;
          if (v < nv) a[r] = __ldcs(p4 + (ia[r] >> 1));
        }
#pragma unroll
        for (int r = 0; r < kStreamUnroll; ++r) {
          if (v0 + r * stride >= nv) break;
          const C a0 = stream_diag_mul<R, KD, NEG>(sd, d, ia[r], make_float2(a[r].x, a[r].y));
          const C a1 = stream_diag_mul<R, KD, NEG>(sd, d, ia[r] | 1, make_float2(a[r].z, a[r].w));
          __stcs(p4 + (ia[r] >> 1), make_float4(a0.x, a0.y, a1.x, a1.y));
        }
      }
      return;
    }
  }
  for (uint64_t u0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u0 < units; u0 += stride * kStreamUnroll) {
    uint64_t ia[kStreamUnroll];
    g_t<R> a[kStreamUnroll];
#pragma unroll
    for (int r = 0; r < kStreamUnroll; ++r) {
      const uint64_t u = u0 + r * stride;
      ia[r] = u < units ? stream_index(sd, u) : 0;
      if (u < units) a[r] = __ldcs(psi + ia[r]);
    }
#pragma unroll
    for (int r = 0; r < kStreamUnroll; ++r) {
      if (u0 + r * stride >= units) break;
      __stcs(psi + ia[r], stream_out<R>(stream_diag_mul<R, KD, NEG>(sd, d, ia[r], stream_in<R>(a[r]))));
    }
  }
}

// ---------------------------------------------------------------------------
// Renormalisation: ||psi||^2 as kNormBlocks FP64 partials (each thread sums
// |a|^2 of two amplitudes in the state's precision, then adds in FP64; fixed
// thread-to-element map and tree order), then one scaling pass whose blocks
// all sum the partials in the same order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_fixed(double v, double *red) {
  v += __shfl_down_sync(0xffffffffu, v, 16);
  v += __shfl_down_sync(0xffffffffu, v, 8);
  v += __shfl_down_sync(0xffffffffu, v, 4);
  v += __shfl_down_sync(0xffffffffu, v, 2);
  v += __shfl_down_sync(0xffffffffu, v, 1);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;  // valid in thread 0
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_norm_partials(const g_t<R> *__restrict__ psi, uint64_t N,
                                                          double *__restrict__ partials) {
  __shared__ double red[kBlock / 32];
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (std::is_same<R, float>::value) {
    const float4 *p4 = reinterpret_cast<const float4 *>(psi);
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < (N >> 1); v += stride) {
      const float4 a = __ldcs(p4 + v);
      acc += (double)fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, a.w * a.w)));
    }
  } else {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
      const g_t<R> a = __ldcs(psi + i);
      acc = fma(a.x, a.x, fma(a.y, a.y, acc));
    }
  }
  const double t = block_sum_fixed(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Jacobian-vector product: partials of Re <a|b> (kNormBlocks blocks, fixed order).
template <typename R>
__global__ void __launch_bounds__(kBlock) k_dot_partials(const g_t<R> *__restrict__ a, const g_t<R> *__restrict__ b,
                                                         uint64_t N, double *__restrict__ partials) {
  __shared__ double red[kBlock / 32];
  double acc = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    const g_t<R> x = __ldcs(a + i), y = __ldcs(b + i);
    acc += (double)x.x * (double)y.x + (double)x.y * (double)y.y;
  }
  const double t = block_sum_fixed(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Sparse observable rows: a group of G lanes per row (G a power of two near
// the mean row length; rows strided over all groups of a fixed grid); lanes
// stride the row's stored entries, FP64 complex sums, a fixed shuffle tree
// within the group.  The result is valid in the group's first lane.
template <typename R, int G>
__device__ __forceinline__ double2 csr_row(const g_t<R> *__restrict__ psi, const SparseDev &h, int64_t row, int gl,
                                           bool active) {
  double yr = 0.0, yi = 0.0;
  const int64_t e = active ? __ldg(h.indptr + row + 1) : 0;
  for (int64_t k = active ? __ldg(h.indptr + row) + gl : 0; k < e; k += G) {
    const double2 v = __ldg(h.vals + k);
    const g_t<R> x = psi[__ldg(h.indices + k)];
    yr += v.x * (double)x.x - v.y * (double)x.y;
    yi += v.x * (double)x.y + v.y * (double)x.x;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    yr += __shfl_down_sync(0xffffffffu, yr, o, G);
    yi += __shfl_down_sync(0xffffffffu, yi, o, G);
  }
  return make_double2(yr, yi);
}

template <typename R, int G>
__global__ void __launch_bounds__(kBlock) k_csr_spmv(const g_t<R> *__restrict__ psi, const SparseDev h,
                                                     g_t<R> *__restrict__ out) {
  const int gl = threadIdx.x & (G - 1);
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  const int64_t rows = 1ll << h.n;
  const int64_t first = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
  // every lane of a warp runs the same number of iterations (shuffles need the whole warp)
  const int64_t iters = (rows + groups - 1) / groups;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t row = first + it * groups;
    const bool ok = row < rows;
    const double2 y = csr_row<R, G>(psi, h, row, gl, ok);  // groups past the last row sum nothing
    if (ok && gl == 0) {
      g_t<R> v;
      v.x = y.x;
      v.y = y.y;
      out[row] = v;
    }
  }
}

template <typename R, int G>
__global__ void __launch_bounds__(kBlock) k_csr_expval_partials(const g_t<R> *__restrict__ psi, const SparseDev h,
                                                                double *__restrict__ partials) {
  __shared__ double red[kBlock];
  const int gl = threadIdx.x & (G - 1);
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  const int64_t rows = 1ll << h.n;
  const int64_t first = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
  const int64_t iters = (rows + groups - 1) / groups;
  double acc = 0.0;  // group leader: sum over the group's rows of Re(conj(psi_row) (H psi)_row)
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t row = first + it * groups;
    const bool ok = row < rows;
    const double2 y = csr_row<R, G>(psi, h, row, gl, ok);
    if (ok && gl == 0) {
      const g_t<R> x = psi[row];
      acc += (double)x.x * y.x + (double)x.y * y.y;
    }
  }
  red[threadIdx.x] = gl == 0 ? acc : 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; i += G) t += red[i];
    partials[blockIdx.x] = t;
  }
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_norm_scale(g_t<R> *__restrict__ psi, uint64_t N,
                                                       const double *__restrict__ partials, int nb) {
  __shared__ double sc;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += partials[b];
    sc = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
  }
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (std::is_same<R, float>::value) {
    const float f = (float)sc;
    float4 *p4 = reinterpret_cast<float4 *>(psi);
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < (N >> 1); v += stride) {
      float4 a = __ldcs(p4 + v);
      a.x *= f;
      a.y *= f;
      a.z *= f;
      a.w *= f;
      __stcs(p4 + v, a);
    }
  } else {
    const double f = sc;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
      g_t<R> a = __ldcs(psi + i);
      a.x *= f;
      a.y *= f;
      __stcs(psi + i, a);
    }
  }
}

// Marginal probabilities: block c sums |psi_i|^2 over enumeration indices
// [c L, (c + 1) L), L = 2^chunk_log <= 2^(n-k), so one bin per block; per-thread
// strided FP64 sums, fixed tree (bitwise repeatable).
template <typename R>
__global__ void __launch_bounds__(kBlock) k_probs_partials(const g_t<R> *__restrict__ psi, const ProbsDev pd,
                                                           double *__restrict__ partials) {
  __shared__ double red[kBlock / 32];
  const uint64_t L = 1ull << pd.chunk_log;
  const uint64_t j0 = (uint64_t)blockIdx.x * L;
  const uint64_t bin = j0 >> (pd.n - pd.k);
  uint64_t binmask = 0;
  for (int j = 0; j < pd.k; ++j)
    if ((bin >> (pd.k - 1 - j)) & 1) binmask |= 1ull << pd.bitpos[j];
  const uint64_t other0 = j0 & ((1ull << (pd.n - pd.k)) - 1);
  double acc = 0.0;
  for (uint64_t t = threadIdx.x; t < L; t += blockDim.x) {
    uint64_t i = other0 + t;
    for (int q = 0; q < pd.k; ++q) {
      const int b = pd.pos[q];
      i = ((i >> b) << (b + 1)) | (i & ((1ull << b) - 1));
    }
    const g_t<R> a = __ldcs(psi + (i | binmask));
    acc += (double)a.x * (double)a.x + (double)a.y * (double)a.y;
  }
  const double t = block_sum_fixed(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Marginal probabilities with small bins (2^(n-k) <= 64 amplitudes each): one
// thread per bin sums its amplitudes in ascending order and writes the bin.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_probs_small(const g_t<R> *__restrict__ psi, const ProbsDev pd,
                                                        double *__restrict__ out) {
  const uint64_t bin = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (bin >> pd.k) return;
  uint64_t binmask = 0;
  for (int j = 0; j < pd.k; ++j)
    if ((bin >> (pd.k - 1 - j)) & 1) binmask |= 1ull << pd.bitpos[j];
  double acc = 0.0;
  for (uint64_t o = 0; o < (1ull << (pd.n - pd.k)); ++o) {
    uint64_t i = o;
    for (int q = 0; q < pd.k; ++q) {
      const int b = pd.pos[q];
      i = ((i >> b) << (b + 1)) | (i & ((1ull << b) - 1));
    }
    const g_t<R> a = __ldcs(psi + (i | binmask));
    acc += (double)a.x * (double)a.x + (double)a.y * (double)a.y;
  }
  out[bin] = acc;
}

template <typename R>
__global__ void k_set_basis(g_t<R> *psi, uint64_t N, uint64_t index) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    g_t<R> v;
    v.x = (i == index) ? 1 : 0;
    v.y = 0;
    psi[i] = v;
  }
}

// ---------------------------------------------------------------------------
// Batched circuits: one persistent launch drains a queue of work items
// (circuit, pass, tile).  Items are numbered so that every tile of pass p of a
// circuit precedes every tile of its pass p + 1; a CTA holding an item of pass
// p + 1 waits (bounded, %globaltimer) until all tiles of pass p are done.  An
// item is only ever taken by a running CTA, so the oldest unfinished item
// always has its inputs and the queue cannot deadlock.  States live in L2-sized
// waves of circuits (the item order interleaves the circuits of a wave).
// Loads bypass L1 (cp.async.cg): another SM may have written the amplitudes
// in the previous pass.  The first pass writes the basis state straight into
// shared memory; the last pass adds the Z-word expectation partials of its
// tile (one slot per term and tile, summed later in fixed order) and stores
// the final state only when asked.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kBatchChunk = 8;  // work items a CTA takes from the queue at once

// Z-word partials of a batch tile in its last pass (as in k_expval_z): thread
// u holds p_i = |psi|^2 at l = u + kBlock i (i < 2^NB, NB = T - 8), one
// Walsh-Hadamard transform gives every word's signed sum over them, written to
// the thread's own column of sw; zs[t] holds word t's local mask (low 32 bits)
// and its parity over the tile bits (bit 32).  Per-warp sums go to accs.
template <typename R, int NB>
__device__ __forceinline__ void batch_zsums(const R (&p)[1 << NB], R *sw, const uint64_t *zs, int n_terms,
                                            double *accs, int nwarps, int warp, int lane) {
  constexpr int NA = 1 << NB;
  R w[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) w[i] = p[i];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int i = 0; i < NA; ++i)
      if (!(i >> b & 1)) {
        const R x = w[i], y = w[i | (1 << b)];
        w[i] = x + y;
        w[i | (1 << b)] = x - y;
      }
  const int u = threadIdx.x;
#pragma unroll
  for (int i = 0; i < NA; ++i) sw[i * kBlock + u] = w[i];
  for (int t0 = 0; t0 < n_terms; t0 += 32) {
    R v[32][1];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      v[t][0] = R(0);
      if (t0 + t < n_terms) {
        const uint64_t z = zs[t0 + t];
        const uint32_t zl = (uint32_t)z;
        const uint32_t neg = (uint32_t)(z >> 32 & 1) ^ (uint32_t)(__popc(zl & (uint32_t)u & 0xFFu) & 1);
        v[t][0] = flip_sign(sw[((zl >> 8) & (NA - 1)) * kBlock + u], neg);
      }
    }
    int slot;
    const bool writer = warp_reduce_scatter<R, 32, 1>(v, lane, slot);
    if (writer && t0 + slot < n_terms) accs[(t0 + slot) * nwarps + warp] = (double)v[0][0];
  }
}

template <typename R, int NB>
__device__ __forceinline__ void batch_load_p(const c_t<R> *s, R (&p)[1 << NB]) {
#pragma unroll
  for (int i = 0; i < (1 << NB); ++i) {
    const c_t<R> a = s[threadIdx.x + kBlock * i];
    p[i] = a.x * a.x + a.y * a.y;
  }
}

template <typename R, int MAXK>
__global__ void __launch_bounds__(kBlock, 3) k_batch(g_t<R> *__restrict__ states, const BatchCircuit *__restrict__ circs,
                                                   const PassDev *__restrict__ passes, const OpDev *__restrict__ ops,
                                                   const c_t<R> *__restrict__ mats, const uint64_t *__restrict__ aux,
                                                   const BatchSeg *__restrict__ segs,
                                                   int n_segs, long long total_items, const ZTerm *__restrict__ terms,
                                                   double *__restrict__ partials, int *done,
                                                   unsigned long long *head, int *err, int store_final,
                                                   unsigned long long timeout_ns, int max_T, int max_terms,
                                                   int no_publish) {
  using C = c_t<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  C *s = reinterpret_cast<C *>(smem);
  uint64_t *lut = reinterpret_cast<uint64_t *>(s + (1 << max_T));
  double *accs = reinterpret_cast<double *>(lut + (1 << max_T));  // [max_terms][nwarps]
  uint64_t *zs = reinterpret_cast<uint64_t *>(accs + max_terms * (blockDim.x >> 5));  // [max_terms]
  __shared__ long long s_first;
  __shared__ int s_seg, s_abort, s_new_seg;
  __shared__ PassDev s_pass;
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int cur_seg = -1;  // segment whose pass / LUT / dependency are in place

  for (;;) {
    if (threadIdx.x == 0) {
      s_abort = *reinterpret_cast<volatile int *>(err);
      s_first = (long long)atomicAdd(head, (unsigned long long)kBatchChunk);
    }
    __syncthreads();
    const long long first = s_first;
    if (first >= total_items || s_abort) break;
    const long long last_item = min(first + (long long)kBatchChunk, total_items);
    if (threadIdx.x == 0) {  // segment of the chunk's first item: last segment with first_item <= item
      int lo = 0, hi = n_segs - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].first_item <= first)
          lo = mid;
        else
          hi = mid - 1;
      }
      s_seg = lo;
    }
    for (long long item = first; item < last_item; ++item) {
      if (threadIdx.x == 0) {
        int sg_i = (item == first) ? s_seg : cur_seg;
        while (sg_i + 1 < n_segs && segs[sg_i + 1].first_item <= item) ++sg_i;
        s_seg = sg_i;
        s_new_seg = sg_i != cur_seg;
        if (s_new_seg) {
          const BatchSeg sg = segs[sg_i];
          const int pidx = circs[sg.circ].pass_begin + sg.pass;
          s_pass = passes[pidx];
          if (sg.pass > 0) {  // all tiles of the previous pass of this circuit must be done
            const unsigned long long t0 = global_ns();
            while (ld_acquire(&done[pidx - 1]) < sg.ntiles) {
              if (*reinterpret_cast<volatile int *>(err) || global_ns() - t0 > timeout_ns) {
                atomicExch(err, 1);
                s_abort = 1;
                break;
              }
              __nanosleep(64);
            }
            __threadfence();
          }
        }
      }
      __syncthreads();
      if (s_abort) break;
      const int seg_i = s_seg;
      const BatchSeg sg = segs[seg_i];
      const BatchCircuit cc = circs[sg.circ];
      const int pidx = cc.pass_begin + sg.pass;
      const PassDev &pass = s_pass;
      if (s_new_seg) {
        build_lut(lut, pass);
        __syncthreads();
      }
      cur_seg = seg_i;
      const uint64_t tile = (uint64_t)(item - sg.first_item);
      TileGeom tg;
      tg.T = pass.T;
      tg.nlow = pass.nlow;
      tg.A = 1 << pass.T;
      tg.lowmask = (1u << pass.nlow) - 1u;
      tg.lut = lut;
      tg.base = tile_base(pass, tile);
      g_t<R> *psi = states + cc.state_off;
      if (sg.pass == 0) {
        for (int l = threadIdx.x; l < tg.A; l += blockDim.x) {
          C v;
          v.x = tg.gidx(l) == cc.basis ? R(1) : R(0);
          v.y = R(0);
          s[l] = v;
        }
      } else {
        load_tile_async<R>(psi, s, tg);  // cp.async.cg: L2 only, as the previous pass ran on other SMs
        tile_async_wait();
        tile_async_convert<R>(s, tg.A);
      }
      __syncthreads();
      for (int o = pass.op_begin; o < pass.op_end; ++o) {
        const OpDev &op = ops[o];
        if (op.sync_prev && o > pass.op_begin) __syncthreads();
        apply_op<R, MAXK>(s, tg, op, mats, aux);
      }
      __syncthreads();
      const bool last = sg.pass == cc.n_pass - 1;
      if (last && cc.n_terms > 0 && pass.T >= 8 && pass.T <= 12) {
        // <Z word> partials of this tile, sum_l (-1)^popcount(g & z) |psi_l|^2, by one
        // Walsh-Hadamard transform per thread (the tile buffer holds the transforms)
        for (int t = threadIdx.x; t < cc.n_terms; t += blockDim.x) {
          const uint64_t z = terms[cc.term_begin + t].z;
          uint32_t zl = 0;
          for (int b = 0; b < pass.T; ++b)
            if (z >> pass.pos[b] & 1) zl |= 1u << b;
          zs[t] = zl | ((uint64_t)(__popcll(tg.base & z) & 1) << 32);
        }
        R pr[16];
        if (pass.T == 12) batch_load_p<R, 4>(s, reinterpret_cast<R(&)[16]>(pr));
        else if (pass.T == 11) batch_load_p<R, 3>(s, reinterpret_cast<R(&)[8]>(pr));
        else if (pass.T == 10) batch_load_p<R, 2>(s, reinterpret_cast<R(&)[4]>(pr));
        else if (pass.T == 9) batch_load_p<R, 1>(s, reinterpret_cast<R(&)[2]>(pr));
        else batch_load_p<R, 0>(s, reinterpret_cast<R(&)[1]>(pr));
        __syncthreads();  // the words' masks are in place; every thread has read its amplitudes
        if (store_final) {
          store_tile<R>(psi, s, tg);
          __syncthreads();
        }
        R *sw = reinterpret_cast<R *>(s);
        if (pass.T == 12) batch_zsums<R, 4>(reinterpret_cast<R(&)[16]>(pr), sw, zs, cc.n_terms, accs, nwarps, warp, lane);
        else if (pass.T == 11) batch_zsums<R, 3>(reinterpret_cast<R(&)[8]>(pr), sw, zs, cc.n_terms, accs, nwarps, warp, lane);
        else if (pass.T == 10) batch_zsums<R, 2>(reinterpret_cast<R(&)[4]>(pr), sw, zs, cc.n_terms, accs, nwarps, warp, lane);
        else if (pass.T == 9) batch_zsums<R, 1>(reinterpret_cast<R(&)[2]>(pr), sw, zs, cc.n_terms, accs, nwarps, warp, lane);
        else batch_zsums<R, 0>(reinterpret_cast<R(&)[1]>(pr), sw, zs, cc.n_terms, accs, nwarps, warp, lane);
        __syncthreads();
        for (int t = threadIdx.x; t < cc.n_terms; t += blockDim.x) {
          double v = 0.0;
          for (int w = 0; w < nwarps; ++w) v += accs[t * nwarps + w];
          partials[cc.part_begin + (int64_t)t * sg.ntiles + (int64_t)tile] = v;
        }
      } else if (last && cc.n_terms > 0) {
        // <Z word> partial of this tile: sum_l (-1)^popcount(g & z) |psi_l|^2
        for (int t = 0; t < cc.n_terms; ++t) {
          const uint64_t z = terms[cc.term_begin + t].z;
          R acc = R(0);
          for (int l = threadIdx.x; l < tg.A; l += blockDim.x) {
            const C a = s[l];
            const R pr = a.x * a.x + a.y * a.y;
            acc += (__popcll(tg.gidx(l) & z) & 1) ? -pr : pr;
          }
          acc = warp_sum(acc);
          if (lane == 0) accs[t * nwarps + warp] = (double)acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cc.n_terms; t += blockDim.x) {
          double v = 0.0;
          for (int w = 0; w < nwarps; ++w) v += accs[t * nwarps + w];
          partials[cc.part_begin + (int64_t)t * sg.ntiles + (int64_t)tile] = v;
        }
      }
      if (!last || (store_final && !(cc.n_terms > 0 && pass.T >= 8 && pass.T <= 12))) store_tile<R>(psi, s, tg);
      __syncthreads();
      if (threadIdx.x == 0 && pidx != no_publish) {  // no_publish >= 0 only in failure-path tests
        __threadfence();
        atomicAdd(&done[pidx], 1);
      }
    }
    if (s_abort) break;
  }
}

}  // namespace sv

// Host runtime and C ABI of libsv.so: argument validation, the gate-fusion
// planner, planned programs (device tables + workspace) and the adjoint sweep
// driver.  Device work goes through the Launch<R> launchers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "df64.cuh"
#include "sv.h"
#include "sv_internal.h"

using namespace sv;

struct sv_state;

namespace {

thread_local std::string g_err;
std::atomic<size_t> g_alloc_cap{0};
std::atomic<size_t> g_alloc_bytes{0};

sv_status fail(sv_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

sv_status cuda_fail(cudaError_t e, const char *where) {
  return fail(SV_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define SV_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

sv_status dev_alloc(void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return SV_OK;
  const size_t cap = g_alloc_cap.load();
  if (cap && g_alloc_bytes.load() + bytes > cap)
    return fail(SV_ERR_OOM, "allocation of %zu bytes exceeds the cap of %zu bytes", bytes, cap);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(SV_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  g_alloc_bytes += bytes;
  return SV_OK;
}

void dev_free(void *p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  g_alloc_bytes -= bytes;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  }
  return n;
}

// ---- kernel timing (roofline accounting) -------------------------------------
struct TimedLaunch {
  cudaEvent_t a, b;
  int cls;
};
std::atomic<bool> g_timing{false};
std::mutex g_timing_mu;  // guards the four below: launches may come from several host threads
std::vector<TimedLaunch> g_pending;
std::vector<cudaEvent_t> g_event_pool;
double g_class_ms[SV_KERNEL_CLASSES] = {0};
int64_t g_class_n[SV_KERNEL_CLASSES] = {0};

// An event from the pool (or a new one); the caller holds g_timing_mu.
cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Bracket one launch with events when timing is on.
struct LaunchTimer {
  cudaStream_t st;
  int cls;
  cudaEvent_t a = nullptr;
  LaunchTimer(cudaStream_t s_, int c) : st(s_), cls(c) {
    if (g_timing.load()) {
      std::lock_guard<std::mutex> lk(g_timing_mu);
      a = take_event();
      cudaEventRecord(a, st);
    }
  }
  ~LaunchTimer() {
    if (a) {
      std::lock_guard<std::mutex> lk(g_timing_mu);
      cudaEvent_t b = take_event();
      cudaEventRecord(b, st);
      g_pending.push_back({a, b, cls});
    }
  }
};

// ---- gate tables -----------------------------------------------------------
int kind_arity(int kind) {
  switch (kind) {
    case SV_SWAP: case SV_ISING_XX: case SV_ISING_YY: case SV_ISING_ZZ: case SV_ISING_XY:
    case SV_SINGLE_EXCITATION: return 2;
    case SV_DOUBLE_EXCITATION: return 4;
    case SV_MATRIX: return -1;
    default: return 1;
  }
}

int kind_nparams(int kind) {
  switch (kind) {
    case SV_PHASE_SHIFT: case SV_RX: case SV_RY: case SV_RZ: case SV_ISING_XX: case SV_ISING_YY:
    case SV_ISING_ZZ: case SV_ISING_XY: case SV_SINGLE_EXCITATION: case SV_DOUBLE_EXCITATION: return 1;
    case SV_ROT: return 3;
    default: return 0;
  }
}

bool kind_diag(int kind) {
  switch (kind) {
    case SV_IDENTITY: case SV_PAULI_Z: case SV_S: case SV_T: case SV_PHASE_SHIFT: case SV_RZ:
    case SV_ISING_ZZ: return true;
    default: return false;
  }
}

// s of U(t) = exp(i s t G) for the one-angle kinds.
double kind_gen_s(int kind) {
  switch (kind) {
    case SV_PHASE_SHIFT: return 1.0;
    case SV_ISING_XY: return 0.25;
    default: return -0.5;
  }
}

// ---- host op ---------------------------------------------------------------
struct HOp {
  int kind = 0, k = 1;
  int tw[kMaxTargets] = {0};
  int nc = 0;
  int cw[SV_MAX_CONTROLS] = {0};
  int cv[SV_MAX_CONTROLS] = {0};
  int pidx[3] = {-1, -1, -1};
  double cang[3] = {0, 0, 0};
  double scale = 1.0;
  int adjoint = 0;
  int64_t msrc = 0;
  bool diag = false;
  bool train = false;   // adjoint plan: one angle bound to a parameter
};

sv_status validate_op(int n, const sv_op &op, int n_params, const double *matrices, int64_t n_mat,
                      const double *params, bool params_on_host) {
  if (op.kind < 0 || op.kind >= SV_OP_KIND_COUNT) return fail(SV_ERR_ARG, "unknown op kind %d", op.kind);
  const int ar = kind_arity(op.kind);
  if (op.kind == SV_MATRIX) {
    if (op.n_targets < 1 || op.n_targets > SV_MAX_TARGETS)
      return fail(SV_ERR_ARG, "SV_MATRIX takes 1..%d targets, got %d", SV_MAX_TARGETS, op.n_targets);
    const int64_t need = (int64_t)1 << (2 * op.n_targets);
    if (!matrices || op.matrix_offset < 0 || op.matrix_offset > n_mat - need)  // no overflow in the sum
      return fail(SV_ERR_ARG, "SV_MATRIX data out of range (offset %lld, %lld entries needed)",
                  (long long)op.matrix_offset, (long long)need);
    for (int64_t e = 0; e < 2 * need; ++e)
      if (!std::isfinite(matrices[2 * op.matrix_offset + e])) return fail(SV_ERR_ARG, "SV_MATRIX entry is not finite");
  } else if (op.n_targets != ar) {
    return fail(SV_ERR_ARG, "op kind %d takes %d target wires, got %d", op.kind, ar, op.n_targets);
  }
  if (op.n_controls < 0 || op.n_controls > SV_MAX_CONTROLS)
    return fail(SV_ERR_ARG, "n_controls %d out of range", op.n_controls);
  uint64_t seen = 0;
  for (int j = 0; j < op.n_targets; ++j) {
    const int w = op.targets[j];
    if (w < 0 || w >= n) return fail(SV_ERR_ARG, "target wire %d out of range [0, %d)", w, n);
    if (seen >> w & 1) return fail(SV_ERR_ARG, "wire %d used twice in one op", w);
    seen |= 1ull << w;
  }
  for (int c = 0; c < op.n_controls; ++c) {
    const int w = op.controls[c];
    if (w < 0 || w >= n) return fail(SV_ERR_ARG, "control wire %d out of range [0, %d)", w, n);
    if (seen >> w & 1) return fail(SV_ERR_ARG, "wire %d used twice in one op", w);
    seen |= 1ull << w;
    if (op.control_values[c] != 0 && op.control_values[c] != 1)
      return fail(SV_ERR_ARG, "control value must be 0 or 1");
  }
  const int np = kind_nparams(op.kind);
  for (int a = 0; a < np; ++a) {
    const int pi = op.param_index[a];
    if (pi >= 0) {
      if (pi >= n_params) return fail(SV_ERR_ARG, "param_index %d >= n_params %d", pi, n_params);
      if (!std::isfinite(op.scale)) return fail(SV_ERR_ARG, "op scale is not finite");
      if (params_on_host && params && !std::isfinite(params[pi]))
        return fail(SV_ERR_ARG, "parameter %d is not finite", pi);
    } else if (!std::isfinite(op.const_angle[a])) {
      return fail(SV_ERR_ARG, "constant angle is not finite");
    }
  }
  return SV_OK;
}

bool user_matrix_diag(const double *m, int64_t off, int k) {
  const int D = 1 << k;
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c)
      if (r != c && (m[2 * (off + (int64_t)r * D + c)] != 0.0 || m[2 * (off + (int64_t)r * D + c) + 1] != 0.0))
        return false;
  return true;
}

HOp to_hop(const sv_op &op, const double *matrices) {
  HOp h;
  h.kind = op.kind;
  h.k = op.kind == SV_MATRIX ? op.n_targets : kind_arity(op.kind);
  for (int j = 0; j < h.k; ++j) h.tw[j] = op.targets[j];
  h.nc = op.n_controls;
  for (int c = 0; c < h.nc; ++c) {
    h.cw[c] = op.controls[c];
    h.cv[c] = op.control_values[c];
  }
  for (int a = 0; a < 3; ++a) {
    h.pidx[a] = a < kind_nparams(op.kind) ? op.param_index[a] : -1;
    h.cang[a] = op.const_angle[a];
  }
  h.scale = op.scale;
  h.adjoint = op.adjoint ? 1 : 0;
  h.msrc = op.matrix_offset;
  h.diag = op.kind == SV_MATRIX ? user_matrix_diag(matrices, op.matrix_offset, h.k) : kind_diag(op.kind);
  return h;
}

// Rot(a, b, c) = RZ(c) RY(b) RZ(a): three one-angle ops (reversed and each
// inverted under adjoint).  Every other op maps to itself.
void expand_op(const HOp &h, std::vector<HOp> &out) {
  if (h.kind != SV_ROT) {
    HOp e = h;
    e.train = kind_nparams(h.kind) == 1 && h.pidx[0] >= 0;
    out.push_back(e);
    return;
  }
  const int kinds[3] = {SV_RZ, SV_RY, SV_RZ};
  int order[3] = {0, 1, 2};
  if (h.adjoint) std::swap(order[0], order[2]);
  for (int q = 0; q < 3; ++q) {
    const int a = order[q];
    HOp e = h;
    e.kind = kinds[a];
    e.pidx[0] = h.pidx[a];
    e.pidx[1] = e.pidx[2] = -1;
    e.cang[0] = h.cang[a];
    e.diag = kind_diag(e.kind);
    e.train = h.pidx[a] >= 0;
    out.push_back(e);
  }
}

// ---- planner -----------------------------------------------------------------
struct Step {
  int dense_k;  // 0: fused pass `index`; 1: dense k>4 op `index` (dk_ops)
  int index;
};

struct Plan {
  std::vector<PassDev> passes;
  std::vector<OpDev> ops;      // micro-op tables of all passes, concatenated
  std::vector<Step> steps;
  std::vector<OpDev> dk_ops;   // one op per dense_k step (global targets)
  std::vector<int> train_hop;  // trainable slot -> HOp index (sweep order)
  int n_train = 0;
  std::vector<uint64_t> aux;   // phase-run member records (two words each)
};

// Matrix-slot allocator shared by the forward and adjoint plans of a program.
struct SlotTable {
  std::vector<MatSlot> slots;
  size_t entries = 0;
  int add(const HOp &h, bool dagger, int mode, int a = 0, int b = 0) {
    MatSlot m;
    memset(&m, 0, sizeof(m));
    m.kind = h.kind;
    m.k = h.k;
    m.dagger = dagger ? 1 : 0;
    m.mode = mode;
    m.a = a;
    m.b = b;
    m.out = (int)entries;
    for (int q = 0; q < 3; ++q) {
      m.pidx[q] = h.pidx[q];
      m.cangle[q] = h.cang[q];
    }
    m.scale = h.scale;
    m.src = h.msrc;
    slots.push_back(m);
    entries += mode == 0 ? (size_t)1 << (2 * h.k) : (mode == 1 ? (size_t)1 << h.k : 4);
    return m.out;
  }
  // Fused run: a head slot (the run's 2x2 product) followed by its members;
  // gens[i] is member i's generator (code, g0, g1) or code gNone.  Returns the
  // product's offset; gmat = first generator output (consecutive, 4 each).
  struct Gen {
    int code;
    double g0, g1;
  };
  int add_run(const std::vector<const HOp *> &mem, const std::vector<Gen> &gens, bool dagger, int &gmat) {
    MatSlot hd;
    memset(&hd, 0, sizeof(hd));
    hd.kind = SV_MATRIX;
    hd.k = 1;
    hd.dagger = dagger ? 1 : 0;
    hd.mode = 3;
    hd.a = (int)slots.size() + 1;
    hd.b = (int)mem.size();
    hd.out = (int)entries;
    entries += 4;
    slots.push_back(hd);
    gmat = (int)entries;
    for (size_t i = 0; i < mem.size(); ++i) {
      const HOp &h = *mem[i];
      MatSlot m;
      memset(&m, 0, sizeof(m));
      m.kind = h.kind;
      m.k = 1;
      m.dagger = h.adjoint ? 1 : 0;
      m.mode = 4;
      m.a = gens[i].code;
      m.g0 = gens[i].g0;
      m.g1 = gens[i].g1;
      for (int q = 0; q < 3; ++q) {
        m.pidx[q] = h.pidx[q];
        m.cangle[q] = h.cang[q];
      }
      m.scale = h.scale;
      m.src = h.msrc;
      if (gens[i].code != gNone) {
        m.out = (int)entries;
        entries += 4;
      }
      slots.push_back(m);
    }
    return hd.out;
  }
  // Phase run of r members sharing h's angle: entries E[0..r].
  int add_phase(const HOp &h, int r, bool dagger) {
    MatSlot m;
    memset(&m, 0, sizeof(m));
    m.kind = h.kind;
    m.k = h.k;
    m.dagger = dagger ? 1 : 0;
    m.mode = 5;
    m.b = r;
    m.out = (int)entries;
    for (int q = 0; q < 3; ++q) {
      m.pidx[q] = h.pidx[q];
      m.cangle[q] = h.cang[q];
    }
    m.scale = h.scale;
    slots.push_back(m);
    entries += (size_t)r + 1;
    return m.out;
  }
};

int popc(uint64_t x) { return __builtin_popcountll(x); }

uint64_t fill_bits(uint64_t bits, int n, int T, int nlow_pref) {
  for (int b = 0; b < nlow_pref && b < n && popc(bits) < T; ++b) bits |= 1ull << b;
  for (int b = 0; b < n && popc(bits) < T; ++b) bits |= 1ull << b;
  return bits;
}

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

uint64_t low_bits(int n, int T, int nlow_pref) {
  uint64_t b = 0;
  for (int i = 0; i < nlow_pref && i < n && i < T; ++i) b |= 1ull << i;
  return b;
}

// Gate structure: the 2x2 blocks (member patterns a, b) of a non-diagonal gate,
// each block's matrix code and its generator restricted to the block.
struct Block {
  int a, b;
  int8_t code, gcode;
  float gs;
};

bool gate_blocks(const HOp &h, std::vector<Block> &out) {
  out.clear();
  switch (h.kind) {
    case SV_PAULI_X: out.push_back({0, 1, mSwap, gNone, 0}); return true;
    case SV_PAULI_Y: out.push_back({0, 1, mY, gNone, 0}); return true;
    case SV_HADAMARD: out.push_back({0, 1, mReal, gNone, 0}); return true;
    case SV_RX: out.push_back({0, 1, mImOff, gX, 1}); return true;
    case SV_RY: out.push_back({0, 1, mReal, gY, 1}); return true;
    case SV_ROT: out.push_back({0, 1, mGen, gNone, 0}); return true;
    case SV_SWAP: out.push_back({1, 2, mSwap, gNone, 0}); return true;
    case SV_ISING_XX:
      out.push_back({0, 3, mImOff, gX, 1});
      out.push_back({1, 2, mImOff, gX, 1});
      return true;
    case SV_ISING_YY:
      out.push_back({0, 3, mImOff, gX, -1});
      out.push_back({1, 2, mImOff, gX, 1});
      return true;
    case SV_ISING_XY: out.push_back({1, 2, mImOff, gX, 2}); return true;
    case SV_SINGLE_EXCITATION: out.push_back({1, 2, mReal, gY, 1}); return true;
    case SV_DOUBLE_EXCITATION: out.push_back({3, 12, mReal, gY, 1}); return true;
    case SV_MATRIX:
      if (h.k == 1) {
        out.push_back({0, 1, mGen, gNone, 0});
        return true;
      }
      return false;  // dense block
    default: return false;
  }
}

// Diagonal generator restricted to the pattern: g = ga / gb by parity of pattern & zmask.
void diag_generator(int kind, int &zmask, float &ga, float &gb) {
  zmask = 1;
  ga = 1.f;
  gb = -1.f;
  if (kind == SV_PHASE_SHIFT) {
    ga = 0.f;
    gb = 1.f;
  } else if (kind == SV_ISING_ZZ) {
    zmask = 3;
  }
}

OpDev blank_op(int n, const HOp &h) {
  OpDev o;
  memset(&o, 0, sizeof(o));
  o.k = (int8_t)h.k;
  for (int j = 0; j < h.k; ++j) o.tg[j] = (int8_t)(n - 1 - h.tw[j]);
  for (int c = 0; c < h.nc; ++c) {
    const uint64_t b = 1ull << (n - 1 - h.cw[c]);
    o.cmask |= b;
    if (h.cv[c]) o.cval |= b;
  }
  o.train = -1;
  o.slot = -1;
  o.sync_prev = 1;
  return o;
}

// Split an op's controls into the pass's local bits and fixed tile bits; for
// diagonal ops record which targets are local (tl[j], else -1).
void localise(OpDev &o, const PassDev &pd) {
  o.lcmask = o.lcval = 0;
  o.hcmask = o.hcval = 0;
  for (int b = 0; b < 64; ++b) {
    if (!((o.cmask >> b) & 1)) continue;
    const bool v = (o.cval >> b) & 1;
    int li = -1;
    for (int i = 0; i < pd.T; ++i)
      if (pd.pos[i] == b) li = i;
    if (li >= 0) {
      o.lcmask |= 1u << li;
      if (v) o.lcval |= 1u << li;
    } else {
      o.hcmask |= 1ull << b;
      if (v) o.hcval |= 1ull << b;
    }
  }
  if (o.kind == kDiag)
    for (int j = 0; j < o.k && j < 4; ++j) {
      o.tl[j] = -1;
      for (int i = 0; i < pd.T; ++i)
        if (pd.pos[i] == o.tg[j]) o.tl[j] = (int8_t)i;
    }
}

// Lower one gate into micro-ops inside a pass (dagger: store U^dagger blocks).
void lower_gate(int n, const HOp &h, const PassDev &pd, bool dagger, int train, int slot, SlotTable &st,
                std::vector<OpDev> &out) {
  const size_t first_out = out.size();
  struct Fin {
    std::vector<OpDev> &v;
    size_t f;
    const PassDev &pd;
    ~Fin() {
      for (size_t i = f; i < v.size(); ++i) localise(v[i], pd);
    }
  } fin{out, first_out, pd};
  const bool eff_dagger = (h.adjoint != 0) != dagger;
  OpDev base = blank_op(n, h);
  base.train = h.train ? train : -1;
  base.slot = h.train ? slot : -1;
  if (h.diag) {
    OpDev o = base;
    o.kind = kDiag;
    o.code = (h.kind == SV_PAULI_Z) ? dNeg : dGen;
    if (o.code == dGen) o.mat = st.add(h, eff_dagger, 1);
    if (h.train) {
      o.gcode = gDiag;
      diag_generator(h.kind, o.zmask, o.ga, o.gb);
    }
    out.push_back(o);
    return;
  }
  int tl[kMaxTargets];
  for (int j = 0; j < h.k; ++j) {
    tl[j] = -1;
    for (int i = 0; i < pd.T; ++i)
      if (pd.pos[i] == n - 1 - h.tw[j]) tl[j] = i;
  }
  int ts[4] = {0, 0, 0, 0};
  for (int j = 0; j < h.k && j < 4; ++j) ts[j] = tl[j];
  std::sort(ts, ts + std::min(h.k, 4));
  std::vector<Block> blocks;
  if (gate_blocks(h, blocks)) {
    bool first = true;
    for (const Block &bl : blocks) {
      OpDev o = base;
      o.kind = kPair;
      o.code = bl.code;
      for (int j = 0; j < 4; ++j) o.ts[j] = (int8_t)ts[j];
      for (int j = 0; j < h.k; ++j) o.tl[j] = (int8_t)tl[j];
      o.oa = o.ob = 0;
      for (int j = 0; j < h.k; ++j) {
        if ((bl.a >> (h.k - 1 - j)) & 1) o.oa += 1 << tl[j];
        if ((bl.b >> (h.k - 1 - j)) & 1) o.ob += 1 << tl[j];
      }
      if (bl.code == mGen || bl.code == mReal || bl.code == mImOff) o.mat = st.add(h, eff_dagger, 2, bl.a, bl.b);
      if (h.train) {
        o.gcode = bl.gcode;
        o.gs = bl.gs;
      }
      o.sync_prev = first ? 1 : 0;  // blocks of one gate are disjoint
      first = false;
      out.push_back(o);
    }
    return;
  }
  OpDev o = base;  // dense user block on 2-4 local wires
  o.kind = kDense;
  for (int j = 0; j < 4; ++j) o.ts[j] = (int8_t)ts[j];
  for (int j = 0; j < h.k; ++j) o.tl[j] = (int8_t)tl[j];
  o.mat = st.add(h, eff_dagger, 0);
  out.push_back(o);
}

// Generator of a trainable single-wire gate as the kernels accumulate it:
// gs X or gs Y on the pair, diag(ga, gb) for a diagonal.
bool single_wire_generator(const HOp &h, SlotTable::Gen &g) {
  g = {gNone, 0.0, 0.0};
  if (!h.train) return true;
  if (h.diag) {
    int zm;
    float ga, gb;
    diag_generator(h.kind, zm, ga, gb);
    g = {gDiag, ga, gb};
    return true;
  }
  std::vector<Block> bl;
  if (!gate_blocks(h, bl) || bl.size() != 1 || bl[0].gcode == gNone) return false;
  g = {bl[0].gcode, bl[0].gs, 0.0};
  return true;
}

bool fusable(const HOp &h) {
  if (h.kind == SV_IDENTITY || h.k != 1 || h.nc != 0) return false;
  SlotTable::Gen g;
  return single_wire_generator(h, g);
}

// Phase runs: adjacent uncontrolled RZ / IsingZZ ops with one angle source
// (same parameter and scale, or the same constant, and the same adjoint flag)
// multiply by exp(-i theta/2 sum_j (-1)^p_j): one diagonal pass.
bool phase_member(const HOp &h) {
  return h.diag && h.nc == 0 && (h.kind == SV_RZ || h.kind == SV_ISING_ZZ);
}

// Same angle source; trainable members (adjoint plans) then share one
// Jacobian slot: their contributions all go to the same parameter column.
bool same_angle(const HOp &a, const HOp &b) {
  if (a.adjoint != b.adjoint || a.pidx[0] != b.pidx[0] || a.train != b.train) return false;
  return a.pidx[0] >= 0 ? a.scale == b.scale : a.cang[0] == b.cang[0];
}

enum GroupKind { gSingle = 0, gRun = 1, gPhaseRun = 2 };
struct Group {
  GroupKind kind;
  std::vector<int> m;  // member op indices, forward order
};

// Runs of single-wire gates: op i joins the open run on its wire when no gate
// since the run's first member touched that wire (the ops in between act on
// other wires and commute with it).  A run is kept when it has >= 2 members,
// one of them non-diagonal, and at most kMaxFuseGen trainable members; it is
// emitted at its first member's position.  Phase runs (when asked) are taken
// first, from adjacent ops.  Other ops keep their order.
std::vector<Group> fuse_groups(int n, const std::vector<HOp> &ops, bool fuse, bool phase) {
  std::vector<int> phase_of(ops.size(), -1);
  std::vector<std::vector<int>> pruns;
  if (phase) {
    for (int i = 0; i < (int)ops.size();) {
      if (!phase_member(ops[i])) {
        ++i;
        continue;
      }
      int j = i + 1;
      while (j < (int)ops.size() && j - i < kMaxPhaseMembers && phase_member(ops[j]) && same_angle(ops[i], ops[j])) ++j;
      if (j - i >= 2) {
        pruns.emplace_back();
        for (int q = i; q < j; ++q) {
          phase_of[q] = (int)pruns.size() - 1;
          pruns.back().push_back(q);
        }
      }
      i = j;
    }
  }
  std::vector<std::vector<int>> runs;
  std::vector<int> run_of(ops.size(), -1);
  if (fuse) {
    std::vector<int> open(n, -1);
    std::vector<int> gens;
    for (int i = 0; i < (int)ops.size(); ++i) {
      const HOp &h = ops[i];
      if (h.kind == SV_IDENTITY) continue;
      if (phase_of[i] < 0 && fusable(h)) {
        const int w = h.tw[0];
        const int r = open[w];
        if (r >= 0 && (int)runs[r].size() < kMaxFuseMembers && gens[r] + (h.train ? 1 : 0) <= kMaxFuseGen) {
          runs[r].push_back(i);
          gens[r] += h.train ? 1 : 0;
          run_of[i] = r;
          continue;
        }
        open[w] = (int)runs.size();
        run_of[i] = (int)runs.size();
        runs.push_back({i});
        gens.push_back(h.train ? 1 : 0);
        continue;
      }
      for (int j = 0; j < h.k; ++j) open[h.tw[j]] = -1;
      for (int c = 0; c < h.nc; ++c) open[h.cw[c]] = -1;
    }
    for (size_t r = 0; r < runs.size(); ++r) {
      bool any_pair = false;
      for (int i : runs[r]) any_pair |= !ops[i].diag;
      if (runs[r].size() < 2 || !any_pair)
        for (int i : runs[r]) run_of[i] = -1;
    }
  }
  std::vector<Group> out;
  for (int i = 0; i < (int)ops.size(); ++i) {
    if (phase_of[i] >= 0) {
      if (pruns[phase_of[i]][0] == i) out.push_back({gPhaseRun, pruns[phase_of[i]]});
      continue;
    }
    const int r = run_of[i];
    if (r < 0)
      out.push_back({gSingle, {i}});
    else if (runs[r][0] == i)
      out.push_back({gRun, runs[r]});
  }
  return out;
}

// Lower a phase run into one kPhase micro-op: member records (local-bit parity
// mask, tile-bit parity mask) in P.aux, members with local bits first.
void lower_phase(int n, const std::vector<HOp> &ops, const std::vector<int> &mem, const PassDev &pd, bool dagger,
                 int train, int slot, SlotTable &st, std::vector<OpDev> &out, std::vector<uint64_t> &aux) {
  const HOp &h0 = ops[mem[0]];
  OpDev o;
  memset(&o, 0, sizeof(o));
  o.kind = kPhase;
  o.k = 1;
  o.train = -1;
  o.slot = -1;
  o.sync_prev = 1;
  o.mat = st.add_phase(h0, (int)mem.size(), (h0.adjoint != 0) != dagger);
  std::vector<std::pair<uint32_t, uint64_t>> loc, far;
  for (int i : mem) {
    const HOp &h = ops[i];
    uint32_t lm = 0;
    uint64_t hm = 0;
    for (int j = 0; j < h.k; ++j) {
      const int b = n - 1 - h.tw[j];
      int li = -1;
      for (int q = 0; q < pd.T; ++q)
        if (pd.pos[q] == b) li = q;
      if (li >= 0)
        lm |= 1u << li;
      else
        hm |= 1ull << b;
    }
    (lm ? loc : far).push_back({lm, hm});
  }
  o.oa = (int32_t)(aux.size() / 2);
  o.ob = (int32_t)mem.size();
  o.zmask = (int32_t)loc.size();
  if (h0.train) {  // one slot: sum_j Im<lambda|G_j phi> = Im<lambda|(r - 2k) phi>
    o.train = train;
    o.slot = slot;
    o.gcode = gDiag;
  }
  for (auto *v : {&loc, &far})
    for (auto &rec : *v) {
      aux.push_back(rec.first);
      aux.push_back(rec.second);
    }
  // the local masks transposed: word b has bit j set when local member j's mask
  // has local bit b, so the parities of all members over a local index l are
  // the bits of the XOR of the words of l's set bits (padded to an even count)
  for (int b = 0; b < pd.T + (pd.T & 1); ++b) {
    uint64_t w = 0;
    for (size_t j = 0; j < loc.size() && b < pd.T; ++j)
      if (loc[j].first >> b & 1) w |= 1ull << j;
    aux.push_back(w);
  }
  out.push_back(o);
}

// Lower a fused run into one pair micro-op on its wire's local bit.
void lower_fused(int n, const std::vector<HOp> &ops, const std::vector<int> &mem, const PassDev &pd, bool dagger,
                 int train, int slot, SlotTable &st, std::vector<OpDev> &out) {
  const HOp &h0 = ops[mem[0]];
  OpDev o = blank_op(n, h0);
  o.kind = kPair;
  o.code = mGen;
  int tl = -1;
  for (int i = 0; i < pd.T; ++i)
    if (pd.pos[i] == n - 1 - h0.tw[0]) tl = i;
  o.ts[0] = o.tl[0] = (int8_t)tl;
  o.oa = 0;
  o.ob = 1 << tl;
  std::vector<const HOp *> hs;
  std::vector<SlotTable::Gen> gens;
  int ngen = 0;
  for (int i : mem) {
    hs.push_back(&ops[i]);
    SlotTable::Gen g;
    single_wire_generator(ops[i], g);
    gens.push_back(g);
    ngen += g.code != gNone;
  }
  int gmat = 0;
  o.fused = 1;
  o.mat = st.add_run(hs, gens, dagger, gmat);
  if (ngen > 0) {
    o.gcode = gHerm;
    o.ngen = (int8_t)ngen;
    o.gmat = gmat;
    o.train = train;
    o.slot = slot;
  }
  localise(o, pd);
  out.push_back(o);
}

// Greedy order-preserving fusion: gates join the current pass while the
// union of the local bits they need (non-diagonal targets) plus the lowest
// index bits fits in T bits.  The lowest bits are always local, so every tile
// is read as runs of >= 2^nlow_pref consecutive amplitudes (coalesced, and
// 16-byte aligned for the paired complex64 accesses).  Each pass is then
// lowered into micro-ops; dagger selects the adjoint sweep's U^dagger blocks.
// Consecutive uncontrolled, untrained single-wire pair micro-ops of one pass on
// distinct local bits become kMulti micro-ops of up to 3 members.
void merge_multi(std::vector<OpDev> &ops, size_t begin, int lowbits) {
  std::vector<OpDev> out(ops.begin(), ops.begin() + begin);
  std::vector<OpDev> pend;
  auto mergeable = [](const OpDev &o) {
    return o.kind == kPair && o.k == 1 && o.cmask == 0 && o.train < 0 && o.gcode == gNone;
  };
  auto emit = [&]() {
    if (pend.size() == 1) out.push_back(pend[0]);
    if (pend.size() >= 2) {
      OpDev m;
      memset(&m, 0, sizeof(m));
      m.kind = kMulti;
      m.k = (int8_t)pend.size();
      m.train = -1;
      m.slot = -1;
      m.sync_prev = 1;
      int bits[3];
      for (size_t j = 0; j < pend.size(); ++j) {
        m.tl[j] = pend[j].tl[0];
        m.mcode[j] = pend[j].code;
        m.mmat[j] = pend[j].mat;
        bits[j] = pend[j].tl[0];
      }
      std::sort(bits, bits + pend.size());
      for (size_t j = 0; j < pend.size(); ++j) m.ts[j] = (int8_t)bits[j];
      out.push_back(m);
    }
    pend.clear();
  };
  for (size_t i = begin; i < ops.size(); ++i) {
    const OpDev &o = ops[i];
    if (!mergeable(o)) {
      emit();
      out.push_back(o);
      continue;
    }
    bool clash = pend.size() >= 3;  // at most one member on the lowest bits (bank conflicts, as below)
    for (const OpDev &q : pend) clash |= q.tl[0] == o.tl[0] || (q.tl[0] < lowbits && o.tl[0] < lowbits);
    if (clash) emit();
    pend.push_back(o);
  }
  emit();
  ops.swap(out);
}

Plan plan_passes(int n, const std::vector<HOp> &ops, int Tmax, int nlow_pref, int max_train, bool dagger,
                 SlotTable &st, bool fuse = false, bool phase = false, bool multi = false) {
  Plan P;
  const std::vector<Group> groups = fuse_groups(n, ops, fuse, phase);
  const int T = std::min(Tmax, n);
  const uint64_t low = low_bits(n, T, nlow_pref);
  uint64_t cur = low;
  std::vector<int> cur_ops;
  int cur_train = 0;
  auto flush = [&]() {
    if (cur_ops.empty()) return;
    PassDev pd = make_pass(n, fill_bits(cur, n, T, nlow_pref));
    pd.op_begin = (int)P.ops.size();
    pd.train_base = P.n_train;
    int t = 0;
    bool prev_diag = false;
    for (int gi : cur_ops) {
      const std::vector<int> &grp = groups[gi].m;
      const size_t before = P.ops.size();
      if (groups[gi].kind == gPhaseRun) {
        const bool tr = ops[grp[0]].train;
        lower_phase(n, ops, grp, pd, dagger, t, tr ? P.n_train : -1, st, P.ops, P.aux);
        if (tr) {
          ++t;
          ++P.n_train;
          P.train_hop.push_back(grp[0]);
        }
      } else if (groups[gi].kind == gRun) {
        lower_fused(n, ops, grp, pd, dagger, t, P.n_train, st, P.ops);
        for (int i : grp)
          if (ops[i].train) {
            ++t;
            ++P.n_train;
            P.train_hop.push_back(i);
          }
      } else {
        const int i = grp[0];
        const HOp &h = ops[i];
        const int slot = h.train ? P.n_train : -1;
        lower_gate(n, h, pd, dagger, t, slot, st, P.ops);
        if (h.train) {
          ++t;
          ++P.n_train;
          P.train_hop.push_back(i);
        }
      }
      if (P.ops.size() > before) {
        OpDev &first = P.ops[before];
        const bool first_diag = first.kind == kDiag || first.kind == kPhase;
        if (first_diag && prev_diag) first.sync_prev = 0;  // same thread-to-amplitude map
        prev_diag = P.ops.back().kind == kDiag || P.ops.back().kind == kPhase;
      }
      for (size_t q = before; q < P.ops.size(); ++q)
        if (P.ops[q].kind == kDense) pd.max_k = std::max(pd.max_k, (int)P.ops[q].k);
    }
    if (multi) merge_multi(P.ops, (size_t)pd.op_begin, nlow_pref);
    pd.op_end = (int)P.ops.size();
    pd.n_train = t;
    P.steps.push_back({0, (int)P.passes.size()});
    P.passes.push_back(pd);
    cur_ops.clear();
    cur = low;
    cur_train = 0;
  };
  for (int gi = 0; gi < (int)groups.size(); ++gi) {
    const std::vector<int> &grp = groups[gi].m;
    if (groups[gi].kind == gPhaseRun) {  // diagonal: needs no local bits
      const int gt = ops[grp[0]].train ? 1 : 0;
      if (!cur_ops.empty() && cur_train + gt > max_train) flush();
      cur_ops.push_back(gi);
      cur_train += gt;
      continue;
    }
    if (groups[gi].kind == gRun) {
      const uint64_t need = 1ull << (n - 1 - ops[grp[0]].tw[0]);
      int gt = 0;
      for (int i : grp) gt += ops[i].train ? 1 : 0;
      const bool fits = popc(cur | need) <= T && cur_train + gt <= max_train;
      if (!cur_ops.empty() && !fits) flush();
      cur |= need;
      cur_ops.push_back(gi);
      cur_train += gt;
      continue;
    }
    const HOp &h = ops[grp[0]];
    if (h.kind == SV_IDENTITY) continue;
    if (!h.diag && h.k > kMaxTileTargets) {
      flush();
      OpDev o = blank_op(n, h);
      o.kind = kDense;
      o.mat = st.add(h, (h.adjoint != 0) != dagger, 0);
      P.steps.push_back({1, (int)P.dk_ops.size()});
      P.dk_ops.push_back(o);
      continue;
    }
    uint64_t need = 0;
    if (!h.diag)
      for (int j = 0; j < h.k; ++j) need |= 1ull << (n - 1 - h.tw[j]);
    const bool fits = popc(cur | need) <= T && cur_train + (h.train ? 1 : 0) <= max_train;
    if (!cur_ops.empty() && !fits) flush();
    cur |= need;
    cur_ops.push_back(gi);
    cur_train += h.train ? 1 : 0;
  }
  flush();
  return P;
}

// Host-side check of a plan before anything is launched: every non-diagonal
// target is a distinct local bit, pair members lie in the tile, tiles are at
// most kMaxLocalBits wide and their low run covers the 16-byte pair accesses.
sv_status check_plan(const Plan &P, int n, int nlow_pref) {
  for (const PassDev &pd : P.passes) {
    if (pd.T < 1 || pd.T > kMaxLocalBits || pd.T + pd.nhi != n)
      return fail(SV_ERR_UNSUPPORTED, "internal planner error: tile of %d bits", pd.T);
    if (pd.nlow < std::min(std::min(nlow_pref, n), pd.T))
      return fail(SV_ERR_UNSUPPORTED, "internal planner error: low run of %d bits", pd.nlow);
    if (pd.n_train > kMaxTrainPerPass) return fail(SV_ERR_UNSUPPORTED, "internal planner error: trainable ops");
    for (int o = pd.op_begin; o < pd.op_end; ++o) {
      const OpDev &op = P.ops[o];
      if (op.kind == kDiag) continue;
      if (op.kind == kPhase) {
        if (op.ob < 2 || op.ob > kMaxPhaseMembers || op.zmask < 0 || op.zmask > op.ob || op.oa < 0 ||
            2 * (size_t)(op.oa + op.ob) + pd.T > P.aux.size())
          return fail(SV_ERR_UNSUPPORTED, "internal planner error: phase run");
        continue;
      }
      if (op.k > kMaxTileTargets) return fail(SV_ERR_UNSUPPORTED, "internal planner error: wide op in a tile");
      if (op.kind == kMulti && (op.k < 2 || op.k > 3))
        return fail(SV_ERR_UNSUPPORTED, "internal planner error: multi-wire op");
      for (int j = 0; j < op.k; ++j) {
        if (op.tl[j] < 0 || op.tl[j] >= pd.T) return fail(SV_ERR_UNSUPPORTED, "internal planner error: non-local target");
        for (int q = 0; q < j; ++q)
          if (op.tl[q] == op.tl[j]) return fail(SV_ERR_UNSUPPORTED, "internal planner error: repeated target");
        if (j > 0 && op.ts[j] <= op.ts[j - 1]) return fail(SV_ERR_UNSUPPORTED, "internal planner error: target order");
      }
      if (op.kind == kPair && (op.oa < 0 || op.ob < 0 || op.oa >= (1 << pd.T) || op.ob >= (1 << pd.T) || op.oa == op.ob))
        return fail(SV_ERR_UNSUPPORTED, "internal planner error: pair members");
    }
  }
  return SV_OK;
}

// ---- Pauli terms -------------------------------------------------------------
struct HTerm {
  int obs;
  double coeff;
  uint64_t x, z;  // global index bits
  int ny;
};

uint64_t wire_mask_to_global(uint64_t wm, int n) {
  uint64_t g = 0;
  for (int w = 0; w < n; ++w)
    if (wm >> w & 1) g |= 1ull << (n - 1 - w);
  return g;
}

sv_status collect_terms(int n, const sv_pauli_sum *obs, int n_obs, std::vector<HTerm> &terms) {
  if (n_obs < 0) return fail(SV_ERR_ARG, "n_obs < 0");
  if (n_obs > 0 && !obs) return fail(SV_ERR_ARG, "observables pointer is NULL");
  const uint64_t valid = n >= 64 ? ~0ull : ((1ull << n) - 1);
  for (int o = 0; o < n_obs; ++o) {
    const sv_pauli_sum &H = obs[o];
    if (H.n_terms < 0) return fail(SV_ERR_ARG, "observable %d: n_terms < 0", o);
    if (H.n_terms > 0 && (!H.coeffs || !H.x_mask || !H.z_mask))
      return fail(SV_ERR_ARG, "observable %d: NULL term arrays", o);
    for (int t = 0; t < H.n_terms; ++t) {
      if ((H.x_mask[t] | H.z_mask[t]) & ~valid)
        return fail(SV_ERR_ARG, "observable %d term %d acts on a wire >= n = %d", o, t, n);
      if (!std::isfinite(H.coeffs[t])) return fail(SV_ERR_ARG, "observable %d term %d: coefficient not finite", o, t);
      HTerm h;
      h.obs = o;
      h.coeff = H.coeffs[t];
      h.x = wire_mask_to_global(H.x_mask[t], n);
      h.z = wire_mask_to_global(H.z_mask[t], n);
      h.ny = popc(H.x_mask[t] & H.z_mask[t]) & 3;
      terms.push_back(h);
    }
  }
  return SV_OK;
}

struct TermPlan {
  std::vector<PassDev> passes;
  std::vector<int> begin;  // terms of pass p: [begin[p], begin[p+1]) of `placed`
  std::vector<int> placed; // original term index, in pass order
};

constexpr int kMaxTermsPerPass = 512;

// Cover the terms' flip masks by passes: a term joins a pass when its X/Y wires
// fit into the pass's T local bits.  A pass starts from the lowest index bits
// (coalesced tiles) unless its first term needs them.  Words with Z letters
// only (x = 0) go to passes of their own, marked zonly, which the expectation
// kernels sum with one transform of |psi|^2 per thread and tile.
sv_status plan_terms(int n, const std::vector<HTerm> &terms, int Tmax, int nlow_pref, TermPlan &tp) {
  const int T = std::min(Tmax, n);
  std::vector<char> done(terms.size(), 0);
  size_t left = terms.size();
  tp.begin.assign(1, 0);
  {
    std::vector<int> zonly;
    for (size_t t = 0; t < terms.size(); ++t)
      if (terms[t].x == 0) zonly.push_back((int)t);
    for (size_t z0 = 0; z0 < zonly.size(); z0 += kMaxTermsPerPass) {
      const size_t z1 = std::min(zonly.size(), z0 + kMaxTermsPerPass);
      for (size_t i = z0; i < z1; ++i) {
        tp.placed.push_back(zonly[i]);
        done[zonly[i]] = 1;
        --left;
      }
      PassDev pd = make_pass(n, fill_bits(0, n, T, nlow_pref));
      pd.zonly = 1;
      tp.passes.push_back(pd);
      tp.begin.push_back((int)tp.placed.size());
    }
  }
  while (left > 0) {
    uint64_t bits = fill_bits(0, n, std::min(T, nlow_pref), nlow_pref);
    int cnt = 0;
    for (size_t t = 0; t < terms.size() && cnt < kMaxTermsPerPass; ++t) {
      if (done[t]) continue;
      const uint64_t nb = bits | terms[t].x;
      if (cnt == 0 && popc(nb) > T)
        return fail(SV_ERR_UNSUPPORTED, "a Pauli word flips %d wires; a tile has room for %d besides its low bits",
                    popc(terms[t].x), T - std::min(T, nlow_pref));
      if (popc(nb) <= T) {
        bits = nb;
        done[t] = 1;
        tp.placed.push_back((int)t);
        ++cnt;
        --left;
      }
    }
    tp.passes.push_back(make_pass(n, fill_bits(bits, n, T, nlow_pref)));
    tp.begin.push_back((int)tp.placed.size());
  }
  if (tp.passes.empty()) {  // no terms: one empty pass, as before
    tp.passes.push_back(make_pass(n, fill_bits(0, n, T, nlow_pref)));
    tp.begin.push_back(0);
  }
  return SV_OK;
}

TermDev make_termdev(const HTerm &h, const PassDev &p) {
  TermDev t;
  memset(&t, 0, sizeof(t));
  t.xg = h.x;
  t.zg = h.z;
  uint32_t xl = 0, zl = 0;
  for (int i = 0; i < p.T; ++i) {
    if (h.x >> p.pos[i] & 1) xl |= 1u << i;
    if (h.z >> p.pos[i] & 1) zl |= 1u << i;
  }
  t.xl = xl;
  t.zl = zl;
  t.ny = h.ny;
  t.obs = h.obs;
  t.coeff = h.coeff;
  return t;
}


// ---- precision dispatch ---------------------------------------------------------
struct Ops {
  decltype(&Launch<float>::build_matrices) build_matrices;
  decltype(&Launch<float>::tile_forward) tile_forward;
  decltype(&Launch<float>::tile_adjoint) tile_adjoint;
  decltype(&Launch<float>::expval_pass) expval_pass;
  decltype(&Launch<float>::expval_obs_pass) expval_obs_pass;
  decltype(&Launch<float>::lambda_pass) lambda_pass;
  decltype(&Launch<float>::dense_k) dense_k;
  decltype(&Launch<float>::set_basis) set_basis;
  decltype(&Launch<float>::copy) copy;
  decltype(&Launch<float>::stream_op) stream_op;
  decltype(&Launch<float>::tile_tangent) tile_tangent;
  int amp_bytes, Tf, Ta, nlow_pref;
  int adj_bmax, adj_cps;  // lambdas per adjoint CTA (largest variant), adjoint CTAs per SM
};

const Ops &ops_df() {
  static const Ops d = {Launch<df>::build_matrices, Launch<df>::tile_forward, Launch<df>::tile_adjoint,
                        Launch<df>::expval_pass,    Launch<df>::expval_obs_pass, Launch<df>::lambda_pass,
                        Launch<df>::dense_k,
                        Launch<df>::set_basis,      Launch<df>::copy,
                        Launch<df>::stream_op, Launch<df>::tile_tangent,
                        16, Launch<df>::max_T_forward(), Launch<df>::max_T_adjoint(), 3,
                        Launch<df>::adj_lambdas_max(), Launch<df>::adj_ctas_per_sm()};
  return d;
}

const Ops &ops_for(sv_dtype dt) {
  static const Ops f32 = {Launch<float>::build_matrices, Launch<float>::tile_forward,
                          Launch<float>::tile_adjoint,   Launch<float>::expval_pass,
                          Launch<float>::expval_obs_pass, Launch<float>::lambda_pass, Launch<float>::dense_k,
                          Launch<float>::set_basis,      Launch<float>::copy,
                          Launch<float>::stream_op, Launch<float>::tile_tangent,
                          8, Launch<float>::max_T_forward(), Launch<float>::max_T_adjoint(), 4,
                          Launch<float>::adj_lambdas_max(), Launch<float>::adj_ctas_per_sm()};
  static const Ops f64 = {Launch<double>::build_matrices, Launch<double>::tile_forward,
                          Launch<double>::tile_adjoint,   Launch<double>::expval_pass,
                          Launch<double>::expval_obs_pass, Launch<double>::lambda_pass, Launch<double>::dense_k,
                          Launch<double>::set_basis,      Launch<double>::copy,
                          Launch<double>::stream_op, Launch<double>::tile_tangent,
                          16, Launch<double>::max_T_forward(), Launch<double>::max_T_adjoint(), 3,
                          Launch<double>::adj_lambdas_max(), Launch<double>::adj_ctas_per_sm()};
  return dt == SV_C64 ? f32 : f64;
}


}  // namespace

// ---- state -----------------------------------------------------------------------
struct sv_state {
  int n = 0;
  sv_dtype dt = SV_C128;
  void *psi = nullptr;
  bool owns = false;
  size_t bytes = 0;  // bytes of one vector
  cudaStream_t stream = nullptr;
  void *ws = nullptr;        // library-owned workspace arena
  size_t ws_bytes = 0;
  void *user_ws = nullptr;   // caller-provided workspace
  size_t user_ws_bytes = 0;
  void *tab = nullptr;       // table arena for one-shot programs
  size_t tab_bytes = 0;
  int latched = 0;
  int compute = SV_COMPUTE_NATIVE;
  int renorm = 0;            // renormalise after circuit forward passes
  double *d_norm = nullptr;  // kNormBlocks FP64 partials
};

namespace {
const Ops &ops_of(const sv_state *s) {
  return (s->dt == SV_C128 && s->compute == SV_COMPUTE_DOUBLE_FLOAT) ? ops_df() : ops_for(s->dt);
}
}  // namespace

namespace {

sv_status check_state(const sv_state *s) {
  if (!s) return fail(SV_ERR_ARG, "state is NULL");
  if (s->latched) return fail(SV_ERR_STATE, "an earlier device error is latched on this state; call sv_reset");
  return SV_OK;
}

sv_status after_launch(sv_state *s, cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    s->latched = 1;
    return cuda_fail(e, what);
  }
  return SV_OK;
}

// Workspace: the caller's buffer when big enough, else a grow-only library arena.
sv_status get_workspace(sv_state *s, size_t bytes, char **out) {
  if (s->user_ws && s->user_ws_bytes >= bytes) {
    *out = (char *)s->user_ws;
    return SV_OK;
  }
  if (s->ws_bytes < bytes) {
    if (s->ws) {
      cudaStreamSynchronize(s->stream);
      dev_free(s->ws, s->ws_bytes);
      s->ws = nullptr;
      s->ws_bytes = 0;
    }
    sv_status st = dev_alloc(&s->ws, bytes);
    if (st) return st;
    s->ws_bytes = bytes;
  }
  *out = (char *)s->ws;
  return SV_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// ---- program ----------------------------------------------------------------------
struct sv_program {
  sv_state *s = nullptr;
  int n_params = 0, m = 0;
  bool owns_tables = true;
  void *tables = nullptr;
  size_t tables_bytes = 0;
  Plan fwd, adj;
  TermPlan tp;
  std::vector<HTerm> terms;
  std::vector<double> coef;   // per trainable slot: scale * (-2 s_eff)
  int n_slots = 0;
  size_t mats_entries = 0;
  // device pointers into `tables`
  OpDev *d_fwd_ops = nullptr, *d_adj_ops = nullptr, *d_tan_ops = nullptr;
  uint64_t *d_aux = nullptr;      // phase-run member records of the forward plan
  uint64_t *d_adj_aux = nullptr;  // ... of the adjoint plan
  MatSlot *d_slots = nullptr;
  void *d_mats = nullptr;
  double *d_params = nullptr, *d_user = nullptr;
  TermDev *d_terms = nullptr;
  int32_t *d_obs_begin = nullptr, *d_term_order = nullptr;
  TermDev *d_lam_terms = nullptr;
  int32_t *d_lam_begin = nullptr;
  double *d_coef = nullptr;
  int32_t *d_pbegin = nullptr, *d_pslots = nullptr;
  // lambda chunking
  int mc = 0, n_chunks = 0;
  std::vector<int> lam_begin_off;  // per (chunk, pass): offset into d_lam_begin
  // VJP: every placed term with obs 0, coefficient c_t * g_obs(t) set per call
  std::vector<TermDev> vjp_host;
  TermDev *d_vjp_terms = nullptr;
  int32_t *d_vjp_begin = nullptr;
  // grids
  int grid_f = 1, grid_e = 1;
  int ctas_a = 1, ctas_l = 1;        // CTAs per adjoint / lambda launch (split over lambdas)
  uint64_t tiles_a = 1, tiles_l = 1; // tiles per vector in those passes
  int lam_per_cta = 1;               // lambdas sharing one phi tile in the adjoint kernel
  int cfg_compute = -1;              // compute mode the adjoint launch shape was made for
  bool want_lam = false;             // workspace holds lambda vectors without a sweep (variance)
  bool want_tan = false;             // workspace holds the tangent vector and coefficients (JVP)
  Plan tan;                          // forward plan of the expanded tape with trainable micro-ops (JVP)
  std::vector<int> tan_pidx;         // tangent slot -> parameter
  std::vector<double> tan_factor;    // tangent slot -> s_eff * scale (coefficient i * factor * tangent[p])
  int groups_a(int mcc) const { return (mcc + lam_per_cta - 1) / lam_per_cta; }
  int grid_a(int mcc) const {
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles_a, ctas_a / std::max(1, groups_a(mcc))));
  }
  int grid_l(int mcc) const { return (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles_l, ctas_l / std::max(1, mcc))); }
  int launches = 0;
  bool params_set = false;  // gate matrices built at least once
  int mats_compute = SV_COMPUTE_NATIVE;
};

namespace {

void destroy_program(sv_program *p) {
  if (!p) return;
  if (p->owns_tables && p->tables) dev_free(p->tables, p->tables_bytes);
  delete p;
}

int blocks_per_sm(int smem_bytes) {
  const int by_threads = 2048 / kBlock;
  const int by_smem = (228 * 1024) / (smem_bytes + 1024);
  return std::max(1, std::min(by_threads, by_smem));
}

// Adjoint launch shape for the state's current compute mode: lambdas per CTA
// (a compiled power of two that fits the shared-memory budget) and CTAs.
void adj_config(sv_program *p, const Ops &K, int n) {
  const int ta = std::min(K.Ta, n);
  const int tile_b = K.amp_bytes << ta;
  const int budget = (224 / K.adj_cps) * 1024 - tile_b - (8 << ta);
  const int lpc = std::max(1, std::min({K.adj_bmax, std::max(1, p->mc),
                                        budget / (tile_b + kMaxTrainPerPass * 8 * (kBlock / 32))}));
  int b = 1;
  while (2 * b <= lpc) b *= 2;
  p->lam_per_cta = b;
  const int smem_a = tile_b * (1 + b) + (8 << ta) + kMaxTrainPerPass * 8 * (kBlock / 32) * b;
  const int cps = b <= 2 ? 2 : K.adj_cps;  // few lambdas per CTA: registers allow two CTAs per SM
  p->ctas_a = 2 * sm_count() * std::min(cps, blocks_per_sm(smem_a));
  p->tiles_a = 1ull << (n - ta);
  p->cfg_compute = p->s->compute;
}

void sync_adj_config(sv_program *p) {
  if (p->cfg_compute != p->s->compute) adj_config(p, ops_of(p->s), p->s->n);
}

sv_status build_program(sv_state *s, const sv_tape *tape, const sv_pauli_sum *obs, int n_obs,
                        const double *host_params, bool one_shot, sv_program **out) {
  *out = nullptr;
  const int n = s->n;
  const Ops &K = ops_of(s);
  int n_ops = 0, n_params = 0;
  const sv_op *ops = nullptr;
  const double *umats = nullptr;
  int64_t n_umat = 0;
  if (tape) {
    if (tape->n_ops < 0 || tape->n_params < 0) return fail(SV_ERR_ARG, "negative tape sizes");
    if (tape->n_ops > 0 && !tape->ops) return fail(SV_ERR_ARG, "tape ops pointer is NULL");
    n_ops = tape->n_ops;
    n_params = tape->n_params;
    ops = tape->ops;
    umats = tape->matrices;
    n_umat = tape->n_matrix_entries;
  }
  for (int i = 0; i < n_ops; ++i) {
    sv_status st = validate_op(n, ops[i], n_params, umats, n_umat, host_params, host_params != nullptr);
    if (st) {
      g_err = "op " + std::to_string(i) + ": " + g_err;
      return st;
    }
  }
  std::vector<HTerm> terms;
  if (sv_status st = collect_terms(n, obs, n_obs, terms)) return st;

  sv_program *p = new sv_program();
  p->s = s;
  p->n_params = n_params;
  p->m = n_obs;
  p->owns_tables = !one_shot;
  p->terms = terms;

  // host ops, fused passes lowered to micro-ops, and their matrix slots
  std::vector<HOp> fops, aops;
  for (int i = 0; i < n_ops; ++i) {
    HOp h = to_hop(ops[i], umats);
    fops.push_back(h);
    expand_op(h, aops);
  }
  SlotTable st_tab;
  p->fwd = plan_passes(n, fops, K.Tf, K.nlow_pref, 1 << 30, false, st_tab, true, true, true);
  p->adj = plan_passes(n, aops, K.Ta, K.nlow_pref, kMaxTrainPerPass, true, st_tab, true, true);
  if (sv_status st = check_plan(p->fwd, n, K.nlow_pref)) {
    destroy_program(p);
    return st;
  }
  if (sv_status st = check_plan(p->adj, n, K.nlow_pref)) {
    destroy_program(p);
    return st;
  }
  if (n_params > 0) {
    p->tan = plan_passes(n, aops, K.Tf, K.nlow_pref, kMaxTrainPerPass, false, st_tab, false, false);
    if (sv_status st = check_plan(p->tan, n, K.nlow_pref)) {
      destroy_program(p);
      return st;
    }
    for (int sidx = 0; sidx < p->tan.n_train; ++sidx) {
      const HOp &e = aops[p->tan.train_hop[sidx]];
      p->tan_pidx.push_back(e.pidx[0]);
      p->tan_factor.push_back((e.adjoint ? -kind_gen_s(e.kind) : kind_gen_s(e.kind)) * e.scale);
    }
  }
  std::vector<MatSlot> &slots = st_tab.slots;
  const size_t off = st_tab.entries;
  p->n_slots = (int)slots.size();
  p->mats_entries = off;

  // trainable slots (sweep order) -> coefficient scale * (-2 s_eff) and parameter CSR
  std::vector<int> slot_param(p->adj.n_train);
  p->coef.assign(p->adj.n_train, 0.0);
  for (int sidx = 0; sidx < p->adj.n_train; ++sidx) {
    const HOp &e = aops[p->adj.train_hop[sidx]];
    const double s_eff = e.adjoint ? -kind_gen_s(e.kind) : kind_gen_s(e.kind);
    p->coef[sidx] = e.scale * (-2.0 * s_eff);
    slot_param[sidx] = e.pidx[0];
  }
  std::vector<int32_t> pbegin(n_params + 1, 0), pslots;
  for (int sidx = 0; sidx < (int)slot_param.size(); ++sidx) pbegin[slot_param[sidx] + 1]++;
  for (int q = 0; q < n_params; ++q) pbegin[q + 1] += pbegin[q];
  pslots.resize(slot_param.size());
  {
    std::vector<int32_t> fillp(pbegin.begin(), pbegin.end() - 1);
    for (int sidx = 0; sidx < (int)slot_param.size(); ++sidx) pslots[fillp[slot_param[sidx]]++] = sidx;
  }

  // observables: passes covering the terms
  std::vector<TermDev> tdev;
  std::vector<int32_t> obs_begin(n_obs + 1, 0), term_order;
  if (n_obs > 0) {
    if (sv_status st = plan_terms(n, terms, K.Tf, K.nlow_pref, p->tp)) {
      destroy_program(p);
      return st;
    }
    std::vector<int> dev_index(terms.size());
    for (size_t pi = 0; pi + 1 < p->tp.begin.size(); ++pi)
      for (int q = p->tp.begin[pi]; q < p->tp.begin[pi + 1]; ++q) {
        const int t = p->tp.placed[q];
        dev_index[t] = (int)tdev.size();
        tdev.push_back(make_termdev(terms[t], p->tp.passes[pi]));
      }
    for (size_t t = 0; t < terms.size(); ++t) obs_begin[terms[t].obs + 1]++;
    for (int o = 0; o < n_obs; ++o) obs_begin[o + 1] += obs_begin[o];
    term_order.resize(terms.size());
    std::vector<int32_t> fillo(obs_begin.begin(), obs_begin.end() - 1);
    for (size_t t = 0; t < terms.size(); ++t) term_order[fillo[terms[t].obs]++] = dev_index[t];
  }

  // lambda chunk size from free device memory
  const size_t V = s->bytes;
  int mc = n_obs;
  if (n_obs > 0) {
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) {
      cudaGetLastError();
      freeb = 0;
    }
    size_t have = s->ws_bytes + (size_t)(0.85 * (double)freeb);
    const size_t fixed = 2 * V + ((size_t)64 << 20);
    size_t cap = have > fixed ? (have - fixed) / V : 1;
    if (const char *env = getenv("SV_LAMBDA_CHUNK")) cap = std::max(1, atoi(env));
    mc = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_obs, cap));
  }
  p->mc = mc;
  p->n_chunks = n_obs > 0 ? (n_obs + mc - 1) / mc : 0;

  // lambda term tables per (chunk, pass): terms of each observable in the chunk
  std::vector<TermDev> ltdev;
  std::vector<int32_t> lbegin;
  const int npass_e = (int)p->tp.passes.size();
  for (int c = 0; c < p->n_chunks; ++c) {
    const int j0 = c * mc, j1 = std::min(n_obs, j0 + mc);
    for (int pi = 0; pi < npass_e; ++pi) {
      p->lam_begin_off.push_back((int)lbegin.size());
      for (int o = j0; o < j1; ++o) {
        lbegin.push_back((int)ltdev.size());
        for (int q = p->tp.begin[pi]; q < p->tp.begin[pi + 1]; ++q) {
          const int t = p->tp.placed[q];
          if (terms[t].obs == o) ltdev.push_back(make_termdev(terms[t], p->tp.passes[pi]));
        }
      }
      lbegin.push_back((int)ltdev.size());
    }
  }

  // VJP tables: pass q holds placed terms [tp.begin[q], tp.begin[q+1]) as observable 0
  std::vector<int32_t> vbegin;
  for (int q = 0; q < npass_e; ++q) {
    for (int i = p->tp.begin[q]; i < p->tp.begin[q + 1]; ++i) {
      TermDev t = make_termdev(terms[p->tp.placed[i]], p->tp.passes[q]);
      t.obs = 0;
      p->vjp_host.push_back(t);
    }
    vbegin.push_back(p->tp.begin[q]);
    vbegin.push_back(p->tp.begin[q + 1]);
  }

  // grids
  const int sms = sm_count();
  {
    int tmax = std::min(K.Tf, n);
    p->grid_f = std::max(1, std::min((int)std::min<uint64_t>(1ull << (n - tmax), 1 << 30),
                                     2 * sms * blocks_per_sm((K.amp_bytes << tmax) + 4096)));
    adj_config(p, K, n);
    p->grid_e = std::max(1, std::min((int)std::min<uint64_t>(1ull << (n - tmax), 1 << 30),
                                     sms * blocks_per_sm((K.amp_bytes << tmax) + 4096 + 32768)));
    p->ctas_l = 2 * sms * blocks_per_sm((K.amp_bytes << tmax) + 4096);
    p->tiles_l = 1ull << (n - tmax);
  }

  // one device allocation for every table
  auto sz = [](size_t count, size_t elem) { return align256(count * elem); };
  const size_t umat_doubles = umats ? (size_t)2 * (size_t)n_umat : 0;
  size_t total = sz(p->fwd.ops.size(), sizeof(OpDev)) + sz(p->adj.ops.size(), sizeof(OpDev)) +
                 sz(p->tan.ops.size(), sizeof(OpDev)) +
                 sz(slots.size(), sizeof(MatSlot)) + sz(off, K.amp_bytes) + sz(std::max(n_params, 1), 8) +
                 sz(umat_doubles, 8) + sz(tdev.size(), sizeof(TermDev)) + sz(obs_begin.size(), 4) +
                 sz(term_order.size(), 4) + sz(ltdev.size(), sizeof(TermDev)) + sz(lbegin.size(), 4) +
                 sz(p->coef.size(), 8) + sz(pbegin.size(), 4) + sz(pslots.size(), 4) +
                 sz(p->vjp_host.size(), sizeof(TermDev)) + sz(vbegin.size(), 4) + sz(p->fwd.aux.size(), 8) +
                 sz(p->adj.aux.size(), 8);
  total = std::max<size_t>(total, 256);
  if (one_shot) {
    if (s->tab_bytes < total) {
      if (s->tab) {
        cudaStreamSynchronize(s->stream);
        dev_free(s->tab, s->tab_bytes);
        s->tab = nullptr;
        s->tab_bytes = 0;
      }
      if (sv_status st = dev_alloc(&s->tab, total)) {
        destroy_program(p);
        return st;
      }
      s->tab_bytes = total;
    }
    p->tables = s->tab;
  } else {
    if (sv_status st = dev_alloc(&p->tables, total)) {
      destroy_program(p);
      return st;
    }
  }
  p->tables_bytes = total;
  std::vector<char> host(total, 0);
  size_t cursor = 0;
  auto put = [&](const void *src, size_t count, size_t elem) -> char * {
    char *dptr = (char *)p->tables + cursor;
    if (count) memcpy(host.data() + cursor, src, count * elem);
    cursor += align256(count * elem);
    return dptr;
  };
  p->d_fwd_ops = (OpDev *)put(p->fwd.ops.data(), p->fwd.ops.size(), sizeof(OpDev));
  p->d_aux = (uint64_t *)put(p->fwd.aux.data(), p->fwd.aux.size(), 8);
  p->d_adj_aux = (uint64_t *)put(p->adj.aux.data(), p->adj.aux.size(), 8);
  p->d_tan_ops = (OpDev *)put(p->tan.ops.data(), p->tan.ops.size(), sizeof(OpDev));
  p->d_adj_ops = (OpDev *)put(p->adj.ops.data(), p->adj.ops.size(), sizeof(OpDev));
  p->d_slots = (MatSlot *)put(slots.data(), slots.size(), sizeof(MatSlot));
  p->d_mats = put(nullptr, 0, 1);
  cursor += align256(off * K.amp_bytes);
  p->d_params = (double *)put(nullptr, 0, 1);
  cursor += align256(std::max(n_params, 1) * 8);
  p->d_user = (double *)put(umats, umat_doubles, 8);
  p->d_terms = (TermDev *)put(tdev.data(), tdev.size(), sizeof(TermDev));
  p->d_obs_begin = (int32_t *)put(obs_begin.data(), obs_begin.size(), 4);
  p->d_term_order = (int32_t *)put(term_order.data(), term_order.size(), 4);
  p->d_lam_terms = (TermDev *)put(ltdev.data(), ltdev.size(), sizeof(TermDev));
  p->d_lam_begin = (int32_t *)put(lbegin.data(), lbegin.size(), 4);
  p->d_coef = (double *)put(p->coef.data(), p->coef.size(), 8);
  p->d_pbegin = (int32_t *)put(pbegin.data(), pbegin.size(), 4);
  p->d_pslots = (int32_t *)put(pslots.data(), pslots.size(), 4);
  p->d_vjp_terms = (TermDev *)put(p->vjp_host.data(), p->vjp_host.size(), sizeof(TermDev));
  p->d_vjp_begin = (int32_t *)put(vbegin.data(), vbegin.size(), 4);
  cudaError_t e = cudaMemcpyAsync(p->tables, host.data(), total, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess && one_shot) e = cudaStreamSynchronize(s->stream);  // host staging freed on return
  if (e != cudaSuccess) {
    destroy_program(p);
    return cuda_fail(e, "uploading program tables");
  }
  if (!one_shot) {
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
      destroy_program(p);
      return cuda_fail(e, "uploading program tables");
    }
  }
  *out = p;
  return SV_OK;
}

sv_status program_set_params(sv_program *p, const double *params, int on_device) {
  sv_state *s = p->s;
  const Ops &K = ops_of(s);
  if (p->n_params > 0) {
    if (!params) return fail(SV_ERR_ARG, "params is NULL but the tape has %d parameters", p->n_params);
    if (!on_device)
      for (int i = 0; i < p->n_params; ++i)
        if (!std::isfinite(params[i])) return fail(SV_ERR_ARG, "parameter %d is not finite", i);
    cudaError_t e = cudaMemcpyAsync(p->d_params, params, (size_t)p->n_params * 8,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copying parameters");
  }
  p->launches = 0;
  sv_status st;
  {
    LaunchTimer t(s->stream, 5);
    st = after_launch(s, K.build_matrices(p->d_slots, p->n_slots, p->d_params, p->d_user, p->d_mats, s->stream),
                      "build_matrices");
  }
  p->launches += p->n_slots > 0;
  if (!st) {
    p->params_set = true;
    p->mats_compute = s->compute;
  }
  return st;
}

// Gate matrices are stored in the compute type: rebuild them if the state's
// arithmetic mode changed since the parameters were set.
sv_status ensure_mats(sv_program *p) {
  sv_state *s = p->s;
  sync_adj_config(p);
  if (!p->params_set || p->mats_compute == s->compute || p->n_slots == 0) return SV_OK;
  LaunchTimer t(s->stream, 5);
  sv_status st = after_launch(s, ops_of(s).build_matrices(p->d_slots, p->n_slots, p->d_params, p->d_user, p->d_mats,
                                                           s->stream),
                              "build_matrices");
  if (!st) p->mats_compute = s->compute;
  return st;
}

sv_status require_params(const sv_program *p) {
  if (p->n_slots > 0 && !p->params_set)
    return fail(SV_ERR_STATE, "program parameters were never set (call sv_program_set_params first)");
  return SV_OK;
}

// A pass of one pair op, or one diagonal op on <= 2 targets, runs as a stream
// over the amplitudes it touches (no tile, no shared memory).
bool make_stream(int n, const PassDev &pd, const OpDev &o, bool c64, StreamDev &sd) {
  memset(&sd, 0, sizeof(sd));
  if (o.kind == kDense || o.kind == kPhase || o.kind == kMulti || (o.kind == kDiag && o.k > 2)) return false;
  uint64_t fixed = o.cmask, val = o.cval;
  if (o.kind == kPair) {
    for (int j = 0; j < o.k; ++j) fixed |= 1ull << o.tg[j];
    for (int i = 0; i < pd.T; ++i) {
      if ((o.oa >> i) & 1) sd.oa |= 1ull << pd.pos[i];
      if ((o.ob >> i) & 1) sd.ob |= 1ull << pd.pos[i];
    }
  } else {
    sd.tg0 = o.tg[0];
    sd.tg1 = o.k > 1 ? o.tg[1] : 0;
    if (o.code == dNeg)
      for (int j = 0; j < o.k; ++j) {
        fixed |= 1ull << o.tg[j];
        val |= 1ull << o.tg[j];
      }
  }
  if (popc(fixed) > 16 || popc(fixed) > n) return false;
  for (int b = 0; b < n; ++b)
    if ((fixed >> b) & 1) sd.fix[sd.nfix++] = (int8_t)b;
  sd.kind = o.kind;
  sd.code = o.code;
  sd.k = o.k;
  sd.fixval = val;
  sd.mat = o.mat;
  sd.vec2 = c64 && !(fixed & 1) && n - sd.nfix >= 1;
  sd.pair16 = c64 && o.kind == kPair && sd.oa == 0 && sd.ob == 1;
  return true;
}

// End of a circuit's forward pass: psi <- psi / ||psi|| when the state asks for it.
sv_status finish_forward(sv_state *s) {
  if (!s->renorm) return SV_OK;
  if (!s->d_norm)
    if (sv_status st = dev_alloc((void **)&s->d_norm, kNormBlocks * sizeof(double))) return st;
  const cudaError_t e = s->dt == SV_C64 ? Launch<float>::renormalize(s->psi, s->n, s->d_norm, s->stream)
                                        : Launch<double>::renormalize(s->psi, s->n, s->d_norm, s->stream);
  return after_launch(s, e, "renormalize");
}

sv_status run_steps_forward(sv_program *p, void *psi) {
  sv_state *s = p->s;
  if (sv_status r = ensure_mats(p)) return r;
  const Ops &K = ops_of(s);
  for (const Step &st : p->fwd.steps) {
    cudaError_t e;
    if (st.dense_k) {
      LaunchTimer t(s->stream, 6);
      e = K.dense_k(psi, s->n, p->fwd.dk_ops[st.index], p->d_mats, 0, s->stream);
    } else {
      LaunchTimer t(s->stream, 0);
      const PassDev &pd = p->fwd.passes[st.index];
      StreamDev sd;
      if (pd.op_end - pd.op_begin == 1 &&
          make_stream(s->n, pd, p->fwd.ops[pd.op_begin], s->dt == SV_C64, sd))
        e = K.stream_op(psi, s->n, sd, p->d_mats, s->stream);
      else
        e = K.tile_forward(psi, s->n, pd, p->d_fwd_ops, p->d_mats, p->d_aux, p->grid_f, s->stream);
    }
    if (sv_status r = after_launch(s, e, "forward pass")) return r;
    ++p->launches;
  }
  return SV_OK;
}

// Workspace layout of a Jacobian call.
struct JacWs {
  char *phiA, *phiB, *lam;
  double *partials, *contrib, *term_sums, *expvals, *J;
  double2 *tan_coefs;  // JVP: complex coefficient per tangent slot
};

// Expectation values by observable (one register sum of H_o psi per amplitude,
// one reduction per observable and tile) instead of by word: complex128 (FP64
// or double-float), all observables in one lambda chunk (its term tables), at
// least four words per observable on average, at most 64 observables.
bool expval_by_observable(const sv_program *p) {
  if (!(p->s->dt == SV_C128 && p->m > 0 && p->m <= 64 && p->n_chunks == 1 && p->terms.size() >= 4 * (size_t)p->m))
    return false;
  for (const PassDev &pd : p->tp.passes)  // Z-only words are summed faster word by word
    if (!pd.zonly) return true;
  return false;
}

// Rows of the term-sum buffer: one per word, or one per (pass, observable).
size_t term_sum_rows(const sv_program *p) {
  size_t rows = std::max<size_t>(1, p->terms.size());
  if (expval_by_observable(p)) rows = std::max(rows, p->tp.passes.size() * (size_t)p->m);
  return rows;
}

sv_status jac_workspace(sv_program *p, JacWs &w) {
  sv_state *s = p->s;
  sync_adj_config(p);
  const size_t V = s->bytes;
  size_t max_train = 1;
  for (const PassDev &pd : p->adj.passes) max_train = std::max<size_t>(max_train, pd.n_train);
  size_t max_terms = 1;
  for (size_t q = 0; q + 1 < p->tp.begin.size(); ++q)
    max_terms = std::max<size_t>(max_terms, p->tp.begin[q + 1] - p->tp.begin[q]);
  size_t lam_rows = 1;
  for (int mcc : {p->mc, p->m % std::max(1, p->mc), 1})
    if (mcc > 0) lam_rows = std::max(lam_rows, (size_t)p->grid_a(mcc) * mcc);
  size_t part = std::max(lam_rows * max_train, (size_t)p->grid_e * std::max<size_t>(max_terms, p->m));
  if (p->want_lam) part = std::max(part, (size_t)p->mc * kNormBlocks);
  part = std::max(part, (size_t)std::min(std::max(p->m, 1), 64) * kNormBlocks);  // expvals from lambdas
  if (p->want_tan) part = std::max(part, (size_t)p->mc * kNormBlocks);
  const bool need_vec = p->adj.n_train > 0 || !p->adj.dk_ops.empty() || p->want_tan;  // phi buffers / dpsi
  const bool need_lam = need_vec || p->want_lam;
  const size_t tan_bytes = p->want_tan ? align256((size_t)std::max(1, p->tan.n_train) * 16) : 0;
  const size_t bytes = tan_bytes + (need_vec ? 2 * V : 0) + (need_lam ? (size_t)p->mc * V : 0) + align256(part * 8) +
                       align256((size_t)std::max(1, p->adj.n_train) * std::max(1, p->m) * 8) +
                       align256(term_sum_rows(p) * 8) + align256((size_t)std::max(1, p->m) * 8) +
                       align256((size_t)std::max(1, p->m) * std::max(1, p->n_params) * 8);
  char *base = nullptr;
  if (sv_status st = get_workspace(s, bytes, &base)) return st;
  size_t c = 0;
  w.tan_coefs = (double2 *)(base + c);
  c += tan_bytes;
  w.phiA = base + c;
  c += need_vec ? V : 0;
  w.phiB = base + c;
  c += need_vec ? V : 0;
  w.lam = base + c;
  c += need_lam ? (size_t)p->mc * V : 0;
  w.partials = (double *)(base + c);
  c += align256(part * 8);
  w.contrib = (double *)(base + c);
  c += align256((size_t)std::max(1, p->adj.n_train) * std::max(1, p->m) * 8);
  w.term_sums = (double *)(base + c);
  c += align256(term_sum_rows(p) * 8);
  w.expvals = (double *)(base + c);
  c += align256((size_t)std::max(1, p->m) * 8);
  w.J = (double *)(base + c);
  return SV_OK;
}

sv_status run_expval(sv_program *p, const void *psi, const JacWs &w) {
  sv_state *s = p->s;
  const Ops &K = ops_of(s);
  if (expval_by_observable(p)) {
    // per pass q: term_sums[q * m + o] = sum over CTAs; then expvals[o] = sum over q (fixed orders)
    const int npass = (int)p->tp.passes.size();
    for (int q = 0; q < npass; ++q) {
      const int32_t *begin = (const int32_t *)p->d_lam_begin + p->lam_begin_off[q];
      cudaError_t e;
      {
        LaunchTimer t(s->stream, 2);
        e = K.expval_obs_pass(psi, s->n, p->tp.passes[q], p->d_lam_terms, begin, p->m, w.partials, p->grid_e,
                              s->stream);
      }
      if (sv_status r = after_launch(s, e, "expval pass")) return r;
      {
        LaunchTimer t(s->stream, 4);
        e = reduce_partials(w.partials, p->grid_e, p->m, 1, w.term_sums, p->m, q, 0, s->stream);
      }
      if (sv_status r = after_launch(s, e, "expval reduce")) return r;
      p->launches += 2;
    }
    cudaError_t e;
    {
      LaunchTimer t(s->stream, 4);
      e = reduce_partials(w.term_sums, npass, p->m, 1, w.expvals, 1, 0, 0, s->stream);
    }
    p->launches += 1;
    return after_launch(s, e, "expval combine");
  }
  for (size_t q = 0; q + 1 < p->tp.begin.size(); ++q) {
    const int b = p->tp.begin[q], cnt = p->tp.begin[q + 1] - b;
    if (cnt == 0) continue;
    cudaError_t e;
    {
      LaunchTimer t(s->stream, 2);
      e = K.expval_pass(psi, s->n, p->tp.passes[q], p->d_terms + b, cnt, w.partials, p->grid_e, s->stream);
    }
    if (sv_status r = after_launch(s, e, "expval pass")) return r;
    {
      LaunchTimer t(s->stream, 4);
      e = reduce_partials(w.partials, p->grid_e, 1, cnt, w.term_sums, 1, b, 0, s->stream);
    }
    if (sv_status r = after_launch(s, e, "expval reduce")) return r;
    p->launches += 2;
  }
  cudaError_t e;
  {
    LaunchTimer t(s->stream, 4);
    e = combine_terms(w.term_sums, p->d_terms, p->d_obs_begin, p->m, p->d_term_order, w.expvals, s->stream);
  }
  p->launches += p->m > 0;
  return after_launch(s, e, "combine terms");
}

// One backward sweep (lambda initialisation and reverse passes) for mcc lambdas, written into contrib columns
// [j0, j0 + mcc) (leading dimension ldc).  lam_begin(q) gives the per-observable
// term ranges of expectation pass q in lam_terms.
template <typename BeginFn>
sv_status run_sweep(sv_program *p, const JacWs &w, int mcc, int j0, int ldc, const TermDev *lam_terms,
                    BeginFn lam_begin, bool lam_ready = false) {
  sv_state *s = p->s;
  const Ops &K = ops_of(s);
  const int n = s->n;
  const size_t V = s->bytes;
  const int npass_e = lam_ready ? 0 : (int)p->tp.passes.size();  // lam_ready: lambdas already in w.lam
  for (int q = 0; q < npass_e; ++q) {
    cudaError_t e;
    {
      LaunchTimer t(s->stream, 3);
      e = K.lambda_pass(s->psi, w.lam, n, p->tp.passes[q], lam_terms, lam_begin(q), mcc, q == 0, p->grid_l(mcc),
                        s->stream);
    }
    if (sv_status r = after_launch(s, e, "lambda pass")) return r;
    ++p->launches;
  }
  // phi starts as psi (read only); with one lambda group later passes update phi in place.
  const void *phi_in = s->psi;
  char *phi_out = w.phiA;
  const bool in_place = p->groups_a(mcc) == 1;
  auto advance = [&]() {
    phi_in = phi_out;
    if (!in_place) phi_out = (phi_out == w.phiA) ? w.phiB : w.phiA;
  };
  for (int si = (int)p->adj.steps.size() - 1; si >= 0; --si) {
    const Step &st = p->adj.steps[si];
    if (st.dense_k) {
      if (phi_in == s->psi) {
        if (sv_status r = after_launch(s, K.copy(phi_out, s->psi, n, s->stream), "copy phi")) return r;
        advance();
      }
      const OpDev &op = p->adj.dk_ops[st.index];
      LaunchTimer t(s->stream, 6);
      // the adjoint plan's slot already holds U^dagger: apply it as stored
      cudaError_t e = K.dense_k((void *)phi_in, n, op, p->d_mats, 0, s->stream);
      for (int j = 0; j < mcc && e == cudaSuccess; ++j) e = K.dense_k(w.lam + (size_t)j * V, n, op, p->d_mats, 0, s->stream);
      if (sv_status r = after_launch(s, e, "dense_k adjoint")) return r;
      p->launches += 1 + mcc;
      continue;
    }
    const PassDev &pd = p->adj.passes[st.index];
    const int nb = p->grid_a(mcc);
    cudaError_t e;
    {
      LaunchTimer t(s->stream, 1);
      e = K.tile_adjoint(phi_in, phi_out, w.lam, n, mcc, p->lam_per_cta, pd, p->d_adj_ops, p->d_mats, p->d_adj_aux,
                         w.partials, nb, s->stream);
    }
    if (sv_status r = after_launch(s, e, "adjoint pass")) return r;
    ++p->launches;
    if (pd.n_train > 0) {
      LaunchTimer t(s->stream, 4);
      e = reduce_partials(w.partials, nb, mcc, pd.n_train, w.contrib, ldc, pd.train_base, j0, s->stream);
      if (sv_status r = after_launch(s, e, "adjoint reduce")) return r;
      ++p->launches;
    }
    advance();
  }
  return SV_OK;
}

bool needs_sweep(const sv_program *p) { return p->adj.n_train > 0 || !p->adj.dk_ops.empty(); }

// Expectation values from lambda_j = H_j psi already in w.lam: E_j = Re <psi|lambda_j>
// (fixed-order partials), instead of a second application of the words.
sv_status expvals_from_lambdas(sv_program *p, const JacWs &w) {
  sv_state *s = p->s;
  for (int j = 0; j < p->m; ++j) {
    LaunchTimer t(s->stream, 2);
    const void *lam = w.lam + (size_t)j * s->bytes;
    const cudaError_t e = s->dt == SV_C64
                              ? Launch<float>::dot_partials(lam, s->psi, s->n, w.partials + (size_t)j * kNormBlocks, s->stream)
                              : Launch<double>::dot_partials(lam, s->psi, s->n, w.partials + (size_t)j * kNormBlocks, s->stream);
    if (sv_status r = after_launch(s, e, "expval dot")) return r;
    ++p->launches;
  }
  LaunchTimer t(s->stream, 4);
  ++p->launches;
  return after_launch(s, jvp_combine(w.partials, kNormBlocks, p->m, 0, w.expvals, s->stream, 1.0), "expval combine");
}

// Hamiltonians of several words per observable (any precision): the lambdas
// H_j psi, which the sweep needs anyway, are formed first and give the
// expectation values by one dot product each (2V per observable against a
// pass over the state per word group).  Z-only observables keep their
// transform pass, which reads the state once for all of them.
bool lambda_first(const sv_program *p) {
  if (!(p->m > 0 && p->m <= 64 && p->n_chunks == 1 && p->terms.size() >= 4 * (size_t)p->m && needs_sweep(p)))
    return false;
  for (const PassDev &pd : p->tp.passes)
    if (!pd.zonly) return true;
  return false;
}

sv_status run_jacobian(sv_program *p, const JacWs &w) {
  sv_state *s = p->s;
  if (sv_status r = ensure_mats(p)) return r;
  const bool lam_first = lambda_first(p);
  if (!lam_first)
    if (sv_status r = run_expval(p, s->psi, w)) return r;
  if (needs_sweep(p)) {
    const int npass_e = (int)p->tp.passes.size();
    for (int c = 0; c < p->n_chunks; ++c) {
      const int j0 = c * p->mc, mcc = std::min(p->m, j0 + p->mc) - j0;
      auto begin = [&](int q) { return (const int32_t *)p->d_lam_begin + p->lam_begin_off[c * npass_e + q]; };
      if (lam_first) {
        const Ops &K = ops_of(s);
        for (int q = 0; q < npass_e; ++q) {
          cudaError_t e;
          {
            LaunchTimer t(s->stream, 3);
            e = K.lambda_pass(s->psi, w.lam, s->n, p->tp.passes[q], p->d_lam_terms, begin(q), mcc, q == 0,
                              p->grid_l(mcc), s->stream);
          }
          if (sv_status r = after_launch(s, e, "lambda pass")) return r;
          ++p->launches;
        }
        if (sv_status r = expvals_from_lambdas(p, w)) return r;
      }
      if (sv_status r = run_sweep(p, w, mcc, j0, p->m, p->d_lam_terms, begin, lam_first)) return r;
    }
  }
  cudaError_t e;
  if (p->adj.n_train > 0 && p->n_params > 0) {
    LaunchTimer t(s->stream, 4);
    e = assemble_jacobian(w.contrib, p->d_coef, p->d_pbegin, p->d_pslots, p->n_params, p->m, 0, p->n_params, w.J,
                          s->stream);
    ++p->launches;
  } else {
    e = cudaMemsetAsync(w.J, 0, (size_t)std::max(1, p->m) * std::max(1, p->n_params) * 8, s->stream);
  }
  return after_launch(s, e, "assemble jacobian");
}

// Variances: Var_j = ||H_j psi||^2 - <H_j>^2 (H_j Hermitian), with lambda_j =
// H_j psi from the lambda passes and ||lambda_j||^2 as fixed FP64 partials.
// Output in w.J[0..m).
sv_status run_var(sv_program *p, const JacWs &w) {
  sv_state *s = p->s;
  if (sv_status r = run_expval(p, s->psi, w)) return r;
  const Ops &K = ops_of(s);
  const int npass_e = (int)p->tp.passes.size();
  for (int c = 0; c < p->n_chunks; ++c) {
    const int j0 = c * p->mc, mcc = std::min(p->m, j0 + p->mc) - j0;
    for (int q = 0; q < npass_e; ++q) {
      const int32_t *begin = (const int32_t *)p->d_lam_begin + p->lam_begin_off[c * npass_e + q];
      cudaError_t e;
      {
        LaunchTimer t(s->stream, 3);
        e = K.lambda_pass(s->psi, w.lam, s->n, p->tp.passes[q], p->d_lam_terms, begin, mcc, q == 0, p->grid_l(mcc),
                          s->stream);
      }
      if (sv_status r = after_launch(s, e, "lambda pass")) return r;
      ++p->launches;
    }
    if (npass_e == 0) {  // observables without terms: lambda = 0
      if (sv_status r = after_launch(s, cudaMemsetAsync(w.lam, 0, (size_t)mcc * s->bytes, s->stream), "lambda"))
        return r;
    }
    for (int j = 0; j < mcc; ++j) {
      const void *lam = w.lam + (size_t)j * s->bytes;
      const cudaError_t e = s->dt == SV_C64
                                ? Launch<float>::norm_partials(lam, s->n, w.partials + (size_t)j * kNormBlocks, s->stream)
                                : Launch<double>::norm_partials(lam, s->n, w.partials + (size_t)j * kNormBlocks, s->stream);
      if (sv_status r = after_launch(s, e, "variance norm")) return r;
      ++p->launches;
    }
    if (sv_status r = after_launch(s, var_combine(w.partials, kNormBlocks, mcc, w.expvals, j0, w.J, s->stream),
                                   "variance combine"))
      return r;
    ++p->launches;
  }
  return SV_OK;
}

// Jacobian-vector product along `tangent` (forward mode): one tangent pass
// from the state's current contents carries psi and dpsi (dpsi starts at 0);
// then out_j = 2 Re <H_j psi | dpsi> from the lambda passes and FP64 dots.
// Output in w.J[0..m); the state ends as the forward output.
sv_status run_jvp(sv_program *p, const JacWs &w, const double *tangent) {
  sv_state *s = p->s;
  if (sv_status r = ensure_mats(p)) return r;
  const Ops &K = ops_of(s);
  std::vector<double2> coefs(std::max(1, p->tan.n_train));
  for (int sidx = 0; sidx < p->tan.n_train; ++sidx) {
    const int q = p->tan_pidx[sidx];
    coefs[sidx] = make_double2(0.0, q >= 0 ? p->tan_factor[sidx] * tangent[q] : 0.0);  // i s scale tangent[q]
  }
  cudaError_t e = cudaMemcpyAsync(w.tan_coefs, coefs.data(), coefs.size() * sizeof(double2), cudaMemcpyHostToDevice,
                                  s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.phiA, 0, s->bytes, s->stream);
  if (sv_status r = after_launch(s, e, "tangent setup")) return r;
  for (const Step &st : p->tan.steps) {
    if (st.dense_k) {
      LaunchTimer t(s->stream, 6);
      e = K.dense_k(s->psi, s->n, p->tan.dk_ops[st.index], p->d_mats, 0, s->stream);
      if (e == cudaSuccess) e = K.dense_k(w.phiA, s->n, p->tan.dk_ops[st.index], p->d_mats, 0, s->stream);
      p->launches += 2;
    } else {
      LaunchTimer t(s->stream, 0);
      e = K.tile_tangent(s->psi, w.phiA, s->n, p->tan.passes[st.index], p->d_tan_ops, p->d_mats, w.tan_coefs,
                         p->grid_f, s->stream);
      ++p->launches;
    }
    if (sv_status r = after_launch(s, e, "tangent pass")) return r;
  }
  const int npass_e = (int)p->tp.passes.size();
  for (int c = 0; c < p->n_chunks; ++c) {
    const int j0 = c * p->mc, mcc = std::min(p->m, j0 + p->mc) - j0;
    for (int q = 0; q < npass_e; ++q) {
      const int32_t *begin = (const int32_t *)p->d_lam_begin + p->lam_begin_off[c * npass_e + q];
      LaunchTimer t(s->stream, 3);
      e = K.lambda_pass(s->psi, w.lam, s->n, p->tp.passes[q], p->d_lam_terms, begin, mcc, q == 0, p->grid_l(mcc),
                        s->stream);
      if (sv_status r = after_launch(s, e, "lambda pass")) return r;
      ++p->launches;
    }
    if (npass_e == 0) {
      if (sv_status r = after_launch(s, cudaMemsetAsync(w.lam, 0, (size_t)mcc * s->bytes, s->stream), "lambda"))
        return r;
    }
    for (int j = 0; j < mcc; ++j) {
      const void *lam = w.lam + (size_t)j * s->bytes;
      e = s->dt == SV_C64 ? Launch<float>::dot_partials(lam, w.phiA, s->n, w.partials + (size_t)j * kNormBlocks, s->stream)
                          : Launch<double>::dot_partials(lam, w.phiA, s->n, w.partials + (size_t)j * kNormBlocks, s->stream);
      if (sv_status r = after_launch(s, e, "jvp dot")) return r;
      ++p->launches;
    }
    if (sv_status r = after_launch(s, jvp_combine(w.partials, kNormBlocks, mcc, j0, w.J, s->stream), "jvp combine"))
      return r;
    ++p->launches;
  }
  return SV_OK;
}

// VJP: lambda = sum_j g_j H_j psi, one sweep, one contrib column.
sv_status run_vjp(sv_program *p, const JacWs &w, const double *g) {
  sv_state *s = p->s;
  if (sv_status r = ensure_mats(p)) return r;
  std::vector<TermDev> &vt = p->vjp_host;
  for (size_t q = 0; q < vt.size(); ++q) vt[q].coeff = p->terms[p->tp.placed[q]].coeff * g[p->terms[p->tp.placed[q]].obs];
  cudaError_t e = cudaMemcpyAsync(p->d_vjp_terms, vt.data(), vt.size() * sizeof(TermDev), cudaMemcpyHostToDevice,
                                  s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "uploading vjp coefficients");
  if (needs_sweep(p)) {
    auto begin = [&](int q) { return (const int32_t *)p->d_vjp_begin + 2 * q; };
    if (sv_status r = run_sweep(p, w, 1, 0, 1, p->d_vjp_terms, begin)) return r;
  }
  if (p->adj.n_train > 0 && p->n_params > 0) {
    LaunchTimer t(s->stream, 4);
    e = assemble_jacobian(w.contrib, p->d_coef, p->d_pbegin, p->d_pslots, p->n_params, 1, 0, p->n_params, w.J,
                          s->stream);
    ++p->launches;
  } else {
    e = cudaMemsetAsync(w.J, 0, (size_t)std::max(1, p->n_params) * 8, s->stream);
  }
  return after_launch(s, e, "assemble vjp");
}

sv_status copy_out(sv_state *s, double *dst, const double *src, size_t count, bool on_device) {
  if (!dst || count == 0) return SV_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, count * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying results");
  return SV_OK;
}

sv_status sync_state(sv_state *s) {
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    s->latched = 1;
    return cuda_fail(e, "stream synchronize");
  }
  if (dense5_tc_take_error()) {
    s->latched = 1;
    return fail(SV_ERR_TIMEOUT, "a tensor-core dense-block wait ran out (results of the last call are invalid)");
  }
  return SV_OK;
}

}  // namespace


// ---- batched circuits ---------------------------------------------------------------
struct sv_batch {
  sv_dtype dt = SV_C64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_circ = 0;
  // inputs, kept for re-planning by the autotuner
  std::vector<int> nq;
  std::vector<std::vector<sv_op>> ops;
  std::vector<int> np;
  std::vector<std::vector<double>> umat;
  std::vector<std::vector<ZTerm>> zterms_wire;  // z as wire masks until planned
  std::vector<uint64_t> basis;
  int total_params = 0;
  // plan
  int tile_cap = 0;          // tile bits cap (autotuned)
  int64_t wave_bytes = 64ll << 20;
  int ctas_per_sm_cap = 0;   // CTAs per SM at most (0: as many as fit; autotuned)
  int n_segs = 0, n_pass = 0, n_slots = 0, max_T = 1, max_terms = 1, max_k = 1, grid = 1;
  int64_t total_items = 0, n_partials = 0;
  int no_publish = -1;
  unsigned long long timeout_ns = 2000000000ull;
  // device memory
  void *tables = nullptr;
  size_t tables_bytes = 0;
  void *states = nullptr;
  size_t states_bytes = 0;
  void *work = nullptr;
  size_t work_bytes = 0;
  BatchCircuit *d_circs = nullptr;
  PassDev *d_passes = nullptr;
  OpDev *d_ops = nullptr;
  MatSlot *d_slots = nullptr;
  void *d_mats = nullptr;
  double *d_params = nullptr, *d_user = nullptr;
  BatchSeg *d_segs = nullptr;
  ZTerm *d_terms = nullptr;
  uint64_t *d_aux = nullptr;  // phase-run member records
  double *d_partials = nullptr, *d_out = nullptr;
  int *d_done = nullptr, *d_err = nullptr;
  unsigned long long *d_head = nullptr;
  bool params_set = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
};

namespace {

void batch_free_plan(sv_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  dev_free(b->tables, b->tables_bytes);
  dev_free(b->work, b->work_bytes);
  b->tables = b->work = nullptr;
  b->tables_bytes = b->work_bytes = 0;
}

// Plan every circuit with tile cap `tcap` and L2 waves of `wave` bytes; upload tables.
sv_status batch_plan(sv_batch *b, int tcap, int64_t wave) {
  const Ops &K = ops_for(b->dt);
  std::vector<BatchCircuit> circs(b->n_circ);
  std::vector<PassDev> passes;
  std::vector<OpDev> dops;
  std::vector<ZTerm> terms;
  SlotTable st;
  std::vector<double> user;
  std::vector<uint64_t> aux;
  int param_off = 0;
  uint64_t state_off = 0;
  int64_t part_off = 0;
  int max_T = 1, max_terms = 1, max_k = 1;
  for (int i = 0; i < b->n_circ; ++i) {
    const int n = b->nq[i];
    const int64_t uoff = (int64_t)user.size() / 2;
    user.insert(user.end(), b->umat[i].begin(), b->umat[i].end());
    std::vector<HOp> hops;
    for (const sv_op &o : b->ops[i]) {
      HOp h = to_hop(o, b->umat[i].empty() ? nullptr : b->umat[i].data());
      for (int a = 0; a < 3; ++a)
        if (h.pidx[a] >= 0) h.pidx[a] += param_off;
      h.msrc += uoff;
      if (!h.diag && h.k > kMaxTileTargets)
        return fail(SV_ERR_UNSUPPORTED, "batch circuit %d: dense matrix on more than %d wires", i, kMaxTileTargets);
      hops.push_back(h);
    }
    const int T = std::min(std::min(tcap, K.Tf), n);
    Plan P = plan_passes(n, hops, T, K.nlow_pref, 1 << 30, false, st, true, true, true);
    if (sv_status e = check_plan(P, n, K.nlow_pref)) return e;
    const int aux_base = (int)(aux.size() / 2);
    for (OpDev &o : P.ops)
      if (o.kind == kPhase) o.oa += aux_base;
    aux.insert(aux.end(), P.aux.begin(), P.aux.end());
    BatchCircuit &c = circs[i];
    memset(&c, 0, sizeof(c));
    c.n = n;
    c.pass_begin = (int)passes.size();
    const int op_base = (int)dops.size();
    for (PassDev pd : P.passes) {
      pd.op_begin += op_base;
      pd.op_end += op_base;
      max_k = std::max(max_k, pd.max_k);
      passes.push_back(pd);
    }
    if (P.passes.empty()) {  // empty tape: one pass without ops carries the measurement
      PassDev pd = make_pass(n, fill_bits(low_bits(n, T, K.nlow_pref), n, T, K.nlow_pref));
      pd.op_begin = pd.op_end = op_base;
      passes.push_back(pd);
    }
    dops.insert(dops.end(), P.ops.begin(), P.ops.end());
    c.n_pass = (int)passes.size() - c.pass_begin;
    c.tiles = 1 << (n - T);
    c.term_begin = (int)terms.size();
    for (const ZTerm &z : b->zterms_wire[i]) terms.push_back({wire_mask_to_global(z.z, n), z.coeff});
    c.n_terms = (int)terms.size() - c.term_begin;
    c.out = i;
    c.part_begin = part_off;
    part_off += (int64_t)c.n_terms * c.tiles;
    c.state_off = state_off;
    state_off += 1ull << n;
    c.basis = b->basis[i];
    max_T = std::max(max_T, T);
    max_terms = std::max(max_terms, c.n_terms);
    param_off += b->np[i];
  }
  if (max_terms > 2048) return fail(SV_ERR_UNSUPPORTED, "batch: more than 2048 Z words in one observable");
  // segments: waves of circuits whose states fit in `wave` bytes; inside a wave
  // pass p of every circuit precedes pass p + 1 of any circuit
  std::vector<BatchSeg> segs;
  int64_t items = 0;
  int c0 = 0;
  while (c0 < b->n_circ) {
    int c1 = c0;
    int64_t bytes = 0;
    while (c1 < b->n_circ && (c1 == c0 || bytes + ((int64_t)K.amp_bytes << circs[c1].n) <= wave)) {
      bytes += (int64_t)K.amp_bytes << circs[c1].n;
      ++c1;
    }
    int maxp = 0;
    for (int c = c0; c < c1; ++c) maxp = std::max(maxp, circs[c].n_pass);
    for (int pp = 0; pp < maxp; ++pp)
      for (int c = c0; c < c1; ++c) {
        if (pp >= circs[c].n_pass) continue;
        BatchSeg sg;
        memset(&sg, 0, sizeof(sg));
        sg.first_item = items;
        sg.circ = c;
        sg.pass = pp;
        sg.ntiles = circs[c].tiles;
        segs.push_back(sg);
        items += sg.ntiles;
      }
    c0 = c1;
  }

  batch_free_plan(b);
  b->tile_cap = tcap;
  b->wave_bytes = wave;
  b->n_segs = (int)segs.size();
  b->n_pass = (int)passes.size();
  b->n_slots = (int)st.slots.size();
  b->max_T = max_T;
  b->max_terms = max_terms;
  b->max_k = max_k;
  b->total_items = items;
  b->n_partials = part_off;
  const int sms = sm_count();
  const int per_sm = b->dt == SV_C64 ? Launch<float>::batch_blocks_per_sm(max_T, max_terms, max_k)
                                     : Launch<double>::batch_blocks_per_sm(max_T, max_terms, max_k);
  const int per_sm_used = b->ctas_per_sm_cap > 0 ? std::min(per_sm, b->ctas_per_sm_cap) : per_sm;
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)sms * per_sm_used));
  if (const char *e = getenv("SV_BATCH_DEBUG_NO_PUBLISH")) b->no_publish = atoi(e);
  if (const char *e = getenv("SV_BATCH_TIMEOUT_MS")) b->timeout_ns = 1000000ull * (unsigned long long)atoll(e);

  auto sz = [](size_t count, size_t elem) { return align256(count * elem); };
  size_t total = sz(circs.size(), sizeof(BatchCircuit)) + sz(passes.size(), sizeof(PassDev)) +
                 sz(dops.size(), sizeof(OpDev)) + sz(st.slots.size(), sizeof(MatSlot)) + sz(st.entries, K.amp_bytes) +
                 sz(std::max(b->total_params, 1), 8) + sz(std::max<size_t>(user.size(), 1), 8) +
                 sz(segs.size(), sizeof(BatchSeg)) + sz(std::max<size_t>(terms.size(), 1), sizeof(ZTerm)) +
                 sz(aux.size(), 8);
  if (sv_status e = dev_alloc(&b->tables, total)) return e;
  b->tables_bytes = total;
  std::vector<char> host(total, 0);
  size_t cur = 0;
  auto put = [&](const void *src, size_t count, size_t elem) -> char * {
    char *d = (char *)b->tables + cur;
    if (count && src) memcpy(host.data() + cur, src, count * elem);
    cur += align256(count * elem);
    return d;
  };
  b->d_circs = (BatchCircuit *)put(circs.data(), circs.size(), sizeof(BatchCircuit));
  b->d_passes = (PassDev *)put(passes.data(), passes.size(), sizeof(PassDev));
  b->d_ops = (OpDev *)put(dops.data(), dops.size(), sizeof(OpDev));
  b->d_slots = (MatSlot *)put(st.slots.data(), st.slots.size(), sizeof(MatSlot));
  b->d_mats = put(nullptr, st.entries, K.amp_bytes);
  b->d_params = (double *)put(nullptr, std::max(b->total_params, 1), 8);
  b->d_user = (double *)put(user.data(), std::max<size_t>(user.size(), 1), 8);
  b->d_segs = (BatchSeg *)put(segs.data(), segs.size(), sizeof(BatchSeg));
  b->d_terms = (ZTerm *)put(terms.data(), std::max<size_t>(terms.size(), 1), sizeof(ZTerm));
  b->d_aux = (uint64_t *)put(aux.data(), aux.size(), 8);
  // the parameters survive re-planning: keep the previous values on the host side
  cudaError_t e = cudaMemcpyAsync(b->tables, host.data(), total, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "uploading batch tables");

  const size_t wtotal = align256((size_t)std::max<int64_t>(part_off, 1) * 8) + align256((size_t)b->n_circ * 8) +
                        align256((size_t)b->n_pass * 4) + 256 + 256;
  if (sv_status e2 = dev_alloc(&b->work, wtotal)) return e2;
  b->work_bytes = wtotal;
  char *w = (char *)b->work;
  b->d_partials = (double *)w;
  w += align256((size_t)std::max<int64_t>(part_off, 1) * 8);
  b->d_out = (double *)w;
  w += align256((size_t)b->n_circ * 8);
  b->d_done = (int *)w;
  w += align256((size_t)b->n_pass * 4);
  b->d_head = (unsigned long long *)w;
  w += 256;
  b->d_err = (int *)w;
  if (!b->states) {
    b->states_bytes = (size_t)state_off * K.amp_bytes;
    if (sv_status e3 = dev_alloc(&b->states, b->states_bytes)) return e3;
  }
  return SV_OK;
}

// The launches of one run, in stream order (captured into the graph).
sv_status batch_enqueue(sv_batch *b) {
  const Ops &K = ops_for(b->dt);
  cudaStream_t s = b->stream;
  cudaError_t e = cudaMemsetAsync(b->d_done, 0, (size_t)b->n_pass * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_head, 0, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, 4, s);
  if (e == cudaSuccess) e = K.build_matrices(b->d_slots, b->n_slots, b->d_params, b->d_user, b->d_mats, s);
  if (e == cudaSuccess)
    e = b->dt == SV_C64
            ? Launch<float>::batch(b->states, b->d_circs, b->d_passes, b->d_ops, b->d_mats, b->d_aux, b->d_segs, b->n_segs,
                                   b->total_items, b->d_terms, b->d_partials, b->d_done, b->d_head, b->d_err, 0,
                                   b->timeout_ns, b->max_T, b->max_terms, b->max_k, b->no_publish, b->grid, s)
            : Launch<double>::batch(b->states, b->d_circs, b->d_passes, b->d_ops, b->d_mats, b->d_aux, b->d_segs, b->n_segs,
                                    b->total_items, b->d_terms, b->d_partials, b->d_done, b->d_head, b->d_err, 0,
                                    b->timeout_ns, b->max_T, b->max_terms, b->max_k, b->no_publish, b->grid, s);
  if (e == cudaSuccess) e = batch_reduce(b->d_circs, b->n_circ, b->d_terms, b->d_partials, b->d_out, s);
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "batch launch");
}

sv_status batch_launch(sv_batch *b) {
  if (!b->use_graph) return batch_enqueue(b);
  if (!b->exec) {
    // one plain run first (sets kernel attributes outside the capture), then capture
    if (sv_status st = batch_enqueue(b)) return st;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch warm-up");
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->use_graph = false;  // e.g. the legacy default stream: launch directly
      return batch_enqueue(b);
    }
    sv_status st = batch_enqueue(b);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->stream, &g);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "batch graph instantiate");
    }
    b->graph = g;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "batch graph launch");
}

sv_status batch_check(sv_batch *b) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, b->d_err, 4, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch run");
  if (err) return fail(SV_ERR_TIMEOUT, "batch: a bounded wait for a previous pass gave up");
  return SV_OK;
}

}  // namespace

namespace sv {
void set_error_message(const char *msg) { g_err = msg ? msg : ""; }
}  // namespace sv

// ==== C ABI ==========================================================================
extern "C" {

const char *sv_last_error(void) { return g_err.c_str(); }

const char *sv_version(void) {
  return "libsv 1.0 (sm_103a; complex64/complex128; fused tile passes, adjoint Jacobian)";
}

sv_status sv_set_alloc_cap(size_t bytes) {
  g_alloc_cap = bytes;
  return SV_OK;
}

sv_status sv_create(int n, sv_dtype dtype, sv_state **out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > SV_MAX_QUBITS) return fail(SV_ERR_ARG, "n = %d outside [1, %d]", n, SV_MAX_QUBITS);
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype %d", (int)dtype);
  sv_state *s = new sv_state();
  s->n = n;
  s->dt = dtype;
  s->bytes = (size_t)ops_for(dtype).amp_bytes << n;
  if (sv_status st = dev_alloc(&s->psi, s->bytes)) {
    delete s;
    return st;
  }
  s->owns = true;
  s->renorm = dtype == SV_C64;
  cudaError_t e = ops_for(dtype).set_basis(s->psi, n, 0, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    dev_free(s->psi, s->bytes);
    delete s;
    return cuda_fail(e, "sv_create");
  }
  *out = s;
  return SV_OK;
}

sv_status sv_create_from_device_ptr(int n, sv_dtype dtype, void *device_ptr, sv_state **out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > SV_MAX_QUBITS) return fail(SV_ERR_ARG, "n = %d outside [1, %d]", n, SV_MAX_QUBITS);
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype %d", (int)dtype);
  if (!device_ptr) return fail(SV_ERR_ARG, "device_ptr is NULL");
  if (((uintptr_t)device_ptr) & 255) return fail(SV_ERR_ARG, "device_ptr must be 256-byte aligned");
  sv_state *s = new sv_state();
  s->n = n;
  s->dt = dtype;
  s->bytes = (size_t)ops_for(dtype).amp_bytes << n;
  s->psi = device_ptr;
  s->owns = false;
  s->renorm = dtype == SV_C64;
  *out = s;
  return SV_OK;
}

sv_status sv_destroy(sv_state *s) {
  if (!s) return SV_OK;
  cudaStreamSynchronize(s->stream);
  if (s->owns) dev_free(s->psi, s->bytes);
  dev_free(s->ws, s->ws_bytes);
  dev_free(s->tab, s->tab_bytes);
  dev_free(s->d_norm, s->d_norm ? kNormBlocks * sizeof(double) : 0);
  delete s;
  return SV_OK;
}

sv_status sv_set_stream(sv_state *s, void *cuda_stream) {
  if (!s) return fail(SV_ERR_ARG, "state is NULL");
  s->stream = (cudaStream_t)cuda_stream;
  return SV_OK;
}

sv_status sv_set_workspace(sv_state *s, void *device_ptr, size_t bytes) {
  if (!s) return fail(SV_ERR_ARG, "state is NULL");
  if (device_ptr && ((uintptr_t)device_ptr & 255)) return fail(SV_ERR_ARG, "workspace must be 256-byte aligned");
  s->user_ws = device_ptr;
  s->user_ws_bytes = device_ptr ? bytes : 0;
  return SV_OK;
}

sv_status sv_set_compute(sv_state *s, int compute) {
  if (!s) return fail(SV_ERR_ARG, "state is NULL");
  if (compute != SV_COMPUTE_NATIVE && compute != SV_COMPUTE_DOUBLE_FLOAT)
    return fail(SV_ERR_ARG, "unknown compute mode %d", compute);
  if (compute == SV_COMPUTE_DOUBLE_FLOAT && s->dt != SV_C128)
    return fail(SV_ERR_ARG, "double-float arithmetic applies to complex128 states only");
  s->compute = compute;
  return SV_OK;
}

sv_status sv_set_renormalize(sv_state *s, int on) {
  if (!s) return fail(SV_ERR_ARG, "state is NULL");
  if (on != 0 && on != 1) return fail(SV_ERR_ARG, "renormalize flag must be 0 or 1, got %d", on);
  s->renorm = on;
  return SV_OK;
}

sv_status sv_set_dense_tensor_cores(int on) {
  if (on != 0 && on != 1) return fail(SV_ERR_ARG, "flag must be 0 or 1, got %d", on);
  dense5_tc_enable(on != 0);
  return SV_OK;
}

sv_status sv_info(const sv_state *s, int *n, sv_dtype *dtype, void **device_ptr) {
  if (!s) return fail(SV_ERR_ARG, "state is NULL");
  if (n) *n = s->n;
  if (dtype) *dtype = s->dt;
  if (device_ptr) *device_ptr = s->psi;
  return SV_OK;
}

sv_status sv_reset(sv_state *s, uint64_t basis_index) {
  if (!s) return fail(SV_ERR_ARG, "state is NULL");
  if (basis_index >> s->n) return fail(SV_ERR_ARG, "basis index %llu >= 2^%d", (unsigned long long)basis_index, s->n);
  s->latched = 0;
  return after_launch(s, ops_for(s->dt).set_basis(s->psi, s->n, basis_index, s->stream), "sv_reset");
}

sv_status sv_set_state(sv_state *s, const void *host_amplitudes) {
  if (sv_status st = check_state(s)) return st;
  if (!host_amplitudes) return fail(SV_ERR_ARG, "host buffer is NULL");
  SV_CUDA(cudaMemcpyAsync(s->psi, host_amplitudes, s->bytes, cudaMemcpyHostToDevice, s->stream));
  return sync_state(s);
}

sv_status sv_get_state(sv_state *s, void *host_amplitudes) {
  if (sv_status st = check_state(s)) return st;
  if (!host_amplitudes) return fail(SV_ERR_ARG, "host buffer is NULL");
  SV_CUDA(cudaMemcpyAsync(host_amplitudes, s->psi, s->bytes, cudaMemcpyDeviceToHost, s->stream));
  return sync_state(s);
}

sv_status sv_synchronize(sv_state *s) {
  if (!s) return fail(SV_ERR_ARG, "state is NULL");
  if (sv_status st = sync_state(s)) return st;
  return s->latched ? fail(SV_ERR_STATE, "device error latched") : SV_OK;
}

sv_status sv_apply_op(sv_state *s, const sv_op *op, const double *params, const double *matrices) {
  if (sv_status st = check_state(s)) return st;
  if (!op) return fail(SV_ERR_ARG, "op is NULL");
  int np = 0;
  for (int a = 0; a < 3; ++a) np = std::max(np, op->param_index[a] + 1);
  int64_t nm = 0;  // entries the matrix data must hold; out-of-range sizes are rejected by the op check
  if (op->kind == SV_MATRIX && op->n_targets >= 1 && op->n_targets <= SV_MAX_TARGETS && op->matrix_offset >= 0 &&
      op->matrix_offset < ((int64_t)1 << 48))
    nm = op->matrix_offset + ((int64_t)1 << (2 * op->n_targets));
  sv_tape tape = {1, op, np, matrices, nm};
  sv_program *p = nullptr;
  if (sv_status st = build_program(s, &tape, nullptr, 0, params, true, &p)) return st;
  sv_status st = program_set_params(p, params, 0);
  if (!st) st = run_steps_forward(p, s->psi);
  if (!st) st = sync_state(s);
  destroy_program(p);
  return st;
}

sv_status sv_apply(sv_state *s, int kind, const int *wires, int n_wires, const double *angles, int adjoint) {
  if (sv_status st = check_state(s)) return st;
  if (kind == SV_MATRIX) return fail(SV_ERR_ARG, "use sv_apply_matrix for SV_MATRIX");
  if (kind < 0 || kind >= SV_OP_KIND_COUNT) return fail(SV_ERR_ARG, "unknown op kind %d", kind);
  if (n_wires < 0 || n_wires > SV_MAX_TARGETS || (n_wires > 0 && !wires)) return fail(SV_ERR_ARG, "bad wires");
  const int np = kind_nparams(kind);
  if (np > 0 && !angles) return fail(SV_ERR_ARG, "angles is NULL for a parametric gate");
  sv_op op;
  memset(&op, 0, sizeof(op));
  op.kind = kind;
  op.n_targets = n_wires;
  for (int j = 0; j < n_wires; ++j) op.targets[j] = wires[j];
  for (int a = 0; a < 3; ++a) op.param_index[a] = a < np ? a : -1;
  op.scale = 1.0;
  op.adjoint = adjoint;
  return sv_apply_op(s, &op, angles, nullptr);
}

sv_status sv_apply_matrix(sv_state *s, const int *wires, int k, const double *matrix, int adjoint) {
  if (sv_status st = check_state(s)) return st;
  if (k < 1 || k > SV_MAX_TARGETS || !wires || !matrix) return fail(SV_ERR_ARG, "bad sv_apply_matrix arguments");
  sv_op op;
  memset(&op, 0, sizeof(op));
  op.kind = SV_MATRIX;
  op.n_targets = k;
  for (int j = 0; j < k; ++j) op.targets[j] = wires[j];
  op.param_index[0] = op.param_index[1] = op.param_index[2] = -1;
  op.scale = 1.0;
  op.adjoint = adjoint;
  op.matrix_offset = 0;
  return sv_apply_op(s, &op, nullptr, matrix);
}

sv_status sv_expval(sv_state *s, const sv_pauli_sum *obs, int n_obs, double *out) {
  if (sv_status st = check_state(s)) return st;
  if (n_obs > 0 && !out) return fail(SV_ERR_ARG, "out is NULL");
  if (n_obs == 0) return SV_OK;
  sv_program *p = nullptr;
  if (sv_status st = build_program(s, nullptr, obs, n_obs, nullptr, true, &p)) return st;
  JacWs w;
  sv_status st = jac_workspace(p, w);
  if (!st) st = run_expval(p, s->psi, w);
  if (!st) st = copy_out(s, out, w.expvals, n_obs, false);
  if (!st) st = sync_state(s);
  destroy_program(p);
  return st;
}

sv_status sv_var(sv_state *s, const sv_pauli_sum *obs, int n_obs, double *out) {
  if (sv_status st = check_state(s)) return st;
  if (n_obs > 0 && !out) return fail(SV_ERR_ARG, "out is NULL");
  if (n_obs == 0) return SV_OK;
  sv_program *p = nullptr;
  if (sv_status st = build_program(s, nullptr, obs, n_obs, nullptr, true, &p)) return st;
  p->want_lam = true;
  JacWs w;
  sv_status st = jac_workspace(p, w);
  if (!st) st = run_var(p, w);
  if (!st) st = copy_out(s, out, w.J, n_obs, false);
  if (!st) st = sync_state(s);
  destroy_program(p);
  return st;
}

namespace {
// Marginal probabilities of `wires` into dev_probs (2^k doubles, device).
sv_status probs_device(sv_state *s, const int *wires, int k, double *dev_probs, double *partials) {
  ProbsDev pd;
  memset(&pd, 0, sizeof(pd));
  pd.n = s->n;
  pd.k = k;
  pd.chunk_log = std::min(s->n - k, 12);
  uint64_t mask = 0;
  for (int j = 0; j < k; ++j) {
    pd.bitpos[j] = (int8_t)(s->n - 1 - wires[j]);
    mask |= 1ull << (s->n - 1 - wires[j]);
  }
  int q = 0;
  for (int b = 0; b < s->n; ++b)
    if ((mask >> b) & 1) pd.pos[q++] = (int8_t)b;
  cudaError_t e;
  if (s->n - k <= kProbsSmallLog) {
    e = s->dt == SV_C64 ? Launch<float>::probs_small(s->psi, pd, dev_probs, s->stream)
                        : Launch<double>::probs_small(s->psi, pd, dev_probs, s->stream);
  } else {
    e = s->dt == SV_C64 ? Launch<float>::probs_partials(s->psi, pd, partials, s->stream)
                        : Launch<double>::probs_partials(s->psi, pd, partials, s->stream);
    if (e == cudaSuccess) e = probs_combine(partials, 1ll << k, 1 << (s->n - k - pd.chunk_log), dev_probs, s->stream);
  }
  return after_launch(s, e, "probabilities");
}

sv_status check_wires(const sv_state *s, const int *wires, int k) {
  if (k < 0 || k > std::min(s->n, kMaxProbWires))
    return fail(SV_ERR_ARG, "k = %d wires outside [0, %d]", k, std::min(s->n, kMaxProbWires));
  if (k > 0 && !wires) return fail(SV_ERR_ARG, "wires is NULL");
  uint64_t seen = 0;
  for (int j = 0; j < k; ++j) {
    if (wires[j] < 0 || wires[j] >= s->n) return fail(SV_ERR_ARG, "wire %d outside [0, %d)", wires[j], s->n);
    if ((seen >> wires[j]) & 1) return fail(SV_ERR_ARG, "wire %d repeated", wires[j]);
    seen |= 1ull << wires[j];
  }
  return SV_OK;
}

size_t probs_partials_count(int n, int k) {
  return n - k <= kProbsSmallLog ? 1 : (size_t)1 << (n - std::min(n - k, 12));
}
}  // namespace

sv_status sv_probs(sv_state *s, const int *wires, int k, double *out) {
  if (sv_status st = check_state(s)) return st;
  if (sv_status st = check_wires(s, wires, k)) return st;
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  const size_t bins = (size_t)1 << k, parts = probs_partials_count(s->n, k);
  char *base = nullptr;
  if (sv_status st = get_workspace(s, align256(bins * 8) + align256(parts * 8), &base)) return st;
  double *probs = (double *)base, *partials = (double *)(base + align256(bins * 8));
  sv_status st = probs_device(s, wires, k, probs, partials);
  if (!st) st = copy_out(s, out, probs, bins, false);
  if (!st) st = sync_state(s);
  return st;
}

sv_status sv_sample(sv_state *s, const int *wires, int k, const double *uniforms, int64_t shots, uint64_t *out) {
  if (sv_status st = check_state(s)) return st;
  if (sv_status st = check_wires(s, wires, k)) return st;
  if (shots < 0) return fail(SV_ERR_ARG, "shots < 0");
  if (shots == 0) return SV_OK;
  if (!uniforms || !out) return fail(SV_ERR_ARG, "uniforms / out is NULL");
  for (int64_t t = 0; t < shots; ++t)
    if (!(uniforms[t] >= 0.0 && uniforms[t] < 1.0)) return fail(SV_ERR_ARG, "uniforms[%lld] not in [0, 1)", (long long)t);
  const size_t bins = (size_t)1 << k, parts = probs_partials_count(s->n, k);
  const size_t scan = (bins + 4095) / 4096;
  const size_t bytes = align256(bins * 8) + align256(parts * 8) + align256(scan * 8) + align256((size_t)shots * 8) +
                       align256((size_t)shots * 8);
  char *base = nullptr;
  if (sv_status st = get_workspace(s, bytes, &base)) return st;
  size_t c = 0;
  double *cdf = (double *)(base + c);
  c += align256(bins * 8);
  double *partials = (double *)(base + c);
  c += align256(parts * 8);
  double *scratch = (double *)(base + c);
  c += align256(scan * 8);
  double *u = (double *)(base + c);
  c += align256((size_t)shots * 8);
  uint64_t *dout = (uint64_t *)(base + c);
  cudaError_t e = cudaMemcpyAsync(u, uniforms, (size_t)shots * 8, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying uniforms");
  if (sv_status st = probs_device(s, wires, k, cdf, partials)) return st;
  e = inclusive_scan(cdf, (int64_t)bins, scratch, s->stream);
  if (e == cudaSuccess) e = sample_cdf(cdf, (int64_t)bins, u, shots, dout, s->stream);
  if (sv_status st = after_launch(s, e, "sampling")) return st;
  e = cudaMemcpyAsync(out, dout, (size_t)shots * 8, cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying samples");
  return sync_state(s);
}

// ---- sparse observables ----------------------------------------------------------
struct sv_sparse {
  int n = 0;
  int64_t nnz = 0;
  void *mem = nullptr;
  size_t bytes = 0;
  SparseDev dev;
};

sv_status sv_sparse_create(int n, const int64_t *indptr, const int64_t *indices, const double *values, int64_t nnz,
                           sv_sparse **out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > SV_MAX_QUBITS) return fail(SV_ERR_ARG, "n = %d outside [1, %d]", n, SV_MAX_QUBITS);
  if (nnz < 0) return fail(SV_ERR_ARG, "nnz < 0");
  if (!indptr || (nnz > 0 && (!indices || !values))) return fail(SV_ERR_ARG, "NULL CSR arrays");
  const int64_t rows = 1ll << n;
  if (indptr[0] != 0 || indptr[rows] != nnz) return fail(SV_ERR_ARG, "indptr must run from 0 to nnz");
  for (int64_t r = 0; r < rows; ++r)
    if (indptr[r + 1] < indptr[r]) return fail(SV_ERR_ARG, "indptr decreases at row %lld", (long long)r);
  for (int64_t k = 0; k < nnz; ++k) {
    if (indices[k] < 0 || indices[k] >= rows) return fail(SV_ERR_ARG, "column index %lld out of range", (long long)k);
    if (!std::isfinite(values[2 * k]) || !std::isfinite(values[2 * k + 1]))
      return fail(SV_ERR_ARG, "value %lld is not finite", (long long)k);
  }
  sv_sparse *h = new sv_sparse();
  h->n = n;
  h->nnz = nnz;
  const size_t b_ptr = align256((size_t)(rows + 1) * 8), b_idx = align256((size_t)std::max<int64_t>(nnz, 1) * 8);
  const size_t b_val = align256((size_t)std::max<int64_t>(nnz, 1) * 16);
  h->bytes = b_ptr + b_idx + b_val;
  if (sv_status st = dev_alloc(&h->mem, h->bytes)) {
    delete h;
    return st;
  }
  char *base = (char *)h->mem;
  cudaError_t e = cudaMemcpy(base, indptr, (size_t)(rows + 1) * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(base + b_ptr, indices, (size_t)nnz * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(base + b_ptr + b_idx, values, (size_t)nnz * 16, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    dev_free(h->mem, h->bytes);
    delete h;
    return cuda_fail(e, "sv_sparse_create");
  }
  h->dev.n = n;
  h->dev.nnz_per_row = (double)nnz / (double)rows;
  h->dev.indptr = (const int64_t *)base;
  h->dev.indices = (const int64_t *)(base + b_ptr);
  h->dev.vals = (const double2 *)(base + b_ptr + b_idx);
  *out = h;
  return SV_OK;
}

sv_status sv_sparse_destroy(sv_sparse *h) {
  if (!h) return SV_OK;
  cudaDeviceSynchronize();
  dev_free(h->mem, h->bytes);
  delete h;
  return SV_OK;
}

namespace {
sv_status sparse_expval_device(sv_state *s, const sv_sparse *h, double *partials, double *dev_out) {
  cudaError_t e = s->dt == SV_C64 ? Launch<float>::csr_expval_partials(s->psi, h->dev, partials, s->stream)
                                  : Launch<double>::csr_expval_partials(s->psi, h->dev, partials, s->stream);
  if (e == cudaSuccess) e = probs_combine(partials, 1, kNormBlocks, dev_out, s->stream);  // fixed-order sum
  return after_launch(s, e, "sparse expval");
}
}  // namespace

sv_status sv_sparse_expval(sv_state *s, const sv_sparse *h, double *out) {
  if (sv_status st = check_state(s)) return st;
  if (!h || !out) return fail(SV_ERR_ARG, "NULL sparse observable / out");
  if (h->n != s->n) return fail(SV_ERR_ARG, "sparse observable on %d qubits, state on %d", h->n, s->n);
  char *base = nullptr;
  if (sv_status st = get_workspace(s, align256(kNormBlocks * 8) + 256, &base)) return st;
  double *partials = (double *)base, *dv = (double *)(base + align256(kNormBlocks * 8));
  sv_status st = sparse_expval_device(s, h, partials, dv);
  if (!st) st = copy_out(s, out, dv, 1, false);
  if (!st) st = sync_state(s);
  return st;
}

sv_status sv_adjoint_jacobian_sparse(sv_state *s, const sv_tape *tape, const double *params, const sv_sparse *h,
                                     double *expval_out, double *jacobian_out) {
  if (sv_status st = check_state(s)) return st;
  if (!tape || !h) return fail(SV_ERR_ARG, "NULL tape / sparse observable");
  if (h->n != s->n) return fail(SV_ERR_ARG, "sparse observable on %d qubits, state on %d", h->n, s->n);
  if (tape->n_params > 0 && !jacobian_out) return fail(SV_ERR_ARG, "jacobian_out is NULL");
  // the program's one observable is a placeholder: lambda = H psi comes from the SpMV
  const double one = 1.0;
  const uint64_t zero = 0;
  sv_pauli_sum placeholder = {1, &one, &zero, &zero};
  sv_program *p = nullptr;
  if (sv_status st = build_program(s, tape, &placeholder, 1, params, true, &p)) return st;
  JacWs w;
  sv_status st = program_set_params(p, params, 0);
  if (!st) st = jac_workspace(p, w);
  if (!st) st = ensure_mats(p);
  if (!st) st = sparse_expval_device(s, h, w.partials, w.expvals);
  if (!st && needs_sweep(p)) {  // the workspace holds lambda only when there is a sweep
    const cudaError_t e = s->dt == SV_C64 ? Launch<float>::csr_spmv(s->psi, h->dev, w.lam, s->stream)
                                          : Launch<double>::csr_spmv(s->psi, h->dev, w.lam, s->stream);
    st = after_launch(s, e, "sparse lambda");
    auto begin = [&](int) { return (const int32_t *)nullptr; };
    if (!st) st = run_sweep(p, w, 1, 0, 1, p->d_lam_terms, begin, true);
  }
  if (!st) {
    cudaError_t e;
    if (p->adj.n_train > 0 && p->n_params > 0)
      e = assemble_jacobian(w.contrib, p->d_coef, p->d_pbegin, p->d_pslots, p->n_params, 1, 0, p->n_params, w.J,
                            s->stream);
    else
      e = cudaMemsetAsync(w.J, 0, (size_t)std::max(1, p->n_params) * 8, s->stream);
    st = after_launch(s, e, "assemble jacobian");
  }
  if (!st) st = copy_out(s, expval_out, w.expvals, 1, false);
  if (!st) st = copy_out(s, jacobian_out, w.J, (size_t)tape->n_params, false);
  if (!st) st = sync_state(s);
  destroy_program(p);
  return st;
}

sv_status sv_norm2(sv_state *s, double *out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  const double c = 1.0;
  const uint64_t zero = 0;
  sv_pauli_sum id = {1, &c, &zero, &zero};
  return sv_expval(s, &id, 1, out);
}

sv_status sv_forward(sv_state *s, const sv_tape *tape, const double *params) {
  if (sv_status st = check_state(s)) return st;
  if (!tape) return fail(SV_ERR_ARG, "tape is NULL");
  sv_program *p = nullptr;
  if (sv_status st = build_program(s, tape, nullptr, 0, params, true, &p)) return st;
  sv_status st = program_set_params(p, params, 0);
  if (!st) st = run_steps_forward(p, s->psi);
  if (!st) st = finish_forward(s);
  if (!st) st = sync_state(s);
  destroy_program(p);
  return st;
}

sv_status sv_adjoint_jacobian(sv_state *s, const sv_tape *tape, const double *params, const sv_pauli_sum *obs,
                              int n_obs, double *expvals_out, double *jacobian_out) {
  if (sv_status st = check_state(s)) return st;
  if (!tape) return fail(SV_ERR_ARG, "tape is NULL");
  if (n_obs < 1) return fail(SV_ERR_ARG, "need at least one observable");
  if (tape->n_params > 0 && !jacobian_out) return fail(SV_ERR_ARG, "jacobian_out is NULL");
  sv_program *p = nullptr;
  if (sv_status st = build_program(s, tape, obs, n_obs, params, true, &p)) return st;
  JacWs w;
  sv_status st = program_set_params(p, params, 0);
  if (!st) st = jac_workspace(p, w);
  if (!st) st = run_jacobian(p, w);
  if (!st) st = copy_out(s, expvals_out, w.expvals, n_obs, false);
  if (!st) st = copy_out(s, jacobian_out, w.J, (size_t)n_obs * tape->n_params, false);
  if (!st) st = sync_state(s);
  destroy_program(p);
  return st;
}

sv_status sv_adjoint_vjp(sv_state *s, const sv_tape *tape, const double *params, const sv_pauli_sum *obs, int n_obs,
                         const double *grad_out, double *vjp_out) {
  if (sv_status st = check_state(s)) return st;
  if (!tape || !grad_out || (tape->n_params > 0 && !vjp_out) || n_obs < 1 || !obs)
    return fail(SV_ERR_ARG, "bad sv_adjoint_vjp arguments");
  // lambda = sum_j g_j H_j psi: one merged Pauli sum, one backward sweep
  std::vector<double> c;
  std::vector<uint64_t> x, z;
  for (int j = 0; j < n_obs; ++j) {
    if (!std::isfinite(grad_out[j])) return fail(SV_ERR_ARG, "grad_out[%d] is not finite", j);
    if (obs[j].n_terms < 0) return fail(SV_ERR_ARG, "observable %d: n_terms < 0", j);
    if (obs[j].n_terms > 0 && (!obs[j].coeffs || !obs[j].x_mask || !obs[j].z_mask))
      return fail(SV_ERR_ARG, "observable %d: NULL term arrays", j);
    for (int t = 0; t < obs[j].n_terms; ++t) {
      c.push_back(grad_out[j] * obs[j].coeffs[t]);
      x.push_back(obs[j].x_mask[t]);
      z.push_back(obs[j].z_mask[t]);
    }
  }
  sv_pauli_sum merged = {(int32_t)c.size(), c.data(), x.data(), z.data()};
  return sv_adjoint_jacobian(s, tape, params, &merged, 1, nullptr, vjp_out);
}

sv_status sv_program_create(sv_state *s, const sv_tape *tape, const sv_pauli_sum *obs, int n_obs, sv_program **out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (sv_status st = check_state(s)) return st;
  if (!tape) return fail(SV_ERR_ARG, "tape is NULL");
  return build_program(s, tape, obs, n_obs, nullptr, false, out);
}

sv_status sv_program_destroy(sv_program *p) {
  if (!p) return SV_OK;
  cudaStreamSynchronize(p->s->stream);
  destroy_program(p);
  return SV_OK;
}

sv_status sv_program_set_params(sv_program *p, const double *params, int params_on_device) {
  if (!p) return fail(SV_ERR_ARG, "program is NULL");
  if (sv_status st = check_state(p->s)) return st;
  return program_set_params(p, params, params_on_device);
}

sv_status sv_program_forward(sv_program *p) {
  if (!p) return fail(SV_ERR_ARG, "program is NULL");
  if (sv_status st = check_state(p->s)) return st;
  if (sv_status st = require_params(p)) return st;
  p->launches = 0;
  if (sv_status st = run_steps_forward(p, p->s->psi)) return st;
  if (p->s->renorm) p->launches += 2;
  return finish_forward(p->s);
}

sv_status sv_program_jacobian(sv_program *p, double *expvals_out, double *jacobian_out, int outputs_on_device) {
  if (!p) return fail(SV_ERR_ARG, "program is NULL");
  if (sv_status st = check_state(p->s)) return st;
  if (sv_status st = require_params(p)) return st;
  if (p->m < 1) return fail(SV_ERR_ARG, "program has no observables");
  JacWs w;
  p->launches = 0;
  sv_status st = jac_workspace(p, w);
  if (!st) st = run_jacobian(p, w);
  if (!st) st = copy_out(p->s, expvals_out, w.expvals, p->m, outputs_on_device != 0);
  if (!st) st = copy_out(p->s, jacobian_out, w.J, (size_t)p->m * p->n_params, outputs_on_device != 0);
  if (!st && !outputs_on_device) st = sync_state(p->s);
  return st;
}

sv_status sv_program_expval(sv_program *p, double *expvals_out, int outputs_on_device) {
  if (!p) return fail(SV_ERR_ARG, "program is NULL");
  if (sv_status st = check_state(p->s)) return st;
  if (p->m < 1) return fail(SV_ERR_ARG, "program has no observables");
  if (!expvals_out) return fail(SV_ERR_ARG, "expvals_out is NULL");
  JacWs w;
  p->launches = 0;
  sv_status st = jac_workspace(p, w);
  if (!st) st = run_expval(p, p->s->psi, w);
  if (!st) st = copy_out(p->s, expvals_out, w.expvals, p->m, outputs_on_device != 0);
  if (!st && !outputs_on_device) st = sync_state(p->s);
  return st;
}

sv_status sv_program_vjp(sv_program *p, const double *grad_out, double *vjp_out, int outputs_on_device) {
  if (!p) return fail(SV_ERR_ARG, "program is NULL");
  if (sv_status st = check_state(p->s)) return st;
  if (sv_status st = require_params(p)) return st;
  if (p->m < 1) return fail(SV_ERR_ARG, "program has no observables");
  if (!grad_out || (p->n_params > 0 && !vjp_out)) return fail(SV_ERR_ARG, "NULL grad_out / vjp_out");
  for (int j = 0; j < p->m; ++j)
    if (!std::isfinite(grad_out[j])) return fail(SV_ERR_ARG, "grad_out[%d] is not finite", j);
  JacWs w;
  p->launches = 0;
  const int saved_mc = p->mc;
  p->mc = 1;  // one lambda: workspace of psi + phi + lambda
  sv_status st = jac_workspace(p, w);
  p->mc = saved_mc;
  if (!st) st = run_vjp(p, w, grad_out);
  if (!st) st = copy_out(p->s, vjp_out, w.J, (size_t)p->n_params, outputs_on_device != 0);
  if (!st && !outputs_on_device) st = sync_state(p->s);
  return st;
}

sv_status sv_program_jvp(sv_program *p, const double *tangent, double *jvp_out, int outputs_on_device) {
  if (!p) return fail(SV_ERR_ARG, "program is NULL");
  if (sv_status st = check_state(p->s)) return st;
  if (sv_status st = require_params(p)) return st;
  if (p->m < 1) return fail(SV_ERR_ARG, "the program has no observables");
  if (!jvp_out || (p->n_params > 0 && !tangent)) return fail(SV_ERR_ARG, "NULL tangent / jvp_out");
  for (int q = 0; q < p->n_params; ++q)
    if (!std::isfinite(tangent[q])) return fail(SV_ERR_ARG, "tangent[%d] is not finite", q);
  sv_state *s = p->s;
  JacWs w;
  p->launches = 0;
  p->want_tan = true;
  sv_status st = jac_workspace(p, w);
  p->want_tan = false;
  if (!st) st = run_jvp(p, w, tangent);
  if (!st) st = copy_out(s, jvp_out, w.J, p->m, outputs_on_device != 0);
  if (!st && !outputs_on_device) st = sync_state(s);
  return st;
}

sv_status sv_program_stats(const sv_program *p, int *n_forward_passes, int *n_adjoint_passes, int *launches_last_call) {
  if (!p) return fail(SV_ERR_ARG, "program is NULL");
  if (n_forward_passes) *n_forward_passes = (int)p->fwd.steps.size();
  if (n_adjoint_passes) *n_adjoint_passes = (int)p->adj.steps.size();
  if (launches_last_call) *launches_last_call = p->launches;
  return SV_OK;
}

sv_status sv_kernel_timing_enable(int enable) {
  g_timing = enable != 0;
  return SV_OK;
}

sv_status sv_kernel_timing_reset(void) {
  cudaError_t e = cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (TimedLaunch &t : g_pending) {
    g_event_pool.push_back(t.a);
    g_event_pool.push_back(t.b);
  }
  g_pending.clear();
  for (int c = 0; c < SV_KERNEL_CLASSES; ++c) {
    g_class_ms[c] = 0.0;
    g_class_n[c] = 0;
  }
  return e == cudaSuccess ? SV_OK : cuda_fail(e, "sv_kernel_timing_reset");
}

sv_status sv_kernel_timing_read(double *total_ms, int64_t *launches) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "sv_kernel_timing_read");
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (TimedLaunch &t : g_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      g_class_ms[t.cls] += ms;
      g_class_n[t.cls] += 1;
    }
    g_event_pool.push_back(t.a);
    g_event_pool.push_back(t.b);
  }
  g_pending.clear();
  for (int c = 0; c < SV_KERNEL_CLASSES; ++c) {
    if (total_ms) total_ms[c] = g_class_ms[c];
    if (launches) launches[c] = g_class_n[c];
  }
  return SV_OK;
}


sv_status sv_batch_create(sv_dtype dtype, int n_circuits, const int *n_qubits, const sv_tape *tapes,
                          const sv_pauli_sum *obs, const uint64_t *basis_states, sv_batch **out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  if (n_circuits < 1 || !n_qubits || !tapes || !obs) return fail(SV_ERR_ARG, "bad batch arguments");
  sv_batch *b = new sv_batch();
  b->dt = dtype;
  b->n_circ = n_circuits;
  for (int i = 0; i < n_circuits; ++i) {
    const int n = n_qubits[i];
    if (n < 1 || n > 30) {
      delete b;
      return fail(SV_ERR_ARG, "batch circuit %d: n = %d outside [1, 30]", i, n);
    }
    const sv_tape &t = tapes[i];
    if (t.n_ops < 0 || t.n_params < 0 || (t.n_ops > 0 && !t.ops)) {
      delete b;
      return fail(SV_ERR_ARG, "batch circuit %d: bad tape", i);
    }
    for (int k = 0; k < t.n_ops; ++k)
      if (sv_status st = validate_op(n, t.ops[k], t.n_params, t.matrices, t.n_matrix_entries, nullptr, false)) {
        delete b;
        g_err = "batch circuit " + std::to_string(i) + " op " + std::to_string(k) + ": " + g_err;
        return st;
      }
    b->nq.push_back(n);
    b->ops.emplace_back(t.ops, t.ops + t.n_ops);
    b->np.push_back(t.n_params);
    b->umat.emplace_back();
    if (t.matrices && t.n_matrix_entries > 0) b->umat.back().assign(t.matrices, t.matrices + 2 * t.n_matrix_entries);
    b->total_params += t.n_params;
    const sv_pauli_sum &H = obs[i];
    if (H.n_terms < 0 || (H.n_terms > 0 && (!H.coeffs || !H.x_mask || !H.z_mask))) {
      delete b;
      return fail(SV_ERR_ARG, "batch circuit %d: bad observable", i);
    }
    std::vector<ZTerm> zt;
    for (int k = 0; k < H.n_terms; ++k) {
      if (H.x_mask[k]) {
        delete b;
        return fail(SV_ERR_UNSUPPORTED, "batch circuit %d: observables must be Z-only Pauli words", i);
      }
      if ((H.z_mask[k] >> n) || !std::isfinite(H.coeffs[k])) {
        delete b;
        return fail(SV_ERR_ARG, "batch circuit %d: bad Z word", i);
      }
      zt.push_back({H.z_mask[k], H.coeffs[k]});
    }
    b->zterms_wire.push_back(zt);
    const uint64_t basis = basis_states ? basis_states[i] : 0;
    if (basis >> n) {
      delete b;
      return fail(SV_ERR_ARG, "batch circuit %d: basis state out of range", i);
    }
    b->basis.push_back(basis);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch stream");
  }
  b->own_stream = true;
  const Ops &K = ops_for(dtype);
  if (sv_status st = batch_plan(b, K.Tf, 64ll << 20)) {
    sv_batch_destroy(b);
    return st;
  }
  *out = b;
  return SV_OK;
}

sv_status sv_batch_destroy(sv_batch *b) {
  if (!b) return SV_OK;
  cudaStreamSynchronize(b->stream);
  batch_free_plan(b);
  dev_free(b->states, b->states_bytes);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return SV_OK;
}

sv_status sv_batch_set_stream(sv_batch *b, void *cuda_stream) {
  if (!b) return fail(SV_ERR_ARG, "batch is NULL");
  cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->use_graph = true;
  if (cuda_stream) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    b->own_stream = false;
    b->stream = (cudaStream_t)cuda_stream;
  } else if (!b->own_stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(SV_ERR_CUDA, "batch stream");
    b->own_stream = true;
  }
  return SV_OK;
}

sv_status sv_batch_set_params(sv_batch *b, const double *params, int params_on_device) {
  if (!b) return fail(SV_ERR_ARG, "batch is NULL");
  if (b->total_params > 0) {
    if (!params) return fail(SV_ERR_ARG, "params is NULL");
    if (!params_on_device)
      for (int i = 0; i < b->total_params; ++i)
        if (!std::isfinite(params[i])) return fail(SV_ERR_ARG, "parameter %d is not finite", i);
    cudaError_t e = cudaMemcpyAsync(b->d_params, params, (size_t)b->total_params * 8,
                                    params_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch parameters");
  }
  b->params_set = true;
  return SV_OK;
}

sv_status sv_batch_run(sv_batch *b, double *expvals_out, int outputs_on_device) {
  if (!b) return fail(SV_ERR_ARG, "batch is NULL");
  if (b->total_params > 0 && !b->params_set) return fail(SV_ERR_STATE, "batch parameters were never set");
  if (sv_status st = batch_launch(b)) return st;
  if (expvals_out) {
    cudaError_t e = cudaMemcpyAsync(expvals_out, b->d_out, (size_t)b->n_circ * 8,
                                    outputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch results");
  }
  return outputs_on_device ? SV_OK : batch_check(b);
}

sv_status sv_batch_status(sv_batch *b) {
  if (!b) return fail(SV_ERR_ARG, "batch is NULL");
  return batch_check(b);
}

sv_status sv_batch_autotune(sv_batch *b, double *best_ms) {
  if (!b) return fail(SV_ERR_ARG, "batch is NULL");
  if (b->total_params > 0 && !b->params_set) return fail(SV_ERR_STATE, "batch parameters were never set");
  const Ops &K = ops_for(b->dt);
  // parameters live in the table block: keep them across re-planning
  std::vector<double> params(std::max(b->total_params, 1));
  if (b->total_params > 0) {
    cudaError_t e = cudaMemcpyAsync(params.data(), b->d_params, (size_t)b->total_params * 8, cudaMemcpyDeviceToHost,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  int best_t = K.Tf, best_cap = 0;
  int64_t best_w = b->wave_bytes;
  const int64_t waves[4] = {16ll << 20, 32ll << 20, 64ll << 20, 128ll << 20};
  sv_status result = SV_OK;
  for (int t = K.Tf - 2; t <= K.Tf && !result; ++t) {
    for (int64_t w : waves)
    for (int cap : {0, 2}) {  // CTAs per SM: as many as fit, or two
      if (result) break;      // a failed configuration ends the search
      b->ctas_per_sm_cap = cap;
      if ((result = batch_plan(b, t, w))) break;
      if ((result = sv_batch_set_params(b, params.data(), 0))) break;
      b->use_graph = false;
      if ((result = batch_enqueue(b)) || (result = batch_check(b))) break;  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < 2 && !result; ++r) result = batch_enqueue(b);
      cudaEventRecord(e1, b->stream);
      if (!result) result = batch_check(b);
      if (result) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 2 < best) {
        best = ms / 2;
        best_t = t;
        best_w = w;
        best_cap = cap;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result) return result;
  b->ctas_per_sm_cap = best_cap;
  if (sv_status st = batch_plan(b, best_t, best_w)) return st;
  b->use_graph = true;
  if (sv_status st = sv_batch_set_params(b, params.data(), 0)) return st;
  if (best_ms) *best_ms = best;
  return SV_OK;
}

sv_status sv_batch_info(const sv_batch *b, int64_t *work_items, int *ctas, int *tile_bits, int64_t *wave_bytes,
                        int *graph) {
  if (!b) return fail(SV_ERR_ARG, "batch is NULL");
  if (work_items) *work_items = b->total_items;
  if (ctas) *ctas = b->grid;
  if (tile_bits) *tile_bits = b->max_T;
  if (wave_bytes) *wave_bytes = b->wave_bytes;
  if (graph) *graph = (b->exec != nullptr) ? 1 : 0;
  return SV_OK;
}

namespace {
sv_status plan_both(int n, sv_dtype dtype, const sv_tape *tape, Plan &f, Plan &a) {
  if (n < 1 || n > SV_MAX_QUBITS) return fail(SV_ERR_ARG, "n = %d outside [1, %d]", n, SV_MAX_QUBITS);
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  if (!tape || (tape->n_ops > 0 && !tape->ops)) return fail(SV_ERR_ARG, "bad tape");
  const Ops &K = ops_for(dtype);
  std::vector<HOp> fops, aops;
  for (int i = 0; i < tape->n_ops; ++i) {
    if (sv_status st = validate_op(n, tape->ops[i], tape->n_params, tape->matrices, tape->n_matrix_entries, nullptr,
                                   false))
      return st;
    HOp h = to_hop(tape->ops[i], tape->matrices);
    fops.push_back(h);
    expand_op(h, aops);
  }
  SlotTable st_tab;
  f = plan_passes(n, fops, K.Tf, K.nlow_pref, 1 << 30, false, st_tab, true, true, true);
  a = plan_passes(n, aops, K.Ta, K.nlow_pref, kMaxTrainPerPass, true, st_tab, true, true);
  if (sv_status st = check_plan(f, n, K.nlow_pref)) return st;
  return check_plan(a, n, K.nlow_pref);
}
}  // namespace

sv_status sv_plan_query(int n, sv_dtype dtype, const sv_tape *tape, int *n_forward_passes, int *n_adjoint_passes) {
  Plan f, a;
  if (sv_status st = plan_both(n, dtype, tape, f, a)) return st;
  if (n_forward_passes) *n_forward_passes = (int)f.steps.size();
  if (n_adjoint_passes) *n_adjoint_passes = (int)a.steps.size();
  return SV_OK;
}

// Pauli words of a Hermitian matrix on k wires.  Local index j of the matrix
// has wires[0] as its most significant bit; a word with local flip mask x, sign
// mask z and nY = popcount(x & z) acts as P|j> = i^nY (-1)^popcount(j & z) |j ^ x>,
// so Tr(P A) = i^nY sum_j (-1)^popcount(j & z) A[j][j ^ x] and A = sum_P c_P P
// with c_P = Tr(P A) / 2^k (the Pauli matrices are an orthogonal basis under
// the trace inner product).
sv_status sv_hermitian_to_pauli(int n, const int *wires, int k, const double *matrix, double tol, double *coeffs,
                                uint64_t *x_masks, uint64_t *z_masks, int *n_terms) {
  if (n < 1 || n > 63) return fail(SV_ERR_ARG, "n = %d out of range 1..63", n);
  if (k < 1 || k > SV_MAX_HERMITIAN_WIRES)
    return fail(SV_ERR_ARG, "a Hermitian observable takes 1..%d wires, got %d", SV_MAX_HERMITIAN_WIRES, k);
  if (!wires || !matrix || !coeffs || !x_masks || !z_masks || !n_terms) return fail(SV_ERR_ARG, "NULL argument");
  if (!(tol >= 0.0)) return fail(SV_ERR_ARG, "tol must be >= 0");
  for (int j = 0; j < k; ++j) {
    if (wires[j] < 0 || wires[j] >= n) return fail(SV_ERR_ARG, "wire %d out of range for %d qubits", wires[j], n);
    for (int i = 0; i < j; ++i)
      if (wires[i] == wires[j]) return fail(SV_ERR_ARG, "wire %d used twice", wires[j]);
  }
  const int D = 1 << k;
  double amax = 0.0;
  for (int e = 0; e < 2 * D * D; ++e) {
    if (!std::isfinite(matrix[e])) return fail(SV_ERR_ARG, "matrix entry %d is not finite", e / 2);
    amax = std::max(amax, std::fabs(matrix[e]));
  }
  for (int r = 0; r < D; ++r)
    for (int c = 0; c <= r; ++c) {
      const double *a = matrix + 2 * (r * D + c), *b = matrix + 2 * (c * D + r);
      if (std::fabs(a[0] - b[0]) > 1e-12 * std::max(1.0, amax) || std::fabs(a[1] + b[1]) > 1e-12 * std::max(1.0, amax))
        return fail(SV_ERR_ARG, "matrix is not Hermitian (entries (%d,%d) and (%d,%d))", r, c, c, r);
    }
  int cnt = 0;
  for (int x = 0; x < D; ++x)
    for (int z = 0; z < D; ++z) {
      double re = 0.0, im = 0.0;  // sum_j (-1)^popcount(j & z) A[j][j ^ x]
      for (int j = 0; j < D; ++j) {
        const double *a = matrix + 2 * (j * D + (j ^ x));
        const double sg = (popc((uint64_t)(j & z)) & 1) ? -1.0 : 1.0;
        re += sg * a[0];
        im += sg * a[1];
      }
      // times i^nY: the real part of the (real) coefficient
      double c;
      switch (popc((uint64_t)(x & z)) & 3) {
        case 0: c = re; break;
        case 1: c = -im; break;
        case 2: c = -re; break;
        default: c = im; break;
      }
      c /= (double)D;
      if (std::fabs(c) <= tol) continue;
      uint64_t xm = 0, zm = 0;
      for (int j = 0; j < k; ++j) {
        const int bit = k - 1 - j;  // local bit of wires[j]
        if ((x >> bit) & 1) xm |= 1ull << wires[j];
        if ((z >> bit) & 1) zm |= 1ull << wires[j];
      }
      coeffs[cnt] = c;
      x_masks[cnt] = xm;
      z_masks[cnt] = zm;
      ++cnt;
    }
  *n_terms = cnt;
  return SV_OK;
}

sv_status sv_plan_describe(int n, sv_dtype dtype, const sv_tape *tape, int forward_counts[SV_PLAN_KINDS],
                           int adjoint_counts[SV_PLAN_KINDS]) {
  Plan f, a;
  if (sv_status st = plan_both(n, dtype, tape, f, a)) return st;
  auto count = [](const Plan &P, int *out) {
    if (!out) return;
    for (int k = 0; k < SV_PLAN_KINDS; ++k) out[k] = 0;
    for (const OpDev &o : P.ops) {
      if (o.kind == kPair) out[o.fused ? 4 : 0]++;
      else if (o.kind == kDiag) out[1]++;
      else if (o.kind == kDense) out[2]++;
      else if (o.kind == kPhase) out[3]++;
      else if (o.kind == kMulti) out[5]++;
    }
    out[6] = (int)P.dk_ops.size();
    out[7] = (int)P.passes.size();
  };
  count(f, forward_counts);
  count(a, adjoint_counts);
  return SV_OK;
}

}  // extern "C"

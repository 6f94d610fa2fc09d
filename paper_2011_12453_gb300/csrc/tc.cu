// Tensor-core path: BF16 node-feature GEMMs on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), for the GCN forward and the incremental
// local energy of arXiv:2011.12453 (Eq. gcn; local energy of the scaling section).
//
// One CTA owns one configuration at a time (persistent grid).  Per GCN layer, the rows
// to recompute are gathered into BF16 A tiles of 128 rows x 2F in shared memory, laid
// out in the no-swizzle K-major canonical form the MMA reads: element (r, k) of a tile at
// (r/8)*SBO + (k/8)*128 + (r%8)*16 + (k%8)*2 bytes, SBO = 32F.  B = W^T (F x 2F) uses the
// same form.  One elected thread issues 2F/16 MMAs of M=128, N=F, K=16 per tile into a
// TMEM accumulator (column offset tile*F) and commits them to an mbarrier; all warps
// then read the accumulator with tcgen05.ld (warp w sees lanes 32*(w%4)..+31; the
// 8-column chunks are spread over the four warp groups), add the bias, apply tanh and
// store the new rows.  Feature rows are stored with padded strides (F + 8 BF16, F + 4
// FP32) so that lanes reading rows of different sites do not share banks.
//
// Storage: cached layers H^0..H^{L-1} are BF16, as the GEMM consumes them; for every FP32
// pre-activation Y^1..Y^L the incremental step keeps copysign(exp(-2|Y|), Y).
//
// Incremental ratios propagate differences instead of recomputing rows.  Exchanging
// s_i and s_j changes layer 0 by dH^0 (rows i and j only).  With X = [A_hat H ; H] and
// Y = X W + b, layer l changes by dY = [A_hat dH ; dH] W (the bias cancels), nonzero only
// on ball_l(e), and dH^l = tanh(Y + dY) - tanh(Y) = t (1 - H^2) / (1 + H t) with
// t = tanh(dY) (the addition formula of tanh), H the cached row.  The GEMM operands are
// then the small differences themselves, so BF16 rounding is relative to dH rather than
// to H, and Delta log Psi = w_r[:F] . sum_v dH^L_v accumulates in FP32.  Bond groups
// stack the rows of several antiparallel bonds at the same layer into the same tiles.
//
// Every wait on the mbarrier is bounded: on timeout the kernel records bit 1 in its
// status word, waits (bounded again) for the MMAs in flight, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <atomic>
#include <climits>
#include <cstring>

#include "tc.cuh"

namespace gna {

static __device__ int s_tc_status;

constexpr int kTcThreads = 512;
constexpr int kTcMaxUnits = 4;  // independent units (2 of 256 or 4 of 128 threads) for bond groups
constexpr int kTmemCols = 256;
constexpr uint32_t kWaitLimit = 1u << 26;            // try_wait iterations
constexpr uint64_t kWaitNs = 2000000000ull;          // and at most 2 s of wall time

// ---------------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// limit: try_wait iterations (a launch argument; kWaitLimit unless a test shortens it --
// with 0 the wait gives up at once, which exercises the timeout path without a fault)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
  if (limit > 0 && mbar_try_wait(bar, parity)) return true;  // the usual case, before reading the timer
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulation, M = 128, N = F.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 lanes x 8 columns of FP32 from TMEM; thread i of the warp gets lane (base + i).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4);
  v[5] = __uint_as_float(r5);
  v[6] = __uint_as_float(r6);
  v[7] = __uint_as_float(r7);
}
// Two 8-column loads for the same 32 lanes, one wait.
__device__ __forceinline__ void tmem_ld8x2(uint32_t ta, uint32_t tb, float* va, float* vb) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    va[i] = __uint_as_float(r[i]);
    vb[i] = __uint_as_float(r[8 + i]);
  }
}
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Pairs of float32 in one 64-bit register, for the f32x2 arithmetic of sm_100 and later
// (one instruction does both halves).
__device__ __forceinline__ uint64_t pk2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Common case of the tanh difference for two units: e = exp(-2|Y|), s = a value with the
// sign of Y, t = tanh(dY); returns d = 4 e t / ((1 + e)((1 + e) + sgn(Y)(1 - e) t)) for
// both and the two denominators, in f32x2 arithmetic (used by the local energy; in the
// sampler, whose registers are fuller, the packed form spilled and was slower).
__device__ __forceinline__ void delta_tanh_pair(float e0, float e1, float s0, float s1, float t0, float t1,
                                                float& d0, float& d1, float& den0, float& den1) {
  const uint64_t E = pk2(e0, e1), T = pk2(t0, t1);
  const uint64_t ope = add2(E, pk2(1.f, 1.f));
  const uint64_t g = pk2(copysignf(1.f - e0, s0), copysignf(1.f - e1, s1));
  const uint64_t den = mul2(ope, fma2(g, T, ope));
  upk2(den, den0, den1);
  float r0, r1;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r0) : "f"(den0));
  asm("rcp.approx.f32 %0, %1;" : "=f"(r1) : "f"(den1));
  const uint64_t r4 = mul2(pk2(r0, r1), pk2(4.f, 4.f));
  upk2(mul2(mul2(E, T), r4), d0, d1);
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t M, uint32_t N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// The incremental step needs, per cached unit, only sgn(Y) and e = exp(-2|Y|): they are
// stored together as copysign(e, Y).
__device__ __forceinline__ float sexp(float y) { return copysignf(__expf(-2.f * fabsf(y)), y); }

__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------
// layout (computed on the host, passed in the arguments)
// ---------------------------------------------------------------------------------
struct TcLayout {
  // shared memory byte offsets
  uint32_t oWt, obias, oemb, owr, obr, oA, ospin, oint, odbl, obar, oslot, oregion, smem_total;
  uint32_t orp, owf, orow, opos;  // CSR row starts and weights; per-unit staged rows / positions
  uint32_t row_unit, pos_unit;    // staged rows (int) / neighbour positions (int16) per unit
  // region (shared or global) byte offsets
  uint64_t rcache16, rY, rnew16, rpart, region_bytes;
  int y_global;                   // 1: the Y cache in the workspace (y_bytes per CTA), not in the region
  uint64_t y_bytes;
  uint64_t new16_off[kMaxL + 1];  // per layer l < L: offset of the group's dH rows (bytes from rnew16)
  int T;                          // A tiles per unit (TMEM holds T accumulators of F columns per unit)
  int split;                      // 1: operands as hi + lo BF16 pairs, FP32 feature rows
  uint32_t lo_off;                // split: bytes from a unit's hi tiles to its lo tiles
  int units;                      // bond-group units per CTA
  int G;                          // bonds per group (per unit)
  uint32_t a_unit;                // bytes of one unit's A tiles
  uint32_t int_unit, dbl_unit;    // per-unit slices of the int / double scratch (elements)
  uint64_t new16_unit, part_unit; // per-unit slices of the dH rows and Delta partials (bytes)
  int part_rows;                  // rows of each warp group's Delta partials (>= G * maxball[L])
  uint64_t rstate, state_unit;    // sampler only: per-unit chain-pool state (bytes)
};

struct TcArgs {
  DevGraph g;
  Dims m;
  int op;
  TcLayout lay;
  int maxball[kMaxL + 1];
  const float* theta;
  const int8_t* spins;
  int64_t B;
  double* logpsi;
  double* eloc;
  float* dlogpsi;
  unsigned char* gregion;  // [grid][region_bytes] when the region is not in shared memory
  float* gY;               // [grid][y_bytes] when lay.y_global
  float* gH;               // [grid][N][ldy]: H^L of the local-energy call's forward, when it writes log Psi
  int region_in_smem;
  uint32_t wait_limit;     // try_wait iterations of the MMA waits (teardown waits keep kWaitLimit)
};

// Local energy and forward: BF16 operands four 128-thread units (more independent rounds
// in flight per SM), split operands two 256-thread units (their A tiles and FP32 dH rows are
// twice as large; four units leave room for only small bond groups).  Kagome 108, F = 32,
// 16384 configurations: BF16 four units 24.1 ms, two 26.0 ms; BF16X2 two units 33.7 ms,
// four 45.5 ms.  The sampler takes four units from F = 32 on (two units 31.3 ms per sweep,
// four 26.9 ms).  One 128-row tile per unit and pass: the shared memory goes to larger bond
// groups instead (two tiles per unit: BF16 24.4 ms, BF16X2 40.1 ms).
__host__ inline int tc_units(int F, int split = 0) { return split ? 2 : 4; }
__host__ inline int tcm_units(int F) { return F <= 16 ? 2 : 4; }
__host__ inline int tc_tiles_per_unit(int) { return 1; }

// Passes of rows_per_pass rows that a group of G bonds needs over layers 1..L, per bond
// (x1000): the cost model for the group size (the last pass of each layer is partial).
__host__ inline int tc_passes_per_bond(const int* maxball, int L, int G, int rows_per_pass) {
  int passes = 0;
  for (int l = 1; l <= L; ++l) passes += (G * maxball[l] + rows_per_pass - 1) / rows_per_pass;
  return passes * 1000 / G;
}

// The staged tables of a unit: G bonds' rows of ball_L (packed vertex and entry start) and
// their in-ball neighbour positions (maxspan = max entries of a bond's ball_L).
__host__ inline void tc_stage_layout(const Dims& m, const int* maxball, int maxspan, int G, int U,
                                     uint64_t& o, TcLayout* t) {
  auto take = [&](uint64_t bytes, uint64_t align) {
    o = (o + align - 1) / align * align;
    uint64_t r = o;
    o += bytes;
    return (uint32_t)r;
  };
  t->orp = take((uint64_t)(m.N + 1) * 4, 16);
  t->owf = take((uint64_t)2 * m.E * 4, 16);
  t->row_unit = (uint32_t)(G * maxball[m.L]);
  t->orow = take((uint64_t)U * t->row_unit * 4, 16);
  t->pos_unit = (uint32_t)((G * maxspan + 7) / 8 * 8);
  t->opos = take((uint64_t)U * t->pos_unit * 2, 16);
}

// alias_new16: the group rows' dH layers share the space of the BF16 layer cache, which
// only the forward reads (the incremental step needs the pre-activations alone).
__host__ inline bool tc_layout(const Dims& m, const int* maxball, int maxspan, int G, int region_in_smem,
                               int alias_new16, TcLayout* t, int split = 0, int y_global = 0) {
  const int F = m.F, N = m.N, L = m.L;
  uint64_t o = 0;
  auto take = [&](uint64_t bytes, uint64_t align) {
    o = (o + align - 1) / align * align;
    uint64_t r = o;
    o += bytes;
    return (uint32_t)r;
  };
  t->T = tc_tiles_per_unit(F);
  t->units = tc_units(F, split);
  t->split = split;
  const int U = t->units;
  t->G = G;
  t->lo_off = (uint32_t)t->T * 128 * 2 * F * 2;
  t->a_unit = t->lo_off * (split ? 2 : 1);
  t->oWt = take((uint64_t)F * 2 * F * 2, 1024);
  t->oA = take((uint64_t)U * t->a_unit, 1024);
  t->obias = take(F * 4, 16);
  t->oemb = take(2 * F * 4, 16);
  t->owr = take((F + 2) * 2 * 4, 16);
  t->obr = take(16, 16);
  t->ospin = take(N, 16);
  t->int_unit = (uint32_t)(3 * G + (L + 2) * (G + 1) + 4);
  t->oint = take(((uint64_t)m.E + 16 + (uint64_t)U * t->int_unit) * 4, 16);
  t->dbl_unit = (uint32_t)(3 * G + 64 + 4);  // Delta [2G], couplings [G], lane sums [2 x 32]
  t->odbl = take((uint64_t)(16 + kTcThreads + U * t->dbl_unit) * 8, 16);
  t->obar = take(8 * U, 8);
  t->oslot = take(4, 4);
  tc_stage_layout(m, maxball, maxspan, G, U, o, t);
  // region
  uint64_t r = 0;
  auto rtake = [&](uint64_t bytes) {
    r = (r + 15) / 16 * 16;
    uint64_t x = r;
    r += bytes;
    return x;
  };
  const uint64_t ldh = F + 8, ldy = F + 4;  // padded row strides (BF16 rows, FP32 rows)
  // feature rows of the layer cache and of the dH rows: BF16, or FP32 when split
  const uint64_t row_bytes = split ? ldy * 4 : ldh * 2;
  // Y^1..Y^L (FP32; the forward-only call keeps H^L there): in the region, or in the
  // workspace (L2-resident) when that lets more bonds share a group
  t->y_global = y_global;
  t->y_bytes = ((uint64_t)L * N * ldy * 4 + 255) / 256 * 256;
  t->rY = y_global ? 0 : rtake((uint64_t)L * N * ldy * 4);
  uint64_t n16 = 0;
  for (int l = 0; l < L; ++l) {
    t->new16_off[l] = n16;
    n16 += (uint64_t)G * maxball[l] * row_bytes;
  }
  t->new16_unit = (n16 + 15) / 16 * 16;
  const uint64_t cache_bytes = (uint64_t)L * N * row_bytes, new_bytes = (uint64_t)U * t->new16_unit;
  if (alias_new16) {
    // one area for both: the layer cache during the forward, the dH rows afterwards
    t->rcache16 = rtake(cache_bytes > new_bytes ? cache_bytes : new_bytes);
    t->rnew16 = t->rcache16;
  } else {
    t->rcache16 = rtake(cache_bytes);
    t->rnew16 = rtake(new_bytes);
  }
  t->part_rows = G * maxball[L];
  t->part_unit = (uint64_t)(kTcThreads / U / 128) * t->part_rows * 2 * 4;  // [warp group][row][Re, Im]
  t->rpart = rtake((uint64_t)U * t->part_unit);
  t->region_bytes = (r + 255) / 256 * 256;
  if (region_in_smem) {
    t->oregion = take(t->region_bytes, 16);
  } else {
    t->oregion = 0;
  }
  t->smem_total = (uint32_t)o;
  return true;
}

// ---------------------------------------------------------------------------------
// device pieces
// ---------------------------------------------------------------------------------
struct TcCtx {
  const TcArgs* a;
  int N, F, L, E, T, G;
  int ldh, ldy;  // row strides: BF16 feature rows, FP32 pre-activation rows
  __nv_bfloat16* Wt;
  float *bias, *emb, *wr, *br;
  int8_t* spin;
  const int* rp;     // CSR row starts [N+1] (shared memory)
  const float* wfs;  // CSR weights [2E] (shared memory)
  int* list;     // antiparallel bonds of the configuration
  double* sdbl;  // shared double scratch (readout)
  unsigned char* region;
  float* ycache; // Y^1..Y^L of the configuration (region or workspace)
  float* hL;     // H^L for the readout of the local-energy call's forward (workspace), or NULL
  int* fail;     // shared flag
};

// A group of threads that runs gather -> MMA -> epilogue rounds on its own A tiles, TMEM
// columns and mbarrier: the whole CTA (forward), or one of the units that take
// alternate bond groups so that one unit's waits overlap the other's work.
struct Unit {
  int tid, nthr, bar_id, nwg;  // thread index in the unit, its size, named barrier (0: whole CTA), warp groups
  unsigned char* A;
  uint32_t tbase;
  uint64_t* bar;
  uint32_t phase;              // meaningful in the unit's thread 0 (the waiter)
  __nv_bfloat16* d16;          // this unit's dH rows
  float* part;                 // this unit's Delta partials [nwg][T*128][2]
  int* slot_e;                 // [G]
  int* soff;                   // [(L+1)][G+1]
  int* eoff;                   // [G+1] start of each bond's staged neighbour positions, then
                               // [G] + [G] each bond's start in row_pack and in nbr_pos16
  int* srow;                   // staged row_pack of the group's bonds (bond k at soff[L][k])
  int16_t* spos;               // staged nbr_pos16 of the group's bonds (bond k at eoff[k])
  double* res;                 // [2G] Delta of each bond of the group
};

__device__ __forceinline__ void unit_sync(const Unit& u) {
  if (u.bar_id == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(u.bar_id), "r"(u.nthr) : "memory");
}

// Slot of group row q at layer l (offsets offl[0..nb]).
// Branch-free binary search for the largest k < nb with offl[k] <= q (offl strictly
// increasing, offl[0] = 0 <= q; nb <= 16).
__device__ __forceinline__ int slot_of(const int* offl, int nb, int q) {
  int k = 0;
#pragma unroll
  for (int step = 8; step >= 1; step >>= 1) {
    const int j = k + step;
    if (j < nb && offl[j] <= q) k = j;
  }
  return k;
}

// Offsets of the group's rows per layer (soff) and of its bonds' staged entries (eoff),
// then the bonds' rows and in-ball neighbour positions into shared memory, so that the
// passes of the group look them up without global-memory latency.  Every step is one
// parallel loop (the group's G <= 16 bonds are the lanes of one warp in the prefix sums), so
// the staging costs a few global-load latencies, not one per bond.
// Jout (when not null): each bond's coupling, loaded in the same round.  NL: loads in flight
// per thread in the copies.
template <int NL>
__device__ void stage_group(const DevGraph& g, const Unit& u, int L, int G, int nb, double* Jout = nullptr) {
  const int Lm = g.Lmax;
  int* rbase = u.eoff + G + 1;
  int* ebase = rbase + G;
  // sizes into the offset arrays (shifted by one) and each bond's table starts ...
  for (int i = u.tid; i < (L + 3 + (Jout ? 1 : 0)) * nb; i += u.nthr) {
    const int l = i / nb, k = i - l * nb;
    const int e = u.slot_e[k];
    const size_t eo = (size_t)e * (Lm + 1);
    if (l <= L) {
      u.soff[l * (G + 1) + k + 1] = __ldg(g.ball_size + eo + l);
    } else if (l == L + 1) {
      u.eoff[k + 1] = __ldg(g.ball_span + eo + L);
    } else if (l == L + 2) {
      rbase[k] = __ldg(g.ball_off + e);
      ebase[k] = __ldg(g.bond_ent + e);
    } else {
      Jout[k] = __ldg(g.J + e);
    }
  }
  unit_sync(u);
  // ... then inclusive prefix sums, one warp per array, lane k holding bond k
  const int warp = u.tid >> 5, lane = u.tid & 31, nwarps = u.nthr >> 5;
  for (int w = warp; w <= L + 1; w += nwarps) {
    int* row = w <= L ? u.soff + w * (G + 1) : u.eoff;
    int x = lane < nb ? row[lane + 1] : 0;
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane < nb) row[lane + 1] = x;
    if (lane == 0) row[0] = 0;
  }
  unit_sync(u);
  // ... then the rows and positions of all bonds in one loop each
  // (NL loads in flight per thread before their stores)
  const int* offL = u.soff + L * (G + 1);
  const int nr = offL[nb], ne = u.eoff[nb];
  for (int i0 = u.tid; i0 < nr; i0 += NL * u.nthr) {
    int v[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int i = i0 + j * u.nthr;
      if (i < nr) {
        const int k = slot_of(offL, nb, i);
        v[j] = __ldg(g.row_pack + rbase[k] + (i - offL[k]));
      }
    }
#pragma unroll
    for (int j = 0; j < NL; ++j)
      if (i0 + j * u.nthr < nr) u.srow[i0 + j * u.nthr] = v[j];
  }
  for (int i0 = u.tid; i0 < ne; i0 += NL * u.nthr) {
    int16_t v[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const int i = i0 + j * u.nthr;
      if (i < ne) {
        const int k = slot_of(u.eoff, nb, i);
        v[j] = __ldg(g.nbr_pos16 + ebase[k] + (i - u.eoff[k]));
      }
    }
#pragma unroll
    for (int j = 0; j < NL; ++j)
      if (i0 + j * u.nthr < ne) u.spos[i0 + j * u.nthr] = v[j];
  }
}

__device__ __forceinline__ unsigned char* a_row_chunk(const Unit& u, int F, int q, int chunk) {
  // 16-byte chunk `chunk` (k = 8*chunk .. 8*chunk+7) of row q of the unit's stacked A tiles
  const int tile = q >> 7, qq = q & 127;
  return u.A + (size_t)tile * 128 * 4 * F + (size_t)(qq >> 3) * (32 * F) + chunk * 128 + (qq & 7) * 16;
}

__device__ __forceinline__ const __nv_bfloat16* cache16(const TcCtx& c, int l) {
  return (const __nv_bfloat16*)(c.region + c.a->lay.rcache16) + (size_t)l * c.N * c.ldh;
}
__device__ __forceinline__ __nv_bfloat16* cache16w(const TcCtx& c, int l) {
  return (__nv_bfloat16*)(c.region + c.a->lay.rcache16) + (size_t)l * c.N * c.ldh;
}
// Per site and layer l = 1..L: copysign(exp(-2|Y^l|), Y^l) for the incremental step (Y^l
// the FP32 pre-activation); for the forward-only call the last slot holds H^L instead.
__device__ __forceinline__ float* cacheY(const TcCtx& c, int l) {
  return c.ycache + (size_t)(l - 1) * c.N * c.ldy;
}
__device__ __forceinline__ __nv_bfloat16* new16(const TcCtx& c, const Unit& u, int l) {
  return (__nv_bfloat16*)((unsigned char*)u.d16 + c.a->lay.new16_off[l]);
}
// split mode: the same caches with FP32 rows of stride ldy
__device__ __forceinline__ float* cache32w(const TcCtx& c, int l) {
  return (float*)(c.region + c.a->lay.rcache16) + (size_t)l * c.N * c.ldy;
}
__device__ __forceinline__ float* new32(const TcCtx& c, const Unit& u, int l) {
  return (float*)((unsigned char*)u.d16 + c.a->lay.new16_off[l]);
}

// acc2[0..4) (pairs of float32) += w * bf16 row chunk at p (16 bytes), f32x2 arithmetic
__device__ __forceinline__ void fma_chunk2(uint64_t* acc2, uint64_t w2, const __nv_bfloat16* p) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  acc2[0] = fma2(pk2(bf16lo(u.x), bf16hi(u.x)), w2, acc2[0]);
  acc2[1] = fma2(pk2(bf16lo(u.y), bf16hi(u.y)), w2, acc2[1]);
  acc2[2] = fma2(pk2(bf16lo(u.z), bf16hi(u.z)), w2, acc2[2]);
  acc2[3] = fma2(pk2(bf16lo(u.w), bf16hi(u.w)), w2, acc2[3]);
}

// acc[0..8) += w * bf16 row chunk at p (16 bytes)
__device__ __forceinline__ void fma_chunk(float* acc, float w, const __nv_bfloat16* p) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  acc[0] += w * bf16lo(u.x);
  acc[1] += w * bf16hi(u.x);
  acc[2] += w * bf16lo(u.y);
  acc[3] += w * bf16hi(u.y);
  acc[4] += w * bf16lo(u.z);
  acc[5] += w * bf16hi(u.z);
  acc[6] += w * bf16lo(u.w);
  acc[7] += w * bf16hi(u.w);
}

// 8 FP32 values as hi = bf16(x) and lo = bf16(x - hi), packed two per 32-bit word.
__device__ __forceinline__ void split_hi_lo(const float* x, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * p], x[2 * p + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * p] - hf.x, x[2 * p + 1] - hf.y);
    h[p] = *reinterpret_cast<const uint32_t*>(&hb);
    l[p] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}
// one element as hi and lo BF16
__device__ __forceinline__ void split1(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// acc[0..8) += w * FP32 row chunk at p (two 16-byte loads)
__device__ __forceinline__ void fma_chunk32(float* acc, float w, const float* p) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  acc[0] = fmaf(w, a.x, acc[0]);
  acc[1] = fmaf(w, a.y, acc[1]);
  acc[2] = fmaf(w, a.z, acc[2]);
  acc[3] = fmaf(w, a.w, acc[3]);
  acc[4] = fmaf(w, b.x, acc[4]);
  acc[5] = fmaf(w, b.y, acc[5]);
  acc[6] = fmaf(w, b.z, acc[6]);
  acc[7] = fmaf(w, b.w, acc[7]);
}

// tanh(x) - x for |x| < 0.5: x^3 times the Taylor series of tanh from its x^3 term on
// (coefficients 2^2n (2^2n - 1) B_2n / (2n)!, B_2n the Bernoulli numbers), through x^15;
// the truncation is below 1e-7 of tanh(x) at |x| = 0.5.
__device__ __forceinline__ float tanh_minus_x(float x) {
  const float x2 = x * x;
  float p = -929569.f / 638512875.f;
  p = fmaf(p, x2, 21844.f / 6081075.f);
  p = fmaf(p, x2, -1382.f / 155925.f);
  p = fmaf(p, x2, 62.f / 2835.f);
  p = fmaf(p, x2, -17.f / 315.f);
  p = fmaf(p, x2, 2.f / 15.f);
  p = fmaf(p, x2, -1.f / 3.f);
  return p * x2 * x;
}

// Issue the MMAs of nt tiles (unit thread 0), commit, and wait (bounded).  Returns false on
// timeout (uniform across the unit).  S: each tile's lo part (at lo_off) is multiplied into
// the same accumulator after its hi part.
template <bool S>
__device__ bool run_mmas(const TcCtx& c, Unit& u, int nt) {
  fence_proxy_async();
  unit_sync(u);
  if (u.tid == 0) {
    tc_fence_after();
    const int F = c.F;
    const uint32_t idesc = idesc_bf16(128, F);
    const uint32_t sbo = 32 * F;
    const uint32_t a0 = smem_u32(u.A), b0 = smem_u32(c.Wt);
    for (int t = 0; t < nt; ++t) {
      for (int kb = 0; kb < (2 * F) / 16; ++kb) {
        const uint64_t ad = sdesc(a0 + t * 128 * 4 * F + kb * 256, 128, sbo);
        const uint64_t bd = sdesc(b0 + kb * 256, 128, sbo);
        mma_bf16(u.tbase + t * F, ad, bd, idesc, kb > 0 ? 1u : 0u);
      }
      if (S) {
        const uint32_t alo = a0 + c.a->lay.lo_off;
        for (int kb = 0; kb < (2 * F) / 16; ++kb) {
          const uint64_t ad = sdesc(alo + t * 128 * 4 * F + kb * 256, 128, sbo);
          const uint64_t bd = sdesc(b0 + kb * 256, 128, sbo);
          mma_bf16(u.tbase + t * F, ad, bd, idesc, 1u);
        }
      }
    }
    mma_commit(u.bar);
    const bool ok = mbar_wait_bounded(u.bar, u.phase, c.a->wait_limit);
    if (!ok) {
      *c.fail = 1;
      atomicOr(&s_tc_status, 1);
    }
    u.phase ^= 1u;
  }
  unit_sync(u);
  tc_fence_after();
  return *c.fail == 0;
}

// Forward epilogue for rows [r0, r0 + R) of layer l: Y = acc + b.  l < L: H^l = tanh(Y)
// stored BF16 (and Y in FP32 when the call needs the incremental step).  l == L: Y^L in
// FP32, or, for the forward-only call, H^L = tanh(Y^L) in FP32 for the readout.
// S: H^l (l < L) stored in FP32 with an accurate tanh.
template <bool S>
__device__ void epilogue_fwd(const TcCtx& c, const Unit& u, int nt, int R, int r0, int l, bool keep_y) {
  const int warp = u.tid >> 5, lane = u.tid & 31;
  const int q4 = warp & 3, wg = warp >> 2;
  const int F = c.F, L = c.L, ldh = c.ldh, ldy = c.ldy;
  __nv_bfloat16* h16 = l < L && !S ? cache16w(c, l) + (size_t)r0 * ldh : nullptr;
  float* h32 = l < L && S ? cache32w(c, l) + (size_t)r0 * ldy : nullptr;
  float* y32 = cacheY(c, l) + (size_t)r0 * ldy;
  for (int t = 0; t < nt; ++t) {
    const int q = t * 128 + q4 * 32 + lane;
    for (int ch = wg; ch < F / 8; ch += u.nwg) {
      const int col = ch * 8;
      float v[8];
      tmem_ld8(u.tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(t * F + col), v);
      if (q < R) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] += c.bias[col + i];
        float4* yo = reinterpret_cast<float4*>(y32 + (size_t)q * ldy + col);
        if (l < L) {
          if (keep_y) {
            yo[0] = make_float4(sexp(v[0]), sexp(v[1]), sexp(v[2]), sexp(v[3]));
            yo[1] = make_float4(sexp(v[4]), sexp(v[5]), sexp(v[6]), sexp(v[7]));
          }
          if (S) {
            float4* ho = reinterpret_cast<float4*>(h32 + (size_t)q * ldy + col);
            ho[0] = make_float4(tanhf(v[0]), tanhf(v[1]), tanhf(v[2]), tanhf(v[3]));
            ho[1] = make_float4(tanhf(v[4]), tanhf(v[5]), tanhf(v[6]), tanhf(v[7]));
          } else {
            uint4 w;
            w.x = pack_bf16(tanh_fast(v[0]), tanh_fast(v[1]));
            w.y = pack_bf16(tanh_fast(v[2]), tanh_fast(v[3]));
            w.z = pack_bf16(tanh_fast(v[4]), tanh_fast(v[5]));
            w.w = pack_bf16(tanh_fast(v[6]), tanh_fast(v[7]));
            *reinterpret_cast<uint4*>(h16 + (size_t)q * ldh + col) = w;
          }
        } else if (keep_y) {
          yo[0] = make_float4(sexp(v[0]), sexp(v[1]), sexp(v[2]), sexp(v[3]));
          yo[1] = make_float4(sexp(v[4]), sexp(v[5]), sexp(v[6]), sexp(v[7]));
          if (c.hL) {  // H^L as the forward-only call stores it, for the same readout
            float4* ho = reinterpret_cast<float4*>(c.hL + (size_t)(r0 + q) * ldy + col);
            ho[0] = make_float4(tanhf(v[0]), tanhf(v[1]), tanhf(v[2]), tanhf(v[3]));
            ho[1] = make_float4(tanhf(v[4]), tanhf(v[5]), tanhf(v[6]), tanhf(v[7]));
          }
        } else {
          yo[0] = make_float4(tanhf(v[0]), tanhf(v[1]), tanhf(v[2]), tanhf(v[3]));
          yo[1] = make_float4(tanhf(v[4]), tanhf(v[5]), tanhf(v[6]), tanhf(v[7]));
        }
      }
    }
  }
  tc_fence_before();
  unit_sync(u);
}

// Forward of the configuration in c.spin (unit = whole CTA): fills the cache.  S: the layer
// cache in FP32 and X = [A_hat H ; H] as hi + lo tiles.
template <bool S>
__device__ bool tc_forward(const TcCtx& c, Unit& u) {
  const int N = c.N, F = c.F, L = c.L, ldh = c.ldh, ldy = c.ldy;
  const DevGraph& g = c.a->g;
  if (S) {
    float* c0 = cache32w(c, 0);
    for (int i = u.tid; i < N * F; i += u.nthr)
      c0[(size_t)(i / F) * ldy + i % F] = c.emb[(c.spin[i / F] > 0 ? 0 : 1) * F + i % F];
  } else {
    __nv_bfloat16* c0 = cache16w(c, 0);
    for (int i = u.tid; i < N * F; i += u.nthr)
      c0[(size_t)(i / F) * ldh + i % F] = __float2bfloat16_rn(c.emb[(c.spin[i / F] > 0 ? 0 : 1) * F + i % F]);
  }
  unit_sync(u);
  const int F8 = F / 8;
  const int rows_per_pass = c.T * 128;
  for (int l = 1; l <= L; ++l) {
    const __nv_bfloat16* hp = cache16(c, l - 1);
    for (int r0 = 0; r0 < N; r0 += rows_per_pass) {
      const int R = min(rows_per_pass, N - r0);
      const int nt = (R + 127) / 128;
      // one thread per (row, 8-feature chunk): the message chunk and the self chunk
      for (int idx = u.tid; idx < R * F8; idx += u.nthr) {
        const int q = idx / F8, ch = idx - q * F8, v = r0 + q;
        const int k0 = c.rp[v], k1 = c.rp[v + 1];
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (S) {
          const float* hp32 = cache32w(c, l - 1);
          for (int k = k0; k < k1; ++k) fma_chunk32(acc, c.wfs[k], hp32 + (size_t)__ldg(g.col + k) * ldy + ch * 8);
          const unsigned lo = c.a->lay.lo_off;
          uint4 hi, lw;
          split_hi_lo(acc, hi, lw);
          *reinterpret_cast<uint4*>(a_row_chunk(u, F, q, ch)) = hi;
          *reinterpret_cast<uint4*>(a_row_chunk(u, F, q, ch) + lo) = lw;
          split_hi_lo(hp32 + (size_t)v * ldy + ch * 8, hi, lw);
          *reinterpret_cast<uint4*>(a_row_chunk(u, F, q, F8 + ch)) = hi;
          *reinterpret_cast<uint4*>(a_row_chunk(u, F, q, F8 + ch) + lo) = lw;
          continue;
        }
        for (int k = k0; k < k1; ++k) fma_chunk(acc, c.wfs[k], hp + (size_t)__ldg(g.col + k) * ldh + ch * 8);
        uint4 w;
        w.x = pack_bf16(acc[0], acc[1]);
        w.y = pack_bf16(acc[2], acc[3]);
        w.z = pack_bf16(acc[4], acc[5]);
        w.w = pack_bf16(acc[6], acc[7]);
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, q, ch)) = w;
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, q, F8 + ch)) =
            *reinterpret_cast<const uint4*>(hp + (size_t)v * ldh + ch * 8);
      }
      if (!run_mmas<S>(c, u, nt)) return false;
      epilogue_fwd<S>(c, u, nt, R, r0, l, c.a->op != TC_FWD);
    }
  }
  return true;
}

// log Psi readout from the FP32 last layer (valid in thread 0), deterministic order.
// log Psi from H^L (rows of stride ldy): the readout of Eq. gcn, reduced over the CTA.
__device__ void tc_readout(const TcCtx& c, const float* HL, double out[2]) {
  const int N = c.N, F = c.F;
  float* red = (float*)(c.sdbl + 16);
  const int parts = blockDim.x / F;
  const int f = threadIdx.x % F, part = threadIdx.x / F;
  if (part < parts) {
    float acc = 0.f;
    for (int v = part; v < N; v += parts) acc += HL[(size_t)v * c.ldy + f];
    red[part * F + f] = acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    float re = 0.f, im = 0.f;
    for (int ff = threadIdx.x; ff < F; ff += 32) {
      float z = 0.f;
      for (int p = 0; p < parts; ++p) z += red[p * F + ff];
      re += z * c.wr[2 * ff];
      im += z * c.wr[2 * ff + 1];
    }
    re = warp_sum_t(re);
    im = warp_sum_t(im);
    if (threadIdx.x == 0) {
      int up = 0;
      for (int v = 0; v < N; ++v) up += c.spin[v] > 0;
      const int dn = N - up;
      out[0] = (double)(re + (float)up * c.wr[2 * F] + (float)dn * c.wr[2 * (F + 1)] + c.br[0]);
      out[1] = (double)(im + (float)up * c.wr[2 * F + 1] + (float)dn * c.wr[2 * (F + 1) + 1] + c.br[1]);
    }
  }
  __syncthreads();
}

// dX rows of a bond group at layer l, gathered into the unit's A tiles:
//   [ sum_{u in N(v), u in ball_{l-1}} w_vu dH^{l-1}_u ; dH^{l-1}_v (0 outside ball_{l-1}) ]
// One thread per (row, 16 features): the two 8-feature chunks of the message and of the self
// term, the row's index lookups done once for both (every thread of the unit does the same
// amount of work).  S: dH rows in FP32, the gathered rows stored as hi + lo tiles.
template <bool S>
__device__ void gather_delta(const TcCtx& c, const Unit& u, int l, int nb, int q0, int n) {
  const int F = c.F, G = c.G, ldh = c.ldh;
  const int F8 = F / 8;
  const int* offp = u.soff + (l - 1) * (G + 1);
  const int* offl = u.soff + l * (G + 1);
  const int* offL = u.soff + c.L * (G + 1);
  const __nv_bfloat16* dp = new16(c, u, l - 1);
  const int F16 = F8 / 2;  // F is a multiple of 16
  const int f16s = F16 == 1 ? 0 : F16 == 2 ? 1 : F16 == 4 ? 2 : -1;  // log2(F/16) when a power of two
  if (S) {
    const unsigned lo = c.a->lay.lo_off;
    for (int idx = u.tid; idx < n * F16; idx += u.nthr) {
      const int qa = f16s >= 0 ? idx >> f16s : idx / F16, ch = 2 * (idx - qa * F16), q = q0 + qa;
      const int k = slot_of(offl, nb, q);
      const int r = q - offl[k];
      const int sprev = offp[k + 1] - offp[k];
      const int rec = u.srow[offL[k] + r];
      const int v = rec & 0xFFFF;
      const int16_t* np = u.spos + u.eoff[k] + (rec >> 16);
      const int k0 = c.rp[v], dg = c.rp[v + 1] - k0;
      const float* drow32 = new32(c, u, l - 1) + (size_t)offp[k] * c.ldy + ch * 8;
      float acc[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = 0.f;
      for (int t = 0; t < dg; ++t) {
        const int p0 = np[t];
        if (p0 < sprev) {
          const float w = c.wfs[k0 + t];
          const float* x = drow32 + (size_t)p0 * c.ldy;
          fma_chunk32(acc, w, x);
          fma_chunk32(acc + 8, w, x + 8);
        }
      }
      uint4 hi, lw;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        split_hi_lo(acc + 8 * h, hi, lw);
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, qa, ch + h)) = hi;
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, qa, ch + h) + lo) = lw;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = 0.f;
      if (r < sprev) {
        const float4* x = reinterpret_cast<const float4*>(drow32 + (size_t)r * c.ldy);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 a = x[j];
          acc[4 * j] = a.x;
          acc[4 * j + 1] = a.y;
          acc[4 * j + 2] = a.z;
          acc[4 * j + 3] = a.w;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        split_hi_lo(acc + 8 * h, hi, lw);
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, qa, F8 + ch + h)) = hi;
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, qa, F8 + ch + h) + lo) = lw;
      }
    }
    return;
  }
  {
    // neighbours outside ball_{l-1} have dH = 0: they take weight 0 on a valid row (row 0 of
    // the bond), so the loop has no branch; adding the zero products leaves the sums unchanged
    for (int idx = u.tid; idx < n * F16; idx += u.nthr) {
      const int qa = f16s >= 0 ? idx >> f16s : idx / F16, ch = 2 * (idx - qa * F16), q = q0 + qa;
      const int k = slot_of(offl, nb, q);
      const int r = q - offl[k];
      const int sprev = offp[k + 1] - offp[k];
      const __nv_bfloat16* drow = dp + (size_t)offp[k] * ldh + ch * 8;
      const int rec = u.srow[offL[k] + r];
      const int v = rec & 0xFFFF;
      const int16_t* np = u.spos + u.eoff[k] + (rec >> 16);
      const int k0 = c.rp[v], dg = c.rp[v + 1] - k0;
      uint64_t acc2[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int t = 0; t < dg; ++t) {
        const int p0 = np[t];
        const bool in0 = p0 < sprev;
        const float w0 = in0 ? c.wfs[k0 + t] : 0.f;
        const __nv_bfloat16* x0 = drow + (size_t)(in0 ? p0 : 0) * ldh;
        fma_chunk2(acc2, pk2(w0, w0), x0);
        fma_chunk2(acc2 + 4, pk2(w0, w0), x0 + 8);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float acc[8];
        upk2(acc2[4 * h], acc[0], acc[1]);
        upk2(acc2[4 * h + 1], acc[2], acc[3]);
        upk2(acc2[4 * h + 2], acc[4], acc[5]);
        upk2(acc2[4 * h + 3], acc[6], acc[7]);
        uint4 w;
        w.x = pack_bf16(acc[0], acc[1]);
        w.y = pack_bf16(acc[2], acc[3]);
        w.z = pack_bf16(acc[4], acc[5]);
        w.w = pack_bf16(acc[6], acc[7]);
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, qa, ch + h)) = w;
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, qa, F8 + ch + h)) =
            r < sprev ? *reinterpret_cast<const uint4*>(drow + (size_t)r * ldh + 8 * h) : make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }
}

// dH = tanh(Y + dY) - tanh(Y) of 8 units from se = copysign(exp(-2|Y|), Y) and dY:
// with e = exp(-2|Y|), H = sgn(Y)(1-e)/(1+e) and 1 - H^2 = 4e/(1+e)^2, so
// dH = t (1 - H^2)/(1 + H t) = 4 e t / ((1 + e)((1 + e) + sgn(Y)(1 - e) t)), t = tanh(dY).
// S: t to FP32 accuracy (odd Taylor series) instead of the approximate hardware tanh.
template <bool S>
__device__ __forceinline__ float tanh_small(float x) {
  return S ? x + tanh_minus_x(x) : tanh_fast(x);
}
template <bool S>
__device__ __forceinline__ void delta_tanh8(const float* se, const float* dy, float* d) {
  // common case for all 8 units without branches (|dY| < 0.5 and no swing across
  // saturation); if any unit needs more, all 8 are redone by the full rule below, which gives
  // the same result as the common case wherever that applies
  bool slow = false;
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    float den0, den1;
    delta_tanh_pair(fabsf(se[i]), fabsf(se[i + 1]), se[i], se[i + 1], tanh_small<S>(dy[i]), tanh_small<S>(dy[i + 1]),
                    d[i], d[i + 1], den0, den1);
    slow |= !(fabsf(dy[i]) < 0.5f) | !(den0 > 1e-3f) | !(fabsf(dy[i + 1]) < 0.5f) | !(den1 > 1e-3f);
  }
  if (!slow) return;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float e = fabsf(se[i]);
    const float sg = se[i] < 0.f ? -1.f : 1.f;
    const float tt = fabsf(dy[i]) < 0.5f ? tanh_small<S>(dy[i]) : tanhf(dy[i]);
    const float ope = 1.f + e;
    const float den = ope * (ope + sg * (1.f - e) * tt);
    if (den > 1e-3f) {
      d[i] = __fdividef(4.f * e * tt, den);
    } else {
      // a unit swinging across saturation: dH is O(1) and the direct difference has no
      // cancellation (Y recovered from e)
      const float y = -0.5f * sg * __logf(e);
      d[i] = tanhf(y + dy[i]) - tanhf(y);
    }
  }
}

// dY in TMEM -> dH = t (1 - H^2) / (1 + H t), t = tanh(dY), for group rows [0, R) at layer
// l.  l < L: dH stored (BF16) as the next layer's input.  l == L: each thread reduces its
// columns of dH . w_r into per-row partials (Re, Im) for the Delta reduction.
template <bool S>
__device__ void epilogue_delta(const TcCtx& c, const Unit& u, int l, int nt, int nb, int q0) {
  const int warp = u.tid >> 5, lane = u.tid & 31;
  const int q4 = warp & 3, wg = warp >> 2;
  const int F = c.F, L = c.L, G = c.G, ldh = c.ldh, ldy = c.ldy;
  const int* offl = u.soff + l * (G + 1);
  const int R = offl[nb];
  __nv_bfloat16* dout = l < L && !S ? new16(c, u, l) : nullptr;
  float* dout32 = l < L && S ? new32(c, u, l) : nullptr;
  const float* Yl = cacheY(c, l);
  const int* offL = u.soff + L * (G + 1);
  for (int t = 0; t < nt; ++t) {
    const int q = q0 + t * 128 + q4 * 32 + lane;
    int v = 0;
    if (q < R) {
      const int k = slot_of(offl, nb, q);
      v = u.srow[offL[k] + (q - offl[k])] & 0xFFFF;
    }
    float pre = 0.f, pim = 0.f;
    const uint32_t trow = u.tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(t * F);
    // two chunks per TMEM wait: this warp group's chunks ch and ch + nwg
    for (int ch = wg; ch < F / 8; ch += 2 * u.nwg) {
      const int ch2 = ch + u.nwg;
      const bool two = ch2 < F / 8;
      float dy[2][8];
      if (two)
        tmem_ld8x2(trow + ch * 8, trow + ch2 * 8, dy[0], dy[1]);
      else
        tmem_ld8(trow + ch * 8, dy[0]);
      if (q < R) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          if (h2 == 1 && !two) break;
          const int col = (h2 ? ch2 : ch) * 8;
          const float4 a0 = *reinterpret_cast<const float4*>(Yl + (size_t)v * ldy + col);
          const float4 a1 = *reinterpret_cast<const float4*>(Yl + (size_t)v * ldy + col + 4);
          const float se[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          float d[8];
          delta_tanh8<S>(se, dy[h2], d);
          if (S && l < L) {
            float4* o = reinterpret_cast<float4*>(dout32 + (size_t)q * ldy + col);
            o[0] = make_float4(d[0], d[1], d[2], d[3]);
            o[1] = make_float4(d[4], d[5], d[6], d[7]);
          } else if (l < L) {
            uint4 w;
            w.x = pack_bf16(d[0], d[1]);
            w.y = pack_bf16(d[2], d[3]);
            w.z = pack_bf16(d[4], d[5]);
            w.w = pack_bf16(d[6], d[7]);
            *reinterpret_cast<uint4*>(dout + (size_t)q * ldh + col) = w;
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              pre += d[i] * c.wr[2 * (col + i)];
              pim += d[i] * c.wr[2 * (col + i) + 1];
            }
          }
        }
      }
    }
    if (l == L && q < R) {
      u.part[((size_t)wg * c.a->lay.part_rows + q) * 2] = pre;
      u.part[((size_t)wg * c.a->lay.part_rows + q) * 2 + 1] = pim;
    }
  }
  tc_fence_before();
  unit_sync(u);
}

// Incremental Delta log Psi of the unit's bonds slot_e[0..nb): results in res[2k], res[2k+1].
template <bool S>
__device__ bool tc_group(const TcCtx& c, Unit& u, int nb) {
  const DevGraph& g = c.a->g;
  const int F = c.F, L = c.L, G = c.G;
  stage_group<4>(g, u, L, G, nb, u.res + 2 * G);  // the bonds' couplings after their Delta
  // layer 0: dH^0_i = emb(s_j) - emb(s_i), dH^0_j = -dH^0_i
  __nv_bfloat16* d0 = new16(c, u, 0);
  for (int i = u.tid; i < nb * 2 * F; i += u.nthr) {
    const int k = i / (2 * F), r = (i / F) % 2, f = i % F;
    const int e = u.slot_e[k];
    const int self = __ldg(g.edges + 2 * e + r), other = __ldg(g.edges + 2 * e + (1 - r));
    const float dv = c.emb[(c.spin[other] > 0 ? 0 : 1) * F + f] - c.emb[(c.spin[self] > 0 ? 0 : 1) * F + f];
    if (S)
      new32(c, u, 0)[(size_t)(u.soff[k] + r) * c.ldy + f] = dv;
    else
      d0[(size_t)(u.soff[k] + r) * c.ldh + f] = __float2bfloat16_rn(dv);
  }
  unit_sync(u);
  // each layer in passes of at most T tiles of 128 rows
  for (int l = 1; l <= L; ++l) {
    const int R = u.soff[l * (G + 1) + nb];
    for (int q0 = 0; q0 < R; q0 += c.T * 128) {
      const int n = min(c.T * 128, R - q0);
      gather_delta<S>(c, u, l, nb, q0, n);
      const int nt = (n + 127) / 128;
      if (!run_mmas<S>(c, u, nt)) return false;
      epilogue_delta<S>(c, u, l, nt, nb, q0);
    }
  }
  // Delta_k = sum over the bond's last-layer rows of the per-row partials (one warp per bond)
  const int warp = u.tid >> 5, lane = u.tid & 31, nwarps = u.nthr >> 5;
  const int* offL = u.soff + L * (G + 1);
  const size_t wgs = (size_t)c.a->lay.part_rows;
  for (int k = warp; k < nb; k += nwarps) {
    float dre = 0.f, dim = 0.f;
    for (int q = offL[k] + lane; q < offL[k + 1]; q += 32) {
      for (int w = 0; w < min(u.nwg, F / 8); ++w) {
        dre += u.part[(w * wgs + q) * 2];
        dim += u.part[(w * wgs + q) * 2 + 1];
      }
    }
    dre = warp_sum_t(dre);
    dim = warp_sum_t(dim);
    if (lane == 0) {
      u.res[2 * k] = (double)dre;
      u.res[2 * k + 1] = (double)dim;
    }
  }
  unit_sync(u);
  return true;
}

// S: split operands (hi + lo BF16 on the tensor cores, FP32 feature rows, accurate tanh).
template <bool S>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_fail;
  __shared__ int s_count;
  __shared__ double s_eu[2 * kTcMaxUnits];
  TcCtx c;
  c.a = &a;
  c.N = a.m.N;
  c.F = a.m.F;
  c.L = a.m.L;
  c.E = a.m.E;
  c.T = a.lay.T;
  c.G = a.lay.G;
  c.ldh = a.m.F + 8;
  c.ldy = a.m.F + 4;
  c.Wt = (__nv_bfloat16*)(smem + a.lay.oWt);
  c.bias = (float*)(smem + a.lay.obias);
  c.emb = (float*)(smem + a.lay.oemb);
  c.wr = (float*)(smem + a.lay.owr);
  c.br = (float*)(smem + a.lay.obr);
  c.spin = (int8_t*)(smem + a.lay.ospin);
  c.rp = (const int*)(smem + a.lay.orp);
  c.wfs = (const float*)(smem + a.lay.owf);
  c.list = (int*)(smem + a.lay.oint);
  c.sdbl = (double*)(smem + a.lay.odbl);
  c.region = a.region_in_smem ? smem + a.lay.oregion : a.gregion + (size_t)blockIdx.x * a.lay.region_bytes;
  c.ycache = a.lay.y_global ? a.gY + (size_t)blockIdx.x * (a.lay.y_bytes / 4) : (float*)(c.region + a.lay.rY);
  c.hL = a.op == TC_ELOC && a.logpsi ? a.gH + (size_t)blockIdx.x * a.m.N * (a.m.F + 4) : nullptr;
  c.fail = &s_fail;
  const int F = c.F, N = c.N;
  const Dims& m = a.m;
  const float* th = a.theta;
  uint64_t* bars = (uint64_t*)(smem + a.lay.obar);
  uint32_t* slot = (uint32_t*)(smem + a.lay.oslot);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int h = 0; h < a.lay.units; ++h) mbar_init(bars + h, 1);
  }
  if ((threadIdx.x >> 5) == 0) {
    tmem_alloc(slot, kTmemCols);
    tmem_relinquish();
  }
  // W^T (n = output feature, k = input feature) in the canonical K-major layout
  const float* W = th + m.oW;
  for (int i = threadIdx.x; i < F * 2 * F; i += blockDim.x) {
    const int n = i / (2 * F), k = i % (2 * F);
    unsigned char* p = (unsigned char*)c.Wt + (size_t)(n >> 3) * (32 * F) + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(W[(size_t)k * F + n]);
  }
  for (int i = threadIdx.x; i < F; i += blockDim.x) c.bias[i] = th[m.ob + i];
  for (int i = threadIdx.x; i < 2 * F; i += blockDim.x) c.emb[i] = tanhf(th[m.oWe + i] + th[m.obe + i % F]);
  for (int i = threadIdx.x; i < (F + 2) * 2; i += blockDim.x) c.wr[i] = th[m.owr + i];
  if (threadIdx.x < 2) c.br[threadIdx.x] = th[m.obr + threadIdx.x];
  for (int i = threadIdx.x; i <= c.N; i += blockDim.x) ((int*)c.rp)[i] = __ldg(c.a->g.row_ptr + i);
  for (int i = threadIdx.x; i < 2 * c.E; i += blockDim.x) ((float*)c.wfs)[i] = __ldg(c.a->g.wf + i);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  // the whole CTA as one unit (forward), and this thread's bond-group unit
  Unit whole;
  whole.tid = threadIdx.x;
  whole.nthr = blockDim.x;
  whole.bar_id = 0;
  whole.nwg = blockDim.x / 128;
  whole.A = smem + a.lay.oA;
  whole.tbase = tmem;
  whole.bar = bars;
  whole.phase = 0;
  const int U = a.lay.units, unit_threads = kTcThreads / U;
  const int h = threadIdx.x / unit_threads;
  Unit u;
  u.tid = threadIdx.x % unit_threads;
  u.nthr = unit_threads;
  u.bar_id = 1 + h;
  u.nwg = unit_threads / 128;
  u.A = smem + a.lay.oA + (size_t)h * a.lay.a_unit;
  u.tbase = tmem + (uint32_t)(h * c.T * F);
  u.bar = bars + h;
  u.phase = 0;
  u.d16 = (__nv_bfloat16*)(c.region + a.lay.rnew16 + (size_t)h * a.lay.new16_unit);
  u.part = (float*)(c.region + a.lay.rpart + (size_t)h * a.lay.part_unit);
  u.slot_e = c.list + c.E + 16 + h * a.lay.int_unit;
  u.soff = u.slot_e + c.G;
  u.eoff = u.soff + (c.L + 1) * (c.G + 1);
  u.srow = (int*)(smem + a.lay.orow) + (size_t)h * a.lay.row_unit;
  u.spos = (int16_t*)(smem + a.lay.opos) + (size_t)h * a.lay.pos_unit;
  u.res = c.sdbl + 16 + kTcThreads + h * a.lay.dbl_unit;

  bool ok = true;
  for (int64_t b = blockIdx.x; b < a.B && ok; b += gridDim.x) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) c.spin[i] = a.spins[b * N + i];
    __syncthreads();
    // unit 0 and the whole CTA share mbarrier 0: its waiter (thread 0) carries the phase
    if (threadIdx.x == 0) whole.phase = u.phase;
    ok = tc_forward<S>(c, whole);
    if (threadIdx.x == 0) u.phase = whole.phase;
    if (!ok) break;
    if (a.op == TC_FWD) {
      double lp[2];
      tc_readout(c, cacheY(c, c.L), lp);  // the forward-only call keeps H^L there
      if (threadIdx.x == 0) {
        a.logpsi[2 * b] = lp[0];
        a.logpsi[2 * b + 1] = lp[1];
      }
      continue;
    }
    if (a.logpsi) {  // log Psi from this call's forward, as the forward-only call gives it
      double lp[2];
      tc_readout(c, c.hL, lp);
      if (threadIdx.x == 0) {
        a.logpsi[2 * b] = lp[0];
        a.logpsi[2 * b + 1] = lp[1];
      }
    }
    // antiparallel bonds (ordered) and the diagonal energy
    double diag = 0.0;
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int count = 0;
      double d = 0.0;
      for (int base = 0; base < c.E; base += 32) {
        const int e = base + lane;
        bool anti = false;
        if (e < c.E) {
          const int i = __ldg(a.g.edges + 2 * e), j = __ldg(a.g.edges + 2 * e + 1);
          const int si = c.spin[i], sj = c.spin[j];
          anti = si != sj;
          d += bond_diag(a.g, e, si, sj);
        }
        const unsigned mask = __ballot_sync(0xffffffffu, anti);
        if (anti) c.list[count + __popc(mask & ((1u << lane) - 1u))] = e;
        count += __popc(mask);
      }
      d = warp_sum_t(d);
      if (lane == 0) {
        s_count = count;
        diag = d;
      }
    }
    if (a.dlogpsi)
      for (int e = threadIdx.x; e < c.E; e += blockDim.x) a.dlogpsi[b * c.E + e] = 0.f;
    __syncthreads();
    const int na = s_count;
    // unit h takes the h-th of U equal shares of the antiparallel bonds, in groups of up to
    // G bonds (equal shares keep the units' work balanced up to one bond)
    // lane k of the unit's first warp sums the terms of bond k of each group (in shared
    // memory, not registers, which the passes need)
    double* lsum = u.res + 3 * c.G;
    if (u.tid < 32) {
      lsum[2 * u.tid] = 0.0;
      lsum[2 * u.tid + 1] = 0.0;
    }
    const int b_lo = (int)((int64_t)na * h / U), b_hi = (int)((int64_t)na * (h + 1) / U);
    for (int t0 = b_lo; t0 < b_hi; t0 += c.G) {
      const int nb = min(c.G, b_hi - t0);
      if (u.tid < nb) u.slot_e[u.tid] = c.list[t0 + u.tid];
      unit_sync(u);
      if (!tc_group<S>(c, u, nb)) break;
      // bond k's term Jxy/2 exp(Delta) by lane k of the unit's first warp, added to that
      // lane's own sum (the warp's next writes of slot_e follow its own reads, and the other
      // warps read slot_e only after the next group's barrier)
      if (u.tid < nb) {
        const int k = u.tid, e = u.slot_e[k];
        const float dre = (float)u.res[2 * k], dim = (float)u.res[2 * k + 1];
        const float amp = expf(dre);
        float sn, cs;
        sincosf(dim, &sn, &cs);
        const double hJ = 0.5 * u.res[2 * c.G + k];
        lsum[2 * k] += hJ * (double)(amp * cs);
        lsum[2 * k + 1] += hJ * (double)(amp * sn);
        if (a.dlogpsi) a.dlogpsi[b * c.E + e] = dre;
      }
    }
    // the unit's sum over its bonds: the lanes' sums, added across the first warp
    double er = 0.0, ei = 0.0;
    if (u.tid < 32) {
      er = warp_sum_t(lsum[2 * u.tid]);
      ei = warp_sum_t(lsum[2 * u.tid + 1]);
    }
    if (u.tid == 0) {
      s_eu[2 * h] = er;
      s_eu[2 * h + 1] = ei;
    }
    __syncthreads();
    ok = s_fail == 0;
    if (threadIdx.x == 0 && ok) {
      double re = diag, im = 0.0;
      for (int hh = 0; hh < U; ++hh) {
        re += s_eu[2 * hh];
        im += s_eu[2 * hh + 1];
      }
      a.eloc[2 * b] = re;
      a.eloc[2 * b + 1] = im;
    }
    __syncthreads();
  }
  // teardown: on failure wait (bounded) for the MMAs in flight before freeing TMEM
  if (!ok && u.tid == 0) mbar_wait_bounded(u.bar, u.phase ^ 1u);  // the phase that timed out
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------------
// Metropolis pair-exchange sweeps on the tensor cores (plain moves, BF16 models)
// ---------------------------------------------------------------------------------
// The move rule is the one of the CUDA-core samplers: step t of chain c draws
// Philox4x64-10(key = (seed, c), counter = (t, 0, 0, 0)), bond e = hi64(r0 |E|), a
// parallel bond is a rejected no-op, an antiparallel one is accepted iff
// (r1 >> 40) 2^-24 < exp(2 Re Delta).  Delta is the difference propagation of the local
// energy kernel (BF16 operands on the tensor cores, FP32 accumulation and activations).
//
// Each unit owns a pool of G chains.  In one round every unfinished chain of the pool
// first runs through its no-op steps (a thread per chain), stopping at its next
// antiparallel proposal (or at a sweep whose sample is recorded); the pending proposals
// of the pool are then evaluated together as one bond group -- the rows of all of them
// share the A tiles of each layer -- and accepted or rejected independently.  Chains are
// independent, so this schedule changes nothing in any chain's trajectory.
//
// Per chain, the unit keeps in the workspace (L2-resident: a few hundred KiB per SM) the
// FP32 pre-activations Y^1..Y^L of the current configuration and the dY rows of the
// pending proposal; an accepted move adds dY to Y.  The chain's Y is computed by a
// tensor-core forward when the chain enters the pool.
struct TcmArgs {
  TcArgs base;  // graph, dims, theta and the layout of the A tiles / dH rows / partials
  int8_t* chain_spins;
  int64_t C;
  int n_sweeps, record_every;
  uint64_t seed, step0;
  int8_t* samples_out;
  double* logpsi_out;
  int32_t* n_acc;
  double* trace;
  float* gws;                  // per unit: G slots of slot_elems, then the H scratch
  uint64_t slot_elems;         // Y^1..Y^L [L][N][F], then dY rows (FP32 elements)
  uint64_t unit_elems;         // FP32 elements per unit (slots + two BF16 H layers)
  uint64_t dy_off[kMaxL + 1];  // element offset of the dY^l rows in a slot (l = 1..L)
};

struct TcmSlots {        // per-unit pool state (shared memory)
  int64_t* chain;        // [G] chain index or -1
  int64_t* step;         // [G] steps done in this launch
  int64_t* wbase;        // [G] first step of the cached Philox words
  uint64_t* words;       // [G][32][2] (r0, r1) of steps wbase .. wbase + 31
  uint64_t* r1;          // [G] uniform word of the pending proposal
  double* red;           // [2 * unit threads] reduction scratch
  int* flag;             // [G] bit 0: proposal pending, bit 1: record pending, bit 2: done
  int* acc;              // [G] accepted moves in this launch
  int* bond;             // [G] bond of the pending proposal
  int* gslot;            // [G] slot of group member k
  int* ok;               // [G] group member k accepted
  int8_t* spins;         // [G][N]
};

__host__ __device__ inline size_t tcm_state_bytes(int G, int N, int unit_threads) {
  const size_t b = (size_t)G * 8 * 4 + (size_t)G * 32 * 16 + (size_t)unit_threads * 16 + (size_t)G * 4 * 5 + (size_t)G * N;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ float* tcm_slot(const TcmArgs& a, int unit_global, int s) {
  return a.gws + (size_t)unit_global * a.unit_elems + (size_t)s * a.slot_elems;
}

// Forward of slot s's configuration: fills its Y^1..Y^L (FP32) through the unit's tiles.
__device__ bool tcm_forward(const TcCtx& c, Unit& u, const TcmArgs& a, float* Ys, __nv_bfloat16* Hs,
                            const int8_t* sp) {
  const int N = c.N, F = c.F, L = c.L, ldh = c.ldh, F8 = F / 8;
  const DevGraph& g = c.a->g;
  for (int i = u.tid; i < N * F; i += u.nthr)
    Hs[(size_t)(i / F) * ldh + i % F] = __float2bfloat16_rn(c.emb[(sp[i / F] > 0 ? 0 : 1) * F + i % F]);
  unit_sync(u);
  const int rows_per_pass = c.T * 128;
  const int warp = u.tid >> 5, lane = u.tid & 31, q4 = warp & 3, wg = warp >> 2;
  for (int l = 1; l <= L; ++l) {
    const __nv_bfloat16* hp = Hs + (size_t)((l - 1) & 1) * N * ldh;
    __nv_bfloat16* hn = Hs + (size_t)(l & 1) * N * ldh;
    float* Y = Ys + (size_t)(l - 1) * N * F;
    for (int r0 = 0; r0 < N; r0 += rows_per_pass) {
      const int R = min(rows_per_pass, N - r0);
      const int nt = (R + 127) / 128;
      for (int idx = u.tid; idx < R * F8; idx += u.nthr) {
        const int q = idx / F8, ch = idx - q * F8, v = r0 + q;
        const int k0 = c.rp[v], k1 = c.rp[v + 1];
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = k0; k < k1; ++k) fma_chunk(acc, c.wfs[k], hp + (size_t)__ldg(g.col + k) * ldh + ch * 8);
        uint4 w;
        w.x = pack_bf16(acc[0], acc[1]);
        w.y = pack_bf16(acc[2], acc[3]);
        w.z = pack_bf16(acc[4], acc[5]);
        w.w = pack_bf16(acc[6], acc[7]);
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, q, ch)) = w;
        *reinterpret_cast<uint4*>(a_row_chunk(u, F, q, F8 + ch)) =
            *reinterpret_cast<const uint4*>(hp + (size_t)v * ldh + ch * 8);
      }
      if (!run_mmas<false>(c, u, nt)) return false;
      for (int t = 0; t < nt; ++t) {
        const int q = t * 128 + q4 * 32 + lane;
        for (int ch = wg; ch < F8; ch += u.nwg) {
          float v8[8];
          tmem_ld8(u.tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(t * F + ch * 8), v8);
          if (q < R) {
#pragma unroll
            for (int i = 0; i < 8; ++i) v8[i] += c.bias[ch * 8 + i];
            float4* yo = reinterpret_cast<float4*>(Y + (size_t)(r0 + q) * F + ch * 8);
            yo[0] = make_float4(v8[0], v8[1], v8[2], v8[3]);
            yo[1] = make_float4(v8[4], v8[5], v8[6], v8[7]);
            if (l < L) {
              uint4 w;
              w.x = pack_bf16(tanh_fast(v8[0]), tanh_fast(v8[1]));
              w.y = pack_bf16(tanh_fast(v8[2]), tanh_fast(v8[3]));
              w.z = pack_bf16(tanh_fast(v8[4]), tanh_fast(v8[5]));
              w.w = pack_bf16(tanh_fast(v8[6]), tanh_fast(v8[7]));
              *reinterpret_cast<uint4*>(hn + (size_t)(r0 + q) * ldh + ch * 8) = w;
            }
          }
        }
      }
      tc_fence_before();
      unit_sync(u);
    }
  }
  return true;
}

// dY in TMEM -> dH for the group rows at layer l; the chains' own Y^l rows are read from
// their slots, dY^l rows are kept in the slots for the update on acceptance.
__device__ void tcm_epilogue(const TcCtx& c, const Unit& u, const TcmArgs& a, const TcmSlots& S, int ug, int l,
                             int nt, int nb, int q0) {
  const int warp = u.tid >> 5, lane = u.tid & 31;
  const int q4 = warp & 3, wg = warp >> 2;
  const int F = c.F, L = c.L, N = c.N, G = c.G, ldh = c.ldh;
  const int* offl = u.soff + l * (G + 1);
  const int R = offl[nb];
  __nv_bfloat16* dout = l < L ? new16(c, u, l) : nullptr;
  for (int t = 0; t < nt; ++t) {
    const int q = q0 + t * 128 + q4 * 32 + lane;
    const float* yrow = nullptr;
    float* dyrow = nullptr;
    if (q < R) {
      const int k = slot_of(offl, nb, q);
      const int r = q - offl[k];
      const int v = u.srow[u.soff[L * (G + 1) + k] + r] & 0xFFFF;
      float* sl = tcm_slot(a, ug, S.gslot[k]);
      yrow = sl + (size_t)(l - 1) * N * F + (size_t)v * F;
      dyrow = sl + a.dy_off[l] + (size_t)r * F;
    }
    float pre = 0.f, pim = 0.f;
    const uint32_t trow = u.tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(t * F);
    // two chunks per TMEM wait: this warp group's chunks ch and ch + nwg
    for (int ch = wg; ch < F / 8; ch += 2 * u.nwg) {
      const int ch2 = ch + u.nwg;
      const bool two = ch2 < F / 8;
      float4 y[2][2];
      if (q < R) {
        y[0][0] = *reinterpret_cast<const float4*>(yrow + ch * 8);
        y[0][1] = *reinterpret_cast<const float4*>(yrow + ch * 8 + 4);
        if (two) {
          y[1][0] = *reinterpret_cast<const float4*>(yrow + ch2 * 8);
          y[1][1] = *reinterpret_cast<const float4*>(yrow + ch2 * 8 + 4);
        }
      }
      float dy[2][8];
      if (two)
        tmem_ld8x2(trow + ch * 8, trow + ch2 * 8, dy[0], dy[1]);
      else
        tmem_ld8(trow + ch * 8, dy[0]);
      if (q < R) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          if (h2 == 1 && !two) break;
          const int col = (h2 ? ch2 : ch) * 8;
          const float* dv = dy[h2];
          reinterpret_cast<float4*>(dyrow + col)[0] = make_float4(dv[0], dv[1], dv[2], dv[3]);
          reinterpret_cast<float4*>(dyrow + col)[1] = make_float4(dv[4], dv[5], dv[6], dv[7]);
          const float yv[8] = {y[h2][0].x, y[h2][0].y, y[h2][0].z, y[h2][0].w,
                               y[h2][1].x, y[h2][1].y, y[h2][1].z, y[h2][1].w};
          float d[8];
          // common case without branches, the full rule only when a unit needs it (as delta_tanh8)
          bool slow = false;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float e = __expf(-2.f * fabsf(yv[i]));
            const float sg = yv[i] < 0.f ? -1.f : 1.f;
            const float tt = tanh_fast(dv[i]);
            const float ope = 1.f + e;
            const float den = ope * (ope + sg * (1.f - e) * tt);
            d[i] = __fdividef(4.f * e * tt, den);
            slow |= !(fabsf(dv[i]) < 0.5f) | !(den > 1e-3f);
          }
          if (slow) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float e = __expf(-2.f * fabsf(yv[i]));
              const float sg = yv[i] < 0.f ? -1.f : 1.f;
              const float tt = fabsf(dv[i]) < 0.5f ? tanh_fast(dv[i]) : tanhf(dv[i]);
              const float ope = 1.f + e;
              const float den = ope * (ope + sg * (1.f - e) * tt);
              d[i] = den > 1e-3f ? __fdividef(4.f * e * tt, den) : tanhf(yv[i] + dv[i]) - tanhf(yv[i]);
            }
          }
          if (l < L) {
            uint4 w;
            w.x = pack_bf16(d[0], d[1]);
            w.y = pack_bf16(d[2], d[3]);
            w.z = pack_bf16(d[4], d[5]);
            w.w = pack_bf16(d[6], d[7]);
            *reinterpret_cast<uint4*>(dout + (size_t)q * ldh + col) = w;
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              pre += d[i] * c.wr[2 * (col + i)];
              pim += d[i] * c.wr[2 * (col + i) + 1];
            }
          }
        }
      }
    }
    if (l == L && q < R) {
      u.part[((size_t)wg * c.a->lay.part_rows + q) * 2] = pre;
      u.part[((size_t)wg * c.a->lay.part_rows + q) * 2 + 1] = pim;
    }
  }
  tc_fence_before();
  unit_sync(u);
}

// Delta log Psi of the pending proposals of group members 0..nb-1 (bonds u.slot_e).
__device__ bool tcm_group(const TcCtx& c, Unit& u, const TcmArgs& a, const TcmSlots& S, int ug, int nb) {
  const DevGraph& g = c.a->g;
  const int F = c.F, L = c.L, G = c.G;
  stage_group<1>(g, u, L, G, nb);
  __nv_bfloat16* d0 = new16(c, u, 0);
  for (int i = u.tid; i < nb * 2 * F; i += u.nthr) {
    const int k = i / (2 * F), r = (i / F) % 2, f = i % F;
    const int e = u.slot_e[k];
    const int8_t* sp = S.spins + (size_t)S.gslot[k] * c.N;
    const int self = __ldg(g.edges + 2 * e + r), other = __ldg(g.edges + 2 * e + (1 - r));
    const float dv = c.emb[(sp[other] > 0 ? 0 : 1) * F + f] - c.emb[(sp[self] > 0 ? 0 : 1) * F + f];
    d0[(size_t)(u.soff[k] + r) * c.ldh + f] = __float2bfloat16_rn(dv);
  }
  unit_sync(u);
  for (int l = 1; l <= L; ++l) {
    const int R = u.soff[l * (G + 1) + nb];
    for (int q0 = 0; q0 < R; q0 += c.T * 128) {
      const int n = min(c.T * 128, R - q0);
      gather_delta<false>(c, u, l, nb, q0, n);
      const int nt = (n + 127) / 128;
      if (!run_mmas<false>(c, u, nt)) return false;
      tcm_epilogue(c, u, a, S, ug, l, nt, nb, q0);
    }
  }
  const int warp = u.tid >> 5, lane = u.tid & 31, nwarps = u.nthr >> 5;
  const int* offL = u.soff + L * (G + 1);
  const size_t wgs = (size_t)c.a->lay.part_rows;
  for (int k = warp; k < nb; k += nwarps) {
    float dre = 0.f, dim = 0.f;
    for (int q = offL[k] + lane; q < offL[k + 1]; q += 32) {
      for (int w = 0; w < min(u.nwg, F / 8); ++w) {
        dre += u.part[(w * wgs + q) * 2];
        dim += u.part[(w * wgs + q) * 2 + 1];
      }
    }
    dre = warp_sum_t(dre);
    dim = warp_sum_t(dim);
    if (lane == 0) {
      u.res[2 * k] = (double)dre;
      u.res[2 * k + 1] = (double)dim;
    }
  }
  unit_sync(u);
  return true;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_metro(const TcmArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_fail;
  __shared__ int s_more[kTcMaxUnits];
  __shared__ uint32_t s_dyoff[kMaxL + 1];  // a.dy_off, indexed by a runtime layer
  const TcArgs& b = a.base;
  TcCtx c;
  c.a = &b;
  c.N = b.m.N;
  c.F = b.m.F;
  c.L = b.m.L;
  c.E = b.m.E;
  c.T = b.lay.T;
  c.G = b.lay.G;
  c.ldh = b.m.F + 8;
  c.ldy = b.m.F + 4;
  c.Wt = (__nv_bfloat16*)(smem + b.lay.oWt);
  c.bias = (float*)(smem + b.lay.obias);
  c.emb = (float*)(smem + b.lay.oemb);
  c.wr = (float*)(smem + b.lay.owr);
  c.br = (float*)(smem + b.lay.obr);
  c.spin = nullptr;
  c.rp = (const int*)(smem + b.lay.orp);
  c.wfs = (const float*)(smem + b.lay.owf);
  c.list = (int*)(smem + b.lay.oint);
  c.sdbl = (double*)(smem + b.lay.odbl);
  c.region = smem + b.lay.oregion;
  c.ycache = (float*)(c.region + b.lay.rY);
  c.fail = &s_fail;
  const int F = c.F, N = c.N, L = c.L, G = c.G, E = c.E;
  const Dims& m = b.m;
  const float* th = b.theta;
  uint64_t* bars = (uint64_t*)(smem + b.lay.obar);
  uint32_t* slot = (uint32_t*)(smem + b.lay.oslot);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int h = 0; h < b.lay.units; ++h) mbar_init(bars + h, 1);
    for (int l = 0; l <= kMaxL; ++l) s_dyoff[l] = (uint32_t)a.dy_off[l];
  }
  if ((threadIdx.x >> 5) == 0) {
    tmem_alloc(slot, kTmemCols);
    tmem_relinquish();
  }
  const float* W = th + m.oW;
  for (int i = threadIdx.x; i < F * 2 * F; i += blockDim.x) {
    const int n = i / (2 * F), k = i % (2 * F);
    unsigned char* p = (unsigned char*)c.Wt + (size_t)(n >> 3) * (32 * F) + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(W[(size_t)k * F + n]);
  }
  for (int i = threadIdx.x; i < F; i += blockDim.x) c.bias[i] = th[m.ob + i];
  for (int i = threadIdx.x; i < 2 * F; i += blockDim.x) c.emb[i] = tanhf(th[m.oWe + i] + th[m.obe + i % F]);
  for (int i = threadIdx.x; i < (F + 2) * 2; i += blockDim.x) c.wr[i] = th[m.owr + i];
  if (threadIdx.x < 2) c.br[threadIdx.x] = th[m.obr + threadIdx.x];
  for (int i = threadIdx.x; i <= c.N; i += blockDim.x) ((int*)c.rp)[i] = __ldg(c.a->g.row_ptr + i);
  for (int i = threadIdx.x; i < 2 * c.E; i += blockDim.x) ((float*)c.wfs)[i] = __ldg(c.a->g.wf + i);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  const int U = b.lay.units, unit_threads = kTcThreads / U;
  const int h = threadIdx.x / unit_threads;
  Unit u;
  u.tid = threadIdx.x % unit_threads;
  u.nthr = unit_threads;
  u.bar_id = 1 + h;
  u.nwg = unit_threads / 128;
  u.A = smem + b.lay.oA + (size_t)h * b.lay.a_unit;
  u.tbase = tmem + (uint32_t)(h * c.T * F);
  u.bar = bars + h;
  u.phase = 0;
  const int ug = blockIdx.x * U + h;  // this unit's workspace index
  float* unit_ws = a.gws + (size_t)ug * a.unit_elems;
  u.d16 = b.region_in_smem ? (__nv_bfloat16*)(c.region + b.lay.rnew16 + (size_t)h * b.lay.new16_unit)
                           : (__nv_bfloat16*)(unit_ws + (size_t)G * a.slot_elems + (size_t)N * (F + 8));
  u.part = (float*)(c.region + b.lay.rpart + (size_t)h * b.lay.part_unit);
  u.slot_e = c.list + h * b.lay.int_unit;
  u.soff = u.slot_e + G;
  u.eoff = u.soff + (L + 1) * (G + 1);
  u.srow = (int*)(smem + b.lay.orow) + (size_t)h * b.lay.row_unit;
  u.spos = (int16_t*)(smem + b.lay.opos) + (size_t)h * b.lay.pos_unit;
  u.res = c.sdbl + h * b.lay.dbl_unit;
  // pool state of this unit: after the unit's ints and doubles
  TcmSlots S;
  {
    unsigned char* st = c.region + b.lay.rstate + (size_t)h * b.lay.state_unit;
    S.chain = (int64_t*)st;
    S.step = S.chain + G;
    S.wbase = S.step + G;
    S.r1 = (uint64_t*)(S.wbase + G);
    S.words = S.r1 + G;
    S.red = (double*)(S.words + (size_t)G * 64);
    S.flag = (int*)(S.red + 2 * unit_threads);
    S.acc = S.flag + G;
    S.bond = S.acc + G;
    S.gslot = S.bond + G;
    S.ok = S.gslot + G;
    S.spins = (int8_t*)(S.ok + G);
  }
  float* Hs_f = unit_ws + (size_t)G * a.slot_elems;
  __nv_bfloat16* Hs = (__nv_bfloat16*)Hs_f;
  const int64_t n_steps = (int64_t)a.n_sweeps * N;
  const int64_t pools = (a.C + G - 1) / G;

  bool ok = true;
  for (int64_t pool = (int64_t)blockIdx.x * U + h; pool < pools && ok; pool += (int64_t)gridDim.x * U) {
    // enter the pool's chains
    for (int s = 0; s < G; ++s) {
      const int64_t ch = pool * G + s;
      for (int v = u.tid; v < N; v += u.nthr) S.spins[(size_t)s * N + v] = ch < a.C ? a.chain_spins[ch * N + v] : (int8_t)1;
      if (u.tid == 0) {
        S.chain[s] = ch < a.C ? ch : -1;
        S.step[s] = 0;
        S.wbase[s] = -64;
        S.flag[s] = ch < a.C ? 0 : 4;
        S.acc[s] = 0;
      }
    }
    unit_sync(u);
    for (int s = 0; s < G && ok; ++s) {
      if (S.chain[s] < 0) continue;
      ok = tcm_forward(c, u, a, tcm_slot(a, ug, s), Hs, S.spins + (size_t)s * N);
    }
    if (!ok) break;
    while (true) {
      // 1. each chain runs through its no-op steps up to its next proposal or record (one
      //    warp per chain: its lanes draw the Philox words of 32 steps at once)
      {
        const int warp = u.tid >> 5, lane = u.tid & 31, nwarps = u.nthr >> 5;
        for (int s = warp; s < G; s += nwarps) {
          int fl = S.flag[s] & 4;
          if (fl) continue;
          const int64_t ch = S.chain[s];
          const int8_t* sp = S.spins + (size_t)s * N;
          int64_t k = S.step[s];
          if (k >= n_steps) fl = 4;
          while (!fl) {
            if (k >= S.wbase[s] + 32) {
              __syncwarp();
              const U64x4 w = philox4x64_10(a.seed, (uint64_t)ch, U64x4{a.step0 + (uint64_t)(k + lane), 0, 0, 0});
              S.words[((size_t)s * 32 + lane) * 2] = w.x;
              S.words[((size_t)s * 32 + lane) * 2 + 1] = w.y;
              __syncwarp();
              if (lane == 0) S.wbase[s] = k;
              __syncwarp();
            }
            // lane 0 scans the cached steps; the outcome is broadcast
            int stop = 0, eb = 0;
            int64_t kn = k;
            if (lane == 0) {
              const int64_t wb = S.wbase[s];
              while (kn < wb + 32 && kn < n_steps) {
                const uint64_t r0 = S.words[((size_t)s * 32 + (kn - wb)) * 2];
                const int e = (int)__umul64hi(r0, (uint64_t)E);
                if (sp[__ldg(b.g.edges + 2 * e)] != sp[__ldg(b.g.edges + 2 * e + 1)]) {
                  S.r1[s] = S.words[((size_t)s * 32 + (kn - wb)) * 2 + 1];
                  eb = e;
                  stop = 1;
                  break;
                }
                if (a.trace) {
                  double* tr = a.trace + ((size_t)ch * n_steps + kn) * 4;
                  tr[0] = (double)e;
                  tr[1] = 0.0;
                  tr[2] = __longlong_as_double(0x7ff8000000000000ll);
                  tr[3] = 1.0;
                }
                ++kn;
                if (a.record_every > 0 && kn % N == 0 && (kn / N) % a.record_every == 0) {
                  stop = 2;
                  break;
                }
                if (kn >= n_steps) {
                  stop = 4;
                  break;
                }
              }
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            k = __shfl_sync(0xffffffffu, kn, 0);
            eb = __shfl_sync(0xffffffffu, eb, 0);
            if (stop) {
              fl = stop;
              if (lane == 0 && stop == 1) S.bond[s] = eb;
            }
          }
          if (lane == 0) {
            S.step[s] = k;
            S.flag[s] = fl;
          }
        }
      }
      unit_sync(u);
      // 2. the pending proposals as one group
      if (u.tid == 0) {
        int nb = 0, more = 0;
        for (int s = 0; s < G; ++s) {
          if (S.flag[s] & 1) {
            S.gslot[nb] = s;
            u.slot_e[nb] = S.bond[s];
            ++nb;
          }
          if (!(S.flag[s] & 4)) more = 1;
        }
        u.eoff[G + 1] = nb;  // spare slot after the entry offsets
        s_more[h] = more;
      }
      unit_sync(u);
      const int nb = u.eoff[G + 1];
      if (nb > 0) {
        if (!tcm_group(c, u, a, S, ug, nb)) {
          ok = false;
          break;
        }
        // 3. decisions
        if (u.tid < nb) {
          const int k = u.tid, s = S.gslot[k];
          const float dre = (float)u.res[2 * k];
          const bool acc = (float)(S.r1[s] >> 40) * 0x1.0p-24f < expf(2.0f * dre);
          S.ok[k] = acc ? 1 : 0;
          if (acc) ++S.acc[s];
          if (a.trace) {
            double* tr = a.trace + ((size_t)S.chain[s] * n_steps + S.step[s]) * 4;
            tr[0] = (double)u.slot_e[k];
            tr[1] = acc ? 1.0 : 0.0;
            tr[2] = (double)dre;
            tr[3] = 1.0;
          }
        }
        unit_sync(u);
        // 4. accepted moves: Y += dY on the bond's balls, exchange the spins.  The items
        //    (layer, ball row, 4 features) of an accepted bond are spread over the unit's
        //    threads, two per thread per round with every load issued before the stores,
        //    so that their L2 latencies overlap (rows and sizes from the staged tables)
        for (int k = 0; k < nb; ++k) {
          if (!S.ok[k]) continue;
          const int s = S.gslot[k], e = u.slot_e[k];
          float* sl = tcm_slot(a, ug, s);
          const int F4 = F / 4;
          const int* rows = u.srow + u.soff[L * (G + 1) + k];
          int total = 0;
          for (int l = 1; l <= L; ++l) total += (u.soff[l * (G + 1) + k + 1] - u.soff[l * (G + 1) + k]) * F4;
          for (int i0 = u.tid; i0 < total; i0 += 2 * u.nthr) {
            int yo[2];  // float offset of the item's Y in the slot, -1 past the end
            float4 yv[2], dv[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const int i = i0 + j * u.nthr;
              yo[j] = -1;
              if (i < total) {
                int l = 1, base = 0;
                for (;;) {
                  const int nl = (u.soff[l * (G + 1) + k + 1] - u.soff[l * (G + 1) + k]) * F4;
                  if (i - base < nl || l == L) break;
                  base += nl;
                  ++l;
                }
                const int idx = i - base, r = idx / F4, f4 = idx - r * F4;
                yo[j] = (l - 1) * N * F + (rows[r] & 0xFFFF) * F + 4 * f4;
                yv[j] = *reinterpret_cast<const float4*>(sl + yo[j]);
                dv[j] = *reinterpret_cast<const float4*>(sl + s_dyoff[l] + r * F + 4 * f4);
              }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              if (yo[j] < 0) continue;
              float4 t = yv[j];
              t.x += dv[j].x;
              t.y += dv[j].y;
              t.z += dv[j].z;
              t.w += dv[j].w;
              *reinterpret_cast<float4*>(sl + yo[j]) = t;
            }
          }
          if (u.tid == 0) {
            int8_t* sp = S.spins + (size_t)s * N;
            const int i = __ldg(b.g.edges + 2 * e), j = __ldg(b.g.edges + 2 * e + 1);
            const int8_t t = sp[i];
            sp[i] = sp[j];
            sp[j] = t;
          }
        }
        unit_sync(u);
        if (u.tid < G && (S.flag[u.tid] & 1)) {
          const int s = u.tid;
          const int64_t k = ++S.step[s];
          int fl = k >= n_steps ? 4 : 0;
          if (a.record_every > 0 && k % N == 0 && (k / N) % a.record_every == 0) fl = 2;
          S.flag[s] = fl;
        }
        unit_sync(u);
      }
      // 5. samples of the chains that completed a recorded sweep
      for (int s = 0; s < G; ++s) {
        if (!(S.flag[s] & 2)) continue;
        const int64_t ch = S.chain[s];
        const int rec = (int)(S.step[s] / N) / a.record_every - 1;
        const int8_t* sp = S.spins + (size_t)s * N;
        if (a.samples_out)
          for (int v = u.tid; v < N; v += u.nthr) a.samples_out[((size_t)rec * a.C + ch) * N + v] = sp[v];
        if (a.logpsi_out) {
          const float* YL = tcm_slot(a, ug, s) + (size_t)(L - 1) * N * F;
          float re = 0.f, im = 0.f;
          for (int i = u.tid; i < N * F; i += u.nthr) {
            const float hv = tanhf(YL[i]);
            const int f = i % F;
            re += hv * c.wr[2 * f];
            im += hv * c.wr[2 * f + 1];
          }
          S.red[2 * u.tid] = (double)re;
          S.red[2 * u.tid + 1] = (double)im;
          unit_sync(u);
          if (u.tid == 0) {
            double zr = 0.0, zi = 0.0;
            for (int t = 0; t < u.nthr; ++t) {
              zr += S.red[2 * t];
              zi += S.red[2 * t + 1];
            }
            int up = 0;
            for (int v = 0; v < N; ++v) up += sp[v] > 0;
            const int dn = N - up;
            a.logpsi_out[((size_t)rec * a.C + ch) * 2] =
                zr + (double)up * c.wr[2 * F] + (double)dn * c.wr[2 * (F + 1)] + (double)c.br[0];
            a.logpsi_out[((size_t)rec * a.C + ch) * 2 + 1] =
                zi + (double)up * c.wr[2 * F + 1] + (double)dn * c.wr[2 * (F + 1) + 1] + (double)c.br[1];
          }
        }
        unit_sync(u);
        if (u.tid == 0) S.flag[s] = S.step[s] >= n_steps ? 4 : 0;
        unit_sync(u);
      }
      if (!s_more[h]) break;
    }
    if (!ok) break;
    // leave the pool: configurations and acceptance counts back
    for (int s = 0; s < G; ++s) {
      const int64_t ch = S.chain[s];
      if (ch < 0) continue;
      for (int v = u.tid; v < N; v += u.nthr) a.chain_spins[ch * N + v] = S.spins[(size_t)s * N + v];
      if (u.tid == 0 && a.n_acc) a.n_acc[ch] += S.acc[s];
    }
    unit_sync(u);
  }
  if (!ok) {
    if (u.tid == 0) {
      atomicOr(&s_tc_status, 1);
      mbar_wait_bounded(u.bar, u.phase ^ 1u);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------------
// Backward VJP on the tensor cores (BF16 models), split operands
// ---------------------------------------------------------------------------------
// grad = sum_x [cot_re,x d Re log Psi_x + cot_im,x d Im log Psi_x] / d theta (the ISGO
// cotangents, Eq. isgo).  The cotangents sum to zero over the batch, so where the
// wavefunction is nearly flat the gradient is a small difference of per-sample derivatives
// that are nearly equal: BF16 rounding of the activations (relative 2^-8 of the full
// derivatives) would cost most of the result.  Every FP32 operand x of a tensor-core product
// is therefore carried as two BF16 values, hi = bf16(x) and lo = bf16(x - hi) (about 16
// significant bits), and the products are accumulated in FP32 in tensor memory; W is a BF16
// model parameter and needs no split.  Activations are kept in FP32 with an accurate tanh.
//
// Per configuration: the forward keeps H^1..H^L (FP32), with H^0 the embedding row of each
// site's spin; then, from G^L_v = cot . w_r[:F] (the same for every site), for l = L..1:
//   dY^l = G^l (1 - (H^l)^2)                                   (SIMT, FP32)
//   dW  += X^T dY^l,  X = [A_hat H^{l-1} ; H^{l-1}]            (MMA: M = rows of X^T (2F, hi
//                                                               and lo stacked when 4F <= 128,
//                                                               else one tile each), N = F,
//                                                               K = sites in chunks of 128;
//                                                               the accumulator stays in TMEM
//                                                               for the whole launch -- W is
//                                                               shared)
//   dX   = dY^l W^T                                             (MMA: M = sites, N = 2F, K = F)
//   G^{l-1}_v = dX_v[F:] + sum_u A_hat_vu dX_u[:F]              (SIMT gather, FP32)
//   db  += sum_v dY^l_v
// and the embedding and readout terms in FP64 shared accumulators.  Per-CTA partials of
// all P parameters (FP64) are summed in a fixed order by a second kernel.
struct TcbArgs {
  TcArgs base;         // graph, dims, theta, spins, B; layout of the shared pieces
  const double* cot;   // [B][2]
  double* partial;     // [grid][P]
  uint32_t oWb, oXt, odYt, osp;  // smem: W as the B operand of dX; X^T and dY^T tiles; FP64 accumulators
  int xt_packed;       // 1: X^T hi in rows [0, 2F) and lo in rows [2F, 4F) of one tile (4F <= 128)
  uint64_t rH, rG, rdx;  // region: H^1..H^L [L][N][F+4], G [N][F] and dX [N][2F] (FP32)
};

// element (r, k) of a K-column tile in the no-swizzle K-major canonical layout
__device__ __forceinline__ uint32_t canon(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// D[tmem] (+)= A[128 x K] B[N x K]^T, one elected thread, no commit.
__device__ __forceinline__ void issue_mma(uint32_t d_tmem, uint32_t a_addr, uint32_t b_addr, int K, int Nout,
                                          bool accumulate) {
  const uint32_t idesc = idesc_bf16(128, Nout);
  const uint32_t sbo = (uint32_t)K * 16;
  for (int kb = 0; kb < K / 16; ++kb)
    mma_bf16(d_tmem, sdesc(a_addr + kb * 256, 128, sbo), sdesc(b_addr + kb * 256, 128, sbo), idesc,
             (accumulate || kb > 0) ? 1u : 0u);
}

// small-parameter accumulators: [W_e (2F), b_e (F)] [b (F)] [w_r (2F+4)] [b_r (2)]
__device__ __forceinline__ int sp_We(int F) { return 0; }
__device__ __forceinline__ int sp_b(int F) { return 3 * F; }
__device__ __forceinline__ int sp_wr(int F) { return 4 * F; }
__device__ __forceinline__ int sp_br(int F) { return 6 * F + 4; }

// FP32 row of layer l-1 of site v: the embedding row of its spin (l = 1), else H^{l-1}.
__device__ __forceinline__ const float* tcb_hrow(const TcCtx& c, const float* Hs, int l, int v) {
  return l == 1 ? c.emb + (c.spin[v] > 0 ? 0 : c.F) : Hs + ((size_t)(l - 2) * c.N + v) * c.ldy;
}

// X = [A_hat H^{l-1} ; H^{l-1}] row chunk (8 features of the message, mc < F/8, or of the
// self term) of site v, FP32.
__device__ __forceinline__ void tcb_xchunk(const TcCtx& c, const float* Hs, int l, int v, int mc, float* x) {
  const int F8 = c.F / 8;
  if (mc < F8) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = 0.f;
    const int k0 = c.rp[v], k1 = c.rp[v + 1];
    for (int k = k0; k < k1; ++k) fma_chunk32(x, c.wfs[k], tcb_hrow(c, Hs, l, __ldg(c.a->g.col + k)) + mc * 8);
  } else {
    const float* h = tcb_hrow(c, Hs, l, v) + (mc - F8) * 8;
    const float4 a = *reinterpret_cast<const float4*>(h), b = *reinterpret_cast<const float4*>(h + 4);
    x[0] = a.x;
    x[1] = a.y;
    x[2] = a.z;
    x[3] = a.w;
    x[4] = b.x;
    x[5] = b.y;
    x[6] = b.z;
    x[7] = b.w;
  }
}

// Commit the MMAs issued by thread 0 and wait for them (bounded); false on timeout.
__device__ __forceinline__ bool tcb_commit_wait(Unit& u, int* fail, uint32_t limit) {
  if (threadIdx.x == 0) {
    mma_commit(u.bar);
    if (!mbar_wait_bounded(u.bar, u.phase, limit)) {
      *fail = 1;
      atomicOr(&s_tc_status, 1);
    }
    u.phase ^= 1u;
  }
  __syncthreads();
  tc_fence_after();
  return *fail == 0;
}

// Forward of the configuration in c.spin with split operands: H^1..H^L into Hs (FP32).
__device__ bool tcb_forward(const TcCtx& c, Unit& u, float* Hs) {
  const int N = c.N, F = c.F, L = c.L, ldy = c.ldy, F8 = F / 8;
  const uint32_t a_hi = smem_u32(u.A), a_lo = a_hi + 128u * 4u * (uint32_t)F, wt = smem_u32(c.Wt);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q4 = warp & 3, wg = warp >> 2;
  for (int l = 1; l <= L; ++l) {
    float* Hn = Hs + (size_t)(l - 1) * N * ldy;
    for (int r0 = 0; r0 < N; r0 += 128) {
      const int R = min(128, N - r0);
      for (int idx = threadIdx.x; idx < R * 2 * F8; idx += blockDim.x) {
        const int q = idx / (2 * F8), mc = idx - q * (2 * F8);
        float x[8];
        tcb_xchunk(c, Hs, l, r0 + q, mc, x);
        uint4 hi, lo;
        split_hi_lo(x, hi, lo);
        *reinterpret_cast<uint4*>(u.A + canon(q, mc * 8, 2 * F)) = hi;
        *reinterpret_cast<uint4*>(u.A + 128 * 4 * F + canon(q, mc * 8, 2 * F)) = lo;
      }
      fence_proxy_async();
      __syncthreads();
      if (threadIdx.x == 0) {
        tc_fence_after();
        issue_mma(u.tbase, a_hi, wt, 2 * F, F, false);
        issue_mma(u.tbase, a_lo, wt, 2 * F, F, true);
      }
      if (!tcb_commit_wait(u, c.fail, c.a->wait_limit)) return false;
      const int q = q4 * 32 + lane;
      for (int ch = wg; ch < F8; ch += u.nwg) {
        float v[8];
        tmem_ld8(u.tbase + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(ch * 8), v);
        if (q < R) {
          float* o = Hn + (size_t)(r0 + q) * ldy + ch * 8;
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = tanhf(v[i] + c.bias[ch * 8 + i]);
          reinterpret_cast<float4*>(o)[0] = make_float4(v[0], v[1], v[2], v[3]);
          reinterpret_cast<float4*>(o)[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  return true;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_bwd(const TcbArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_fail;
  const TcArgs& b = a.base;
  TcCtx c;
  c.a = &b;
  c.N = b.m.N;
  c.F = b.m.F;
  c.L = b.m.L;
  c.E = b.m.E;
  c.T = b.lay.T;
  c.G = b.lay.G;
  c.ldh = b.m.F + 8;
  c.ldy = b.m.F + 4;
  c.Wt = (__nv_bfloat16*)(smem + b.lay.oWt);
  c.bias = (float*)(smem + b.lay.obias);
  c.emb = (float*)(smem + b.lay.oemb);
  c.wr = (float*)(smem + b.lay.owr);
  c.br = (float*)(smem + b.lay.obr);
  c.spin = (int8_t*)(smem + b.lay.ospin);
  c.rp = (const int*)(smem + b.lay.orp);
  c.wfs = (const float*)(smem + b.lay.owf);
  c.list = (int*)(smem + b.lay.oint);
  c.sdbl = (double*)(smem + b.lay.odbl);
  c.region = b.region_in_smem ? smem + b.lay.oregion : b.gregion + (size_t)blockIdx.x * b.lay.region_bytes;
  c.ycache = nullptr;  // the backward keeps its own FP32 layers
  c.fail = &s_fail;
  const int F = c.F, N = c.N, L = c.L, ldy = c.ldy;
  const int F8 = F / 8, F2 = 2 * F;
  const Dims& m = b.m;
  const float* th = b.theta;
  uint64_t* bars = (uint64_t*)(smem + b.lay.obar);
  uint32_t* slot = (uint32_t*)(smem + b.lay.oslot);
  unsigned char* Wb = smem + a.oWb;
  unsigned char* Xt = smem + a.oXt;
  unsigned char* dYt = smem + a.odYt;
  double* sp = (double*)(smem + a.osp);
  float* Hs = (float*)(c.region + a.rH);
  float* Gs = (float*)(c.region + a.rG);
  float* dx = (float*)(c.region + a.rdx);
  const int nsp = 6 * F + 6;
  const int packed = a.xt_packed;
  // X^T lo rows: below the hi rows in the same tile, or in a second tile
  unsigned char* Xlo = packed ? Xt : Xt + 128 * 128 * 2;
  const int xlo_row = packed ? F2 : 0;
  unsigned char* dYlo = dYt + F * 128 * 2;

  if (threadIdx.x == 0) {
    s_fail = 0;
    mbar_init(bars, 1);
  }
  if ((threadIdx.x >> 5) == 0) {
    tmem_alloc(slot, kTmemCols);
    tmem_relinquish();
  }
  const float* W = th + m.oW;
  for (int i = threadIdx.x; i < F * F2; i += blockDim.x) {
    const int n = i / F2, k = i % F2;  // forward B: W^T (n = output, k = input)
    const __nv_bfloat16 w = __float2bfloat16_rn(W[(size_t)k * F + n]);
    *reinterpret_cast<__nv_bfloat16*>((unsigned char*)c.Wt + canon(n, k, F2)) = w;
    // backward dX: B = W (n' = input feature k, k' = output feature n), K = F
    *reinterpret_cast<__nv_bfloat16*>(Wb + canon(k, n, F)) = w;
  }
  for (int i = threadIdx.x; i < F; i += blockDim.x) c.bias[i] = th[m.ob + i];
  for (int i = threadIdx.x; i < 2 * F; i += blockDim.x) c.emb[i] = tanhf(th[m.oWe + i] + th[m.obe + i % F]);
  for (int i = threadIdx.x; i < (F + 2) * 2; i += blockDim.x) c.wr[i] = th[m.owr + i];
  if (threadIdx.x < 2) c.br[threadIdx.x] = th[m.obr + threadIdx.x];
  for (int i = threadIdx.x; i <= c.N; i += blockDim.x) ((int*)c.rp)[i] = __ldg(b.g.row_ptr + i);
  for (int i = threadIdx.x; i < 2 * c.E; i += blockDim.x) ((float*)c.wfs)[i] = __ldg(b.g.wf + i);
  for (int i = threadIdx.x; i < nsp; i += blockDim.x) sp[i] = 0.0;
  // rows of X^T past the stacked hi and lo rows stay zero (M is 128)
  for (int i = threadIdx.x; i < (packed ? 1 : 2) * 128 * 128 * 2 / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(Xt)[i] = make_uint4(0, 0, 0, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t t_dx = tmem + (uint32_t)F, t_dw = tmem + (uint32_t)(3 * F);

  Unit u;
  u.tid = threadIdx.x;
  u.nthr = blockDim.x;
  u.bar_id = 0;
  u.nwg = blockDim.x / 128;
  u.A = smem + b.lay.oA;
  u.tbase = tmem;
  u.bar = bars;
  u.phase = 0;
  const uint32_t a_hi = smem_u32(u.A), a_lo = a_hi + 128u * 2u * (uint32_t)F;  // dY rows, K = F
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q4 = warp & 3, wg = warp >> 2;
  bool dw_started = false;  // meaningful in thread 0
  bool ok = true;
  int nsamples = 0;
  for (int64_t bi = blockIdx.x; bi < b.B && ok; bi += gridDim.x) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) c.spin[i] = b.spins[bi * N + i];
    __syncthreads();
    ok = tcb_forward(c, u, Hs);
    if (!ok) break;
    ++nsamples;
    const float c0 = (float)a.cot[2 * bi], c1 = (float)a.cot[2 * bi + 1];
    // readout: d w_r[f] += cot z_f with z = sum_v [H^L_v ; onehot_v]; d b_r += cot.  The
    // column sums over sites run on the whole block: P interleaved site strides per feature,
    // their FP32 partials (in the free dX buffer) added in a fixed order
    const float* HL = Hs + (size_t)(L - 1) * N * ldy;
    const int P = min((int)blockDim.x / F, N), fcol = threadIdx.x % F, part = threadIdx.x / F;
    if (part < P) {
      float zz = 0.f;
      for (int v = part; v < N; v += P) zz += HL[(size_t)v * ldy + fcol];
      dx[part * F + fcol] = zz;
    }
    __syncthreads();
    if (threadIdx.x < F + 2) {
      const int f = threadIdx.x;
      double z = 0.0;
      if (f < F) {
        float zz = 0.f;
        for (int q = 0; q < P; ++q) zz += dx[q * F + f];
        z = (double)zz;
      } else {
        int cnt = 0;
        for (int v = 0; v < N; ++v) cnt += (f == F) ? (c.spin[v] > 0) : (c.spin[v] < 0);
        z = (double)cnt;
      }
      sp[sp_wr(F) + 2 * f] += (double)c0 * z;
      sp[sp_wr(F) + 2 * f + 1] += (double)c1 * z;
    }
    if (threadIdx.x == 0) {
      sp[sp_br(F)] += (double)c0;
      sp[sp_br(F) + 1] += (double)c1;
    }
    for (int i = threadIdx.x; i < N * F; i += blockDim.x) {
      const int f = i % F;
      Gs[i] = c0 * c.wr[2 * f] + c1 * c.wr[2 * f + 1];
    }
    __syncthreads();
    for (int l = L; l >= 1 && ok; --l) {
      const float* Hl = Hs + (size_t)(l - 1) * N * ldy;
      // db += sum_v dY^l_v (block-wide column sums as for the readout; dX is free here)
      if (part < P) {
        float sum = 0.f;
        for (int v = part; v < N; v += P) {
          const float h = Hl[(size_t)v * ldy + fcol];
          sum += Gs[(size_t)v * F + fcol] * fmaf(-h, h, 1.f);
        }
        dx[part * F + fcol] = sum;
      }
      __syncthreads();
      if (threadIdx.x < F) {
        float sum = 0.f;
        for (int q = 0; q < P; ++q) sum += dx[q * F + threadIdx.x];
        sp[sp_b(F) + threadIdx.x] += (double)sum;
      }
      for (int c0s = 0; c0s < N && ok; c0s += 128) {
        const int ns = min(128, N - c0s);
        // dY rows of the chunk, hi and lo: as the A operands of dX (rows, K = F) and,
        // transposed, as the B operands of dW (rows = output features, K = sites); zeros past
        // the last site
        if (F8 % 4 == 0) {
          // F a multiple of 32: as for X^T below, a warp takes 8 sites x 4 chunks and writes
          // the transposed rows 16 bytes at a time after an 8 x 8 shuffle transpose
          const int ncg = F8 / 4, nwi = 16 * ncg, nwarps = (int)blockDim.x >> 5;
          const int j = lane & 7, cc = lane >> 3;
          for (int wi = warp; wi < nwi; wi += nwarps) {
            const int sg = wi / ncg, ch = (wi - sg * ncg) * 4 + cc, r = sg * 8 + j, v = c0s + r;
            float d[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (r < ns) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float h = Hl[(size_t)v * ldy + ch * 8 + i];
                d[i] = Gs[(size_t)v * F + ch * 8 + i] * fmaf(-h, h, 1.f);
              }
            }
            uint4 hi, lo;
            split_hi_lo(d, hi, lo);
            *reinterpret_cast<uint4*>(u.A + canon(r, ch * 8, F)) = hi;
            *reinterpret_cast<uint4*>(u.A + 128 * 2 * F + canon(r, ch * 8, F)) = lo;
#pragma unroll
            for (int st = 1; st < 8; st <<= 1) {
              const bool up = (j & st) != 0;
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                if (k & st) continue;
                const float got = __shfl_xor_sync(0xffffffffu, up ? d[k] : d[k | st], st);
                if (up)
                  d[k] = got;
                else
                  d[k | st] = got;
              }
            }
            // this lane: output feature ch * 8 + j of sites sg * 8 .. sg * 8 + 7
            split_hi_lo(d, hi, lo);
            *reinterpret_cast<uint4*>(dYt + canon(ch * 8 + j, sg * 8, 128)) = hi;
            *reinterpret_cast<uint4*>(dYlo + canon(ch * 8 + j, sg * 8, 128)) = lo;
          }
        } else {
          for (int idx = threadIdx.x; idx < 128 * F8; idx += blockDim.x) {
            const int r = idx / F8, ch = idx - r * F8, v = c0s + r;
            float d[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (r < ns) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float h = Hl[(size_t)v * ldy + ch * 8 + i];
                d[i] = Gs[(size_t)v * F + ch * 8 + i] * fmaf(-h, h, 1.f);
              }
            }
            uint4 hi, lo;
            split_hi_lo(d, hi, lo);
            *reinterpret_cast<uint4*>(u.A + canon(r, ch * 8, F)) = hi;
            *reinterpret_cast<uint4*>(u.A + 128 * 2 * F + canon(r, ch * 8, F)) = lo;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              __nv_bfloat16 h, l2;
              split1(d[i], h, l2);
              *reinterpret_cast<__nv_bfloat16*>(dYt + canon(ch * 8 + i, r, 128)) = h;
              *reinterpret_cast<__nv_bfloat16*>(dYlo + canon(ch * 8 + i, r, 128)) = l2;
            }
          }
        }
        // X = [A_hat H^{l-1} ; H^{l-1}] of the chunk's sites, transposed (rows = input
        // features), hi and lo.  A warp takes 8 sites x 4 feature chunks: each lane gathers
        // the 8 features of one (site, chunk), the 8 lanes of a chunk transpose their 8 x 8
        // block with shuffles (three butterfly stages), and each lane then stores one
        // feature's 8 consecutive sites as 16 bytes (2F is a multiple of 32 features)
        {
          const int ncg = (2 * F8) / 4, nwi = 16 * ncg, nwarps = (int)blockDim.x >> 5;
          const int j = lane & 7, cc = lane >> 3;
          for (int wi = warp; wi < nwi; wi += nwarps) {
            const int sg = wi / ncg, mc = (wi - sg * ncg) * 4 + cc, r = sg * 8 + j;
            float x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (r < ns) tcb_xchunk(c, Hs, l, c0s + r, mc, x);
#pragma unroll
            for (int st = 1; st < 8; st <<= 1) {
              const bool up = (j & st) != 0;
#pragma unroll
              for (int k = 0; k < 8; ++k) {
                if (k & st) continue;
                const float got = __shfl_xor_sync(0xffffffffu, up ? x[k] : x[k | st], st);
                if (up)
                  x[k] = got;
                else
                  x[k | st] = got;
              }
            }
            // this lane: feature mc * 8 + j of sites sg * 8 .. sg * 8 + 7
            uint4 hi, lo;
            split_hi_lo(x, hi, lo);
            *reinterpret_cast<uint4*>(Xt + canon(mc * 8 + j, sg * 8, 128)) = hi;
            *reinterpret_cast<uint4*>(Xlo + canon(xlo_row + mc * 8 + j, sg * 8, 128)) = lo;
          }
        }
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
          tc_fence_after();
          const uint32_t xt = smem_u32(Xt), yh = smem_u32(dYt), yl = smem_u32(dYlo);
          // dW: packed tile rows [0, 2F) = X_hi^T (dY_hi + dY_lo), rows [2F, 4F) = X_lo^T (dY_hi
          // + dY_lo), summed at the end; separate tiles: X_hi^T dY_hi + X_hi^T dY_lo + X_lo^T dY_hi
          issue_mma(t_dw, xt, yh, 128, F, dw_started);
          issue_mma(t_dw, xt, yl, 128, F, true);
          if (!packed) issue_mma(t_dw, smem_u32(Xlo), yh, 128, F, true);
          dw_started = true;
          issue_mma(t_dx, a_hi, smem_u32(Wb), F, F2, false);
          issue_mma(t_dx, a_lo, smem_u32(Wb), F, F2, true);
        }
        if (!tcb_commit_wait(u, c.fail, c.a->wait_limit)) {
          ok = false;
          break;
        }
        // dX rows of the chunk out of TMEM (lanes = sites)
        const int r = q4 * 32 + lane;
        for (int ch = wg; ch < 2 * F8; ch += u.nwg) {
          float v8[8];
          tmem_ld8(t_dx + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(ch * 8), v8);
          if (r < ns) {
            float4* o = reinterpret_cast<float4*>(dx + (size_t)(c0s + r) * F2 + ch * 8);
            o[0] = make_float4(v8[0], v8[1], v8[2], v8[3]);
            o[1] = make_float4(v8[4], v8[5], v8[6], v8[7]);
          }
        }
        tc_fence_before();
        __syncthreads();
      }
      if (!ok) break;
      // G^{l-1}_v = dX_v[F:] + sum_u A_hat_vu dX_u[:F]
      for (int idx = threadIdx.x; idx < N * F8; idx += blockDim.x) {
        const int v = idx / F8, ch = idx - v * F8;
        float acc[8];
        const float4* sf = reinterpret_cast<const float4*>(dx + (size_t)v * F2 + F + ch * 8);
        const float4 s0 = sf[0], s1 = sf[1];
        acc[0] = s0.x;
        acc[1] = s0.y;
        acc[2] = s0.z;
        acc[3] = s0.w;
        acc[4] = s1.x;
        acc[5] = s1.y;
        acc[6] = s1.z;
        acc[7] = s1.w;
        const int k0 = c.rp[v], k1 = c.rp[v + 1];
        for (int k = k0; k < k1; ++k) fma_chunk32(acc, c.wfs[k], dx + (size_t)__ldg(b.g.col + k) * F2 + ch * 8);
        float4* go = reinterpret_cast<float4*>(Gs + (size_t)v * F + ch * 8);
        go[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        go[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
      }
      __syncthreads();
    }
    if (!ok) break;
    // embedding: dY^0 = G^0 (1 - emb^2); d W_e[c] += sum_{v: c_v = c} dY^0_v, d b_e += sum_v dY^0_v
    // (block-wide column sums of the up and the down sites, partials in the free dX buffer)
    if (part < P) {
      float su = 0.f, sd = 0.f;
      for (int v = part; v < N; v += P) {
        if (c.spin[v] > 0)
          su += Gs[(size_t)v * F + fcol];
        else
          sd += Gs[(size_t)v * F + fcol];
      }
      dx[part * F + fcol] = su;
      dx[(P + part) * F + fcol] = sd;
    }
    __syncthreads();
    for (int f = threadIdx.x; f < F; f += blockDim.x) {
      float su = 0.f, sd = 0.f;
      for (int q = 0; q < P; ++q) {
        su += dx[q * F + f];
        sd += dx[(P + q) * F + f];
      }
      const float eu = c.emb[f], ed = c.emb[F + f];
      const double du = (double)(su * fmaf(-eu, eu, 1.f)), dd = (double)(sd * fmaf(-ed, ed, 1.f));
      sp[sp_We(F) + f] += du;
      sp[sp_We(F) + F + f] += dd;
      sp[sp_We(F) + 2 * F + f] += du + dd;
    }
    __syncthreads();
  }
  // partials: dW from TMEM (lanes = rows of X^T: input features, hi then lo when packed), the
  // rest from the FP64 accumulators
  double* part = a.partial + (size_t)blockIdx.x * m.P;
  if (ok) {
    const int mrow = q4 * 32 + lane;
    float* lo_rows = dx;  // [2F][F] the packed lo rows' sums, added to the hi rows below
    for (int ch = wg; ch < F8; ch += u.nwg) {
      float v8[8];
      tmem_ld8(t_dw + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(ch * 8), v8);
      if (packed && mrow >= F2 && mrow < 2 * F2)
#pragma unroll
        for (int i = 0; i < 8; ++i) lo_rows[(size_t)(mrow - F2) * F + ch * 8 + i] = v8[i];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    for (int ch = wg; ch < F8; ch += u.nwg) {
      float v8[8];
      tmem_ld8(t_dw + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(ch * 8), v8);
      if (mrow < F2)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const double lo = packed ? (double)lo_rows[(size_t)mrow * F + ch * 8 + i] : 0.0;
          part[m.oW + (size_t)mrow * F + ch * 8 + i] = nsamples > 0 ? (double)v8[i] + lo : 0.0;
        }
    }
    for (int f = threadIdx.x; f < 3 * F; f += blockDim.x) part[m.oWe + f] = sp[sp_We(F) + f];  // W_e, b_e
    for (int f = threadIdx.x; f < F; f += blockDim.x) part[m.ob + f] = sp[sp_b(F) + f];
    for (int f = threadIdx.x; f < 2 * F + 4; f += blockDim.x) part[m.owr + f] = sp[sp_wr(F) + f];
    if (threadIdx.x < 2) part[m.obr + threadIdx.x] = sp[sp_br(F) + threadIdx.x];
  }
  if (!ok && threadIdx.x == 0) mbar_wait_bounded(u.bar, u.phase ^ 1u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, kTmemCols);
}

__global__ void k_tcb_reduce(const double* partial, int grid, int P, double* grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double s = 0.0;
  for (int cta = 0; cta < grid; ++cta) s += partial[(size_t)cta * P + p];
  grad[p] = s;
  if (!isfinite(s)) atomicOr(&s_tc_status, 2);
}

// ---------------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------------
// Iterations of the MMA waits of the kernels launched from now on (kWaitLimit; tests may
// shorten it to exercise the timeout path).
static std::atomic<uint32_t> g_wait_limit{kWaitLimit};
void set_wait_limit(uint32_t iters) { g_wait_limit.store(iters == UINT32_MAX ? kWaitLimit : iters); }
static uint32_t wait_limit() { return g_wait_limit.load(); }

struct TcPlan {
  TcLayout lay;
  int grid = 0;
  int region_in_smem = 0;
  size_t ws_bytes = 0;
};

static gna_status tc_plan(const gna_graph* g, const Dims& m, int op, int64_t B, TcPlan* p, int* maxball, int split) {
  if (m.F % 16 != 0 || m.F > 64 || m.L < 1 || !m.shared || !g->pack_ok) return GNA_ERR_UNSUPPORTED;
  DeviceInfo di;
  gna_status st = device_info(&di);
  if (st != GNA_OK) return st;
  if (di.cc < 100) return GNA_ERR_UNSUPPORTED;
  for (int l = 0; l <= kMaxL; ++l) maxball[l] = (l <= m.L && l <= g->d.Lmax) ? g->max_ball[l] : 0;
  const int maxspan = g->max_span[m.L];
  const int T = tc_tiles_per_unit(m.F);
  if (tc_units(m.F, split) * T * m.F > kTmemCols) return GNA_ERR_UNSUPPORTED;
  const size_t budget = (size_t)di.smem_optin - 2048;
  // bonds per group: as many as fill the T tiles at the last layer in one pass; a layer with
  // more rows runs in several passes
  int G = op == TC_ELOC ? (T * 128) / (maxball[m.L] > 0 ? maxball[m.L] : 1) : 1;
  if (G > 16) G = 16;
  if (G < 1) G = 1;
  TcLayout lay;
  // prefer the whole region in shared memory with as many bonds per group as fit (the dH
  // rows reuse the layer cache's space where they fit in it)
  // the group size with the fewest passes per bond (ties: the larger) among those that fit
  // (with the Y cache in shared memory; moved to the workspace only when that allows
  // strictly fewer passes per bond -- BF16X2 at Kagome 108: 7 bonds instead of 4)
  int g_fit = 0, best = 1 << 30, y_glob = 0;
  for (int yg = 0; yg <= (op == TC_ELOC ? 1 : 0); ++yg) {
    for (int gg = op == TC_ELOC ? 16 : 1; gg >= 1; --gg) {
      tc_layout(m, maxball, maxspan, gg, 1, op == TC_ELOC, &lay, split, yg);
      if (lay.smem_total > budget) continue;
      const int cost = tc_passes_per_bond(maxball, m.L, gg, T * 128);
      if (cost < best) {
        best = cost;
        g_fit = gg;
        y_glob = yg;
      }
    }
  }
  if (g_fit > 0) {
    p->region_in_smem = 1;
    tc_layout(m, maxball, maxspan, g_fit, 1, op == TC_ELOC, &lay, split, y_glob);
  } else {
    // region in the workspace: the group size by the same cost model among those that fit,
    // up to 8 bonds (larger groups spill the per-CTA regions out of L2: triangular 144,
    // F = 48: 8 bonds 36.8 ms, 16 bonds 42.6 ms per 4096 configurations)
    int Gg = 0;
    for (int gg = op == TC_ELOC ? 8 : 1; gg >= 1; --gg) {
      tc_layout(m, maxball, maxspan, gg, 0, op == TC_ELOC, &lay, split);
      if (lay.smem_total > budget) continue;
      const int cost = tc_passes_per_bond(maxball, m.L, gg, T * 128);
      if (cost < best) {
        best = cost;
        Gg = gg;
      }
    }
    if (Gg < 1) return GNA_ERR_UNSUPPORTED;
    tc_layout(m, maxball, maxspan, Gg, 0, op == TC_ELOC, &lay, split);
    p->region_in_smem = 0;
  }
  // At most 512 / kTmemCols CTAs may hold TMEM on one SM at a time: request enough shared
  // memory that no more than that many are resident.
  const uint32_t min_smem = (uint32_t)(228u * 1024u / (512 / kTmemCols + 1)) + 1024u;
  if (lay.smem_total < min_smem) lay.smem_total = min_smem;
  p->lay = lay;
  const void* kfn = split ? (const void*)k_tc<true> : (const void*)k_tc<false>;
  GNA_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.smem_total));
  int occ = 0;
  GNA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kTcThreads, lay.smem_total));
  if (occ < 1) occ = 1;
  if (occ * kTmemCols > 512) return GNA_ERR_UNSUPPORTED;
  int64_t grid = (int64_t)di.sms * occ;
  if (grid > B) grid = B;
  if (grid < 1) grid = 1;
  p->grid = (int)grid;
  p->ws_bytes = (p->region_in_smem ? 0 : align_up((size_t)grid * lay.region_bytes)) +
                (lay.y_global ? align_up((size_t)grid * lay.y_bytes) : 0) +
                (op == TC_ELOC ? align_up((size_t)grid * m.N * (m.F + 4) * sizeof(float)) : 0);  // H^L for log Psi
  return GNA_OK;
}

gna_status tc_workspace(const gna_graph* g, const Dims& m, int op, int64_t B, size_t* bytes, int split) {
  if (B == 0) {
    *bytes = 0;
    return GNA_OK;
  }
  TcPlan p;
  int maxball[kMaxL + 1];
  gna_status st = tc_plan(g, m, op, B, &p, maxball, split);
  if (st != GNA_OK) return st;
  *bytes = p.ws_bytes;
  return GNA_OK;
}

gna_status tc_run(const TcCall& call, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (call.B == 0) return GNA_OK;
  TcPlan p;
  TcArgs a;
  gna_status st = tc_plan(call.g, call.m, call.op, call.B, &p, a.maxball, call.split);
  if (st != GNA_OK) return st;
  if (ws_bytes < p.ws_bytes || (p.ws_bytes > 0 && !ws)) return GNA_ERR_WORKSPACE;
  a.g = call.g->d;
  a.m = call.m;
  a.op = call.op;
  a.lay = p.lay;
  a.theta = call.theta;
  a.spins = call.spins;
  a.B = call.B;
  a.logpsi = call.logpsi;
  a.eloc = call.eloc;
  a.dlogpsi = call.dlogpsi;
  a.gregion = (unsigned char*)ws;
  const size_t region_ws = p.region_in_smem ? 0 : align_up((size_t)p.grid * p.lay.region_bytes);
  a.gY = (float*)((unsigned char*)ws + region_ws);
  a.gH = (float*)((unsigned char*)ws + region_ws + (p.lay.y_global ? align_up((size_t)p.grid * p.lay.y_bytes) : 0));
  a.region_in_smem = p.region_in_smem;
  a.wait_limit = wait_limit();
  if (call.split)
    k_tc<true><<<p.grid, kTcThreads, p.lay.smem_total, stream>>>(a);
  else
    k_tc<false><<<p.grid, kTcThreads, p.lay.smem_total, stream>>>(a);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

// ---------------------------------------------------------------------------------
// host: tensor-core sampler
// ---------------------------------------------------------------------------------
struct TcmPlan {
  TcLayout lay;
  int grid = 0;
  int new16_in_smem = 1;
  uint64_t slot_elems = 0, unit_elems = 0;
  uint64_t dy_off[kMaxL + 1] = {0};
  size_t ws_bytes = 0;
};

// new16_in_smem = 0: the units' dH rows live in the workspace (after each unit's H scratch).
static void tcm_layout(const Dims& m, const int* maxball, int maxspan, int G, int new16_in_smem, TcLayout* t) {
  const int F = m.F, N = m.N, L = m.L;
  memset(t, 0, sizeof(*t));
  uint64_t o = 0;
  auto take = [&](uint64_t bytes, uint64_t align) {
    o = (o + align - 1) / align * align;
    uint64_t r = o;
    o += bytes;
    return (uint32_t)r;
  };
  t->T = tc_tiles_per_unit(F);
  t->units = tcm_units(F);
  const int U = t->units, unit_threads = kTcThreads / U;
  t->G = G;
  t->a_unit = (uint32_t)t->T * 128 * 2 * F * 2;
  t->oWt = take((uint64_t)F * 2 * F * 2, 1024);
  t->oA = take((uint64_t)U * t->a_unit, 1024);
  t->obias = take(F * 4, 16);
  t->oemb = take(2 * F * 4, 16);
  t->owr = take((F + 2) * 2 * 4, 16);
  t->obr = take(16, 16);
  t->int_unit = (uint32_t)(3 * G + (L + 2) * (G + 1) + 4);
  t->oint = take((uint64_t)U * t->int_unit * 4, 16);
  t->dbl_unit = (uint32_t)(2 * G + 4);
  t->odbl = take((uint64_t)U * t->dbl_unit * 8, 16);
  t->obar = take(8 * U, 8);
  t->oslot = take(4, 4);
  tc_stage_layout(m, maxball, maxspan, G, U, o, t);
  uint64_t r = 0;
  auto rtake = [&](uint64_t bytes) {
    r = (r + 15) / 16 * 16;
    uint64_t x = r;
    r += bytes;
    return x;
  };
  const uint64_t ldh = F + 8;
  uint64_t n16 = 0;
  for (int l = 0; l < L; ++l) {
    t->new16_off[l] = n16;
    n16 += (uint64_t)G * maxball[l] * ldh * 2;
  }
  t->new16_unit = (n16 + 15) / 16 * 16;
  t->rnew16 = new16_in_smem ? rtake((uint64_t)U * t->new16_unit) : 0;
  t->part_rows = G * maxball[L];
  t->part_unit = (uint64_t)(unit_threads / 128) * t->part_rows * 2 * 4;
  t->rpart = rtake((uint64_t)U * t->part_unit);
  t->state_unit = tcm_state_bytes(G, N, unit_threads);
  t->rstate = rtake((uint64_t)U * t->state_unit);
  t->region_bytes = (r + 255) / 256 * 256;
  t->oregion = take(t->region_bytes, 16);
  t->smem_total = (uint32_t)o;
}

static gna_status tcm_plan(const gna_graph* g, const Dims& m, int64_t C, TcmPlan* p, int* maxball) {
  if (m.F % 16 != 0 || m.F > 64 || m.L < 1 || !m.shared || !g->pack_ok) return GNA_ERR_UNSUPPORTED;
  DeviceInfo di;
  gna_status st = device_info(&di);
  if (st != GNA_OK) return st;
  if (di.cc < 100) return GNA_ERR_UNSUPPORTED;
  for (int l = 0; l <= kMaxL; ++l) maxball[l] = (l <= m.L && l <= g->d.Lmax) ? g->max_ball[l] : 0;
  const int maxspan = g->max_span[m.L];
  const int T = tc_tiles_per_unit(m.F), U = tcm_units(m.F);
  if (U * T * m.F > kTmemCols) return GNA_ERR_UNSUPPORTED;
  // pool size: up to 8 chains with their dH rows in shared memory; when fewer than 4 fit
  // there, pools of 8 with the dH rows in the workspace (deep layers then take several
  // passes either way)
  const size_t budget = (size_t)di.smem_optin - 2048;
  TcLayout lay;
  int in_smem = 1;
  int G = 0;
  for (; in_smem >= 0; --in_smem) {
    int best = 1 << 30;
    G = 0;
    for (int gg = 8; gg >= (in_smem ? 4 : 1); --gg) {
      tcm_layout(m, maxball, maxspan, gg, in_smem, &lay);
      if (lay.smem_total > budget) continue;
      const int cost = tc_passes_per_bond(maxball, m.L, gg, T * 128);
      if (cost < best) {
        best = cost;
        G = gg;
      }
    }
    if (G >= 1) {
      tcm_layout(m, maxball, maxspan, G, in_smem, &lay);
      break;
    }
  }
  if (G < 1) return GNA_ERR_UNSUPPORTED;
  p->new16_in_smem = in_smem;
  const uint32_t min_smem = (uint32_t)(228u * 1024u / (512 / kTmemCols + 1)) + 1024u;
  if (lay.smem_total < min_smem) lay.smem_total = min_smem;
  p->lay = lay;
  GNA_CUDA_TRY(cudaFuncSetAttribute((const void*)k_tc_metro, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)lay.smem_total));
  int occ = 0;
  GNA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_tc_metro, kTcThreads, lay.smem_total));
  if (occ < 1) occ = 1;
  if (occ * kTmemCols > 512) return GNA_ERR_UNSUPPORTED;
  const int64_t pools = (C + G - 1) / G;
  int64_t grid = (int64_t)di.sms * occ;
  if (grid * U > pools) grid = (pools + U - 1) / U;
  if (grid < 1) grid = 1;
  p->grid = (int)grid;
  const uint64_t NF = (uint64_t)m.N * m.F;
  uint64_t e = (uint64_t)m.L * NF;
  for (int l = 1; l <= m.L; ++l) {
    p->dy_off[l] = e;
    e += (uint64_t)maxball[l] * m.F;
  }
  p->slot_elems = (e + 3) / 4 * 4;
  p->unit_elems = (uint64_t)G * p->slot_elems + (uint64_t)m.N * (m.F + 8);  // + two BF16 H layers
  if (!in_smem) p->unit_elems += lay.new16_unit / sizeof(float);           // + the dH rows
  p->ws_bytes = align_up((size_t)grid * U * p->unit_elems * sizeof(float));
  return GNA_OK;
}

gna_status tcm_workspace(const gna_graph* g, const Dims& m, int64_t C, size_t* bytes) {
  if (C == 0) {
    *bytes = 0;
    return GNA_OK;
  }
  TcmPlan p;
  int maxball[kMaxL + 1];
  gna_status st = tcm_plan(g, m, C, &p, maxball);
  if (st != GNA_OK) return st;
  *bytes = p.ws_bytes;
  return GNA_OK;
}

gna_status tcm_run(const TcmCall& call, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (call.C == 0 || call.n_sweeps == 0) return GNA_OK;
  TcmPlan p;
  TcmArgs a;
  memset(&a, 0, sizeof(a));
  gna_status st = tcm_plan(call.g, call.m, call.C, &p, a.base.maxball);
  if (st != GNA_OK) return st;
  if (ws_bytes < p.ws_bytes || !ws) return GNA_ERR_WORKSPACE;
  a.base.g = call.g->d;
  a.base.m = call.m;
  a.base.op = TC_ELOC;
  a.base.lay = p.lay;
  a.base.theta = call.theta;
  a.base.region_in_smem = p.new16_in_smem;  // here: where the units' dH rows live
  a.base.wait_limit = wait_limit();
  a.chain_spins = call.chain_spins;
  a.C = call.C;
  a.n_sweeps = call.n_sweeps;
  a.record_every = call.record_every;
  a.seed = call.seed;
  a.step0 = call.step0;
  a.samples_out = call.samples_out;
  a.logpsi_out = call.logpsi_out;
  a.n_acc = call.n_acc;
  a.trace = call.trace;
  a.gws = (float*)ws;
  a.slot_elems = p.slot_elems;
  a.unit_elems = p.unit_elems;
  for (int l = 0; l <= kMaxL; ++l) a.dy_off[l] = p.dy_off[l];
  k_tc_metro<<<p.grid, kTcThreads, p.lay.smem_total, stream>>>(a);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

// ---------------------------------------------------------------------------------
// host: tensor-core backward
// ---------------------------------------------------------------------------------
struct TcbPlan {
  TcbArgs a;
  int grid = 0;
  size_t smem = 0, ws_bytes = 0, partial_bytes = 0;
};

static void tcb_layout(const Dims& m, int region_in_smem, TcbArgs* A) {
  TcLayout* t = &A->base.lay;
  memset(t, 0, sizeof(*t));
  const int F = m.F, N = m.N, L = m.L;
  uint64_t o = 0;
  auto take = [&](uint64_t bytes, uint64_t align) {
    o = (o + align - 1) / align * align;
    uint64_t r = o;
    o += bytes;
    return (uint32_t)r;
  };
  t->T = 1;
  t->units = 1;
  t->G = 1;
  // A operands: the forward's hi and lo tiles of 128 rows x 2F (the backward's dY tiles,
  // 128 x F each, use the same space)
  t->a_unit = 2 * 128 * 2 * F * 2;
  A->xt_packed = 4 * F <= 128;
  t->oWt = take((uint64_t)F * 2 * F * 2, 1024);
  A->oWb = take((uint64_t)2 * F * F * 2, 1024);
  t->oA = take(t->a_unit, 1024);
  A->oXt = take((uint64_t)(A->xt_packed ? 1 : 2) * 128 * 128 * 2, 1024);
  A->odYt = take((uint64_t)2 * F * 128 * 2, 1024);
  t->obias = take(F * 4, 16);
  t->oemb = take(2 * F * 4, 16);
  t->owr = take((F + 2) * 2 * 4, 16);
  t->obr = take(16, 16);
  t->ospin = take(N, 16);
  t->oint = take(64, 16);
  t->odbl = take((uint64_t)(16 + kTcThreads + 16) * 8, 16);
  A->osp = take((uint64_t)(6 * F + 6) * 8, 16);
  t->obar = take(8, 8);
  t->oslot = take(4, 4);
  t->orp = take((uint64_t)(N + 1) * 4, 16);
  t->owf = take((uint64_t)2 * m.E * 4, 16);
  uint64_t r = 0;
  auto rtake = [&](uint64_t bytes) {
    r = (r + 15) / 16 * 16;
    uint64_t x = r;
    r += bytes;
    return x;
  };
  const uint64_t ldy = F + 4;
  A->rH = rtake((uint64_t)L * N * ldy * 4);
  A->rG = rtake((uint64_t)N * F * 4);
  // dX rows; also the scratch of the column sums and of the stacked lo rows of dW
  A->rdx = rtake((uint64_t)(N > F ? N : F) * 2 * F * 4);
  t->region_bytes = (r + 255) / 256 * 256;
  t->oregion = region_in_smem ? take(t->region_bytes, 16) : 0;
  t->smem_total = (uint32_t)o;
}

static gna_status tcb_plan(const gna_graph* g, const Dims& m, int64_t B, TcbPlan* p) {
  if (m.F % 16 != 0 || m.F > 64 || m.L < 1 || !m.shared) return GNA_ERR_UNSUPPORTED;
  DeviceInfo di;
  gna_status st = device_info(&di);
  if (st != GNA_OK) return st;
  if (di.cc < 100) return GNA_ERR_UNSUPPORTED;
  if (4 * m.F > kTmemCols) return GNA_ERR_UNSUPPORTED;
  const size_t budget = (size_t)di.smem_optin - 2048;
  memset(&p->a, 0, sizeof(p->a));
  int in_smem = 1;
  tcb_layout(m, 1, &p->a);
  if (p->a.base.lay.smem_total > budget) {
    in_smem = 0;
    tcb_layout(m, 0, &p->a);
    if (p->a.base.lay.smem_total > budget) return GNA_ERR_UNSUPPORTED;
  }
  p->a.base.region_in_smem = in_smem;
  const uint32_t min_smem = (uint32_t)(228u * 1024u / (512 / kTmemCols + 1)) + 1024u;
  uint32_t smem = p->a.base.lay.smem_total;
  if (smem < min_smem) smem = min_smem;
  p->a.base.lay.smem_total = smem;
  GNA_CUDA_TRY(cudaFuncSetAttribute((const void*)k_tc_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  GNA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_tc_bwd, kTcThreads, smem));
  if (occ < 1) occ = 1;
  if (occ * kTmemCols > 512) return GNA_ERR_UNSUPPORTED;
  int64_t grid = (int64_t)di.sms * occ;
  if (grid > B) grid = B;
  if (grid < 1) grid = 1;
  p->grid = (int)grid;
  p->smem = smem;
  p->partial_bytes = align_up((size_t)grid * m.P * sizeof(double));
  p->ws_bytes = p->partial_bytes + (in_smem ? 0 : align_up((size_t)grid * p->a.base.lay.region_bytes));
  return GNA_OK;
}

gna_status tcb_workspace(const gna_graph* g, const Dims& m, int64_t B, size_t* bytes) {
  if (B == 0) {
    *bytes = 0;
    return GNA_OK;
  }
  TcbPlan p;
  gna_status st = tcb_plan(g, m, B, &p);
  if (st != GNA_OK) return st;
  *bytes = p.ws_bytes;
  return GNA_OK;
}

// Launches the backward with its per-CTA partials (and per-CTA regions when they do not fit
// in shared memory) in ws.  max_bytes > 0: ws is a fixed array of that size and the grid is
// reduced to fit it (a single CTA that does not fit is GNA_ERR_WORKSPACE); otherwise ws must
// hold tcb_workspace() bytes.
static gna_status tcb_launch(const TcbCall& call, void* ws, size_t ws_bytes, size_t max_bytes, cudaStream_t stream) {
  if (call.B == 0) {
    GNA_CUDA_TRY(cudaMemsetAsync(call.grad, 0, (size_t)call.m.P * sizeof(double), stream));
    return GNA_OK;
  }
  TcbPlan p;
  gna_status st = tcb_plan(call.g, call.m, call.B, &p);
  if (st != GNA_OK) return st;
  if (max_bytes > 0) {
    const size_t region = p.a.base.region_in_smem ? 0 : (size_t)p.a.base.lay.region_bytes;
    const size_t per_cta = (size_t)call.m.P * sizeof(double) + region;
    int64_t grid = (int64_t)((max_bytes - 512) / per_cta);  // two 256-byte alignment pads
    if (grid < 1) return GNA_ERR_WORKSPACE;
    if (grid < p.grid) p.grid = (int)grid;
    p.partial_bytes = align_up((size_t)p.grid * call.m.P * sizeof(double));
    p.ws_bytes = p.partial_bytes + align_up((size_t)p.grid * region);
    ws_bytes = max_bytes;
  }
  if (ws_bytes < p.ws_bytes || !ws) return GNA_ERR_WORKSPACE;
  TcbArgs& a = p.a;
  a.base.g = call.g->d;
  a.base.m = call.m;
  a.base.op = TC_BWD;
  a.base.theta = call.theta;
  a.base.spins = call.spins;
  a.base.B = call.B;
  a.base.gregion = (unsigned char*)ws + p.partial_bytes;
  a.base.wait_limit = wait_limit();
  a.cot = call.cot;
  a.partial = (double*)ws;
  k_tc_bwd<<<p.grid, kTcThreads, p.smem, stream>>>(a);
  GNA_CUDA_TRY(cudaGetLastError());
  k_tcb_reduce<<<(call.m.P + 255) / 256, 256, 0, stream>>>(a.partial, p.grid, call.m.P, call.grad);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

gna_status tcb_run(const TcbCall& call, void* ws, size_t ws_bytes, cudaStream_t stream) {
  return tcb_launch(call, ws, ws_bytes, 0, stream);
}

gna_status tcb_run_fixed(const TcbCall& call, void* scratch, size_t scratch_bytes, cudaStream_t stream) {
  return tcb_launch(call, scratch, scratch_bytes, scratch_bytes, stream);
}

gna_status tc_read_status(int* flags, int clear) {
  int v = 0;
  GNA_CUDA_TRY(cudaMemcpyFromSymbol(&v, s_tc_status, sizeof(int)));
  *flags |= v;
  if (clear) {
    int z = 0;
    GNA_CUDA_TRY(cudaMemcpyToSymbol(s_tc_status, &z, sizeof(int)));
  }
  return GNA_OK;
}

}  // namespace gna

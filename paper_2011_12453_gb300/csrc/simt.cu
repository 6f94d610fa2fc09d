// SIMT kernels (float64 and float32) of the GCN wavefunction, the Heisenberg local
// energy, the Metropolis pair-exchange sampler and the reverse-mode derivative.
//
// One CTA owns one configuration at a time (persistent grid: CTA c handles samples
// c, c + grid, ...).  The per-configuration node features live in a "region" that is
// in shared memory when it fits, else in a per-CTA slice of the caller's workspace.
//
// Eq. (gcn) of arXiv:2011.12453, one layer:   H' = tanh([A_hat H ; H] W + b)
// is evaluated as a gather phase that writes the rows X = [A_hat H ; H] (R x 2F) and a
// dense phase that writes tanh(X W + b).  The incremental local energy runs the same two
// phases on the rows of ball_l(e) only, reading unchanged rows from the cached layers.
#include <climits>
#include <mutex>

#include "common.cuh"
#include "prop.cuh"

namespace gna {

// ---------------------------------------------------------------------------------
// scalar helpers
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double f_tanh(double x) { return tanh(x); }
__device__ __forceinline__ float f_tanh(float x) { return tanhf(x); }
__device__ __forceinline__ double f_exp(double x) { return exp(x); }
__device__ __forceinline__ float f_exp(float x) { return expf(x); }
__device__ __forceinline__ void f_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void f_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
template <typename T>
__device__ __forceinline__ T edge_w(const DevGraph& g, int k);
template <>
__device__ __forceinline__ double edge_w<double>(const DevGraph& g, int k) { return __ldg(g.wd + k); }
template <>
__device__ __forceinline__ float edge_w<float>(const DevGraph& g, int k) { return __ldg(g.wf + k); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------
// kernel arguments and shared-memory carve (same arithmetic on host and device)
// ---------------------------------------------------------------------------------
enum SimtOp { OP_FWD = 0, OP_ELOC_FULL = 1, OP_ELOC_INCR = 2, OP_METRO = 3, OP_BWD = 4, OP_METRO_LEARNED = 5 };

template <typename T>
struct SimtArgs {
  DevGraph g;
  Dims m;
  int op;
  int G;  // bonds per group (incremental)
  int maxball[kMaxL + 1];
  const T* theta;
  const int8_t* spins;
  int64_t B;
  double* logpsi;
  double* eloc;
  float* dlogpsi;
  const double* cot;
  double* partial;  // [grid][P] when the gradient partial is not in shared memory
  int8_t* chain_spins;
  int32_t n_sweeps, record_every;
  uint64_t seed, step0;
  int8_t* samples_out;
  double* logpsi_out;
  int32_t* n_acc;
  double* trace;
  T* gregion;  // [grid][region_elems] when the region is not in shared memory
  size_t region_elems;
  int region_in_smem, partial_in_smem;
  // learned exchange proposal (Metropolis only): network parameters or NULL
  const float* prop;
  double prop_eps;
  int prop_rows;  // capacity of the per-step row buffer (4 x max degree)
};

struct Carve {
  size_t oW, ob, oemb, owr, obr, ospin, oint, odbl, opart, oprop, ophi, oh1, oh2, ologit, orow, oregion, total;
};

// ints: bond list [E] + slot bonds [G] + row offsets [(L+1)][G+1] + misc 16
__host__ __device__ inline size_t carve_ints(int E, int G, int L) {
  return (size_t)E + G + (size_t)(L + 1) * (G + 1) + 16;
}

__host__ __device__ inline Carve carve(const Dims& m, int G, size_t sizeT, int part_smem,
                                       size_t region_elems_smem, int prop_rows = 0) {
  Carve c;
  const int F = m.F, ldw = F + 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 15) / 16 * 16;
    return r;
  };
  c.oW = take((size_t)2 * F * ldw * sizeT);
  c.ob = take((size_t)F * sizeT);
  c.oemb = take((size_t)2 * F * sizeT);
  c.owr = take((size_t)(F + 2) * 2 * sizeT);
  c.obr = take(2 * sizeT);
  c.ospin = take((size_t)2 * m.N);
  c.oint = take(carve_ints(m.E, G, m.L) * 4);
  c.odbl = take((size_t)(2 * G + 2 * kThreads + 8) * 8);
  c.opart = take(part_smem ? (size_t)m.P * 8 : 0);
  const size_t pr = (size_t)prop_rows;
  c.oprop = take(pr ? (size_t)kPropParams * sizeT : 0);
  c.ophi = take(pr * (kPropIn + 1) * sizeT);
  c.oh1 = take(pr * (kPropHid + 1) * sizeT);
  c.oh2 = take(pr * (kPropHid + 1) * sizeT);
  c.ologit = take(pr * sizeT);
  c.orow = take(pr * 3 * 4);
  c.oregion = take(region_elems_smem * sizeT);
  c.total = o;
  return c;
}

// Region sizes in elements of T (shared by the host planner and the kernels).
__host__ __device__ inline size_t xrows_incr(const Dims& m, int G, const int* maxball) {
  size_t r = (size_t)G * maxball[m.L];
  return r > (size_t)m.N ? r : (size_t)m.N;
}
__host__ __device__ inline size_t region_elems(int op, const Dims& m, int G, const int* maxball) {
  const size_t NF = (size_t)m.N * m.F;
  switch (op) {
    case OP_FWD:
    case OP_ELOC_FULL:
      return 3 * NF;  // H (N x F) + X (N x 2F)
    case OP_ELOC_INCR:
    case OP_METRO:
    case OP_METRO_LEARNED: {
      size_t newrows = 0;
      for (int l = 0; l <= m.L; ++l) newrows += (size_t)G * maxball[l];
      return (size_t)(m.L + 1) * NF + newrows * m.F + xrows_incr(m, G, maxball) * 2 * m.F;
    }
    case OP_BWD:
      return (size_t)(m.L + 1) * NF + 2 * NF + 2 * NF;  // cache, G, dY, X (N x 2F)
  }
  return 0;
}

// ---------------------------------------------------------------------------------
// per-CTA context
// ---------------------------------------------------------------------------------
template <typename T>
struct Ctx {
  const SimtArgs<T>* a;
  int N, F, L, E, ldw;
  T *sW, *sb, *semb, *swr, *sbr;
  int8_t *sspin, *sspin2;
  int* sint;
  double* sdbl;
  double* part;  // gradient partial [P]
  T* region;
  // learned proposal buffers
  T *pW, *phi, *h1, *h2, *logit;
  int* rows;  // [prop_rows][3]: centre i, other j, 1 if evaluated in the exchanged state
};

template <typename T>
__device__ inline void make_ctx(const SimtArgs<T>& a, Ctx<T>& c, unsigned char* smem) {
  c.a = &a;
  c.N = a.m.N;
  c.F = a.m.F;
  c.L = a.m.L;
  c.E = a.m.E;
  c.ldw = a.m.F + 1;
  Carve cv = carve(a.m, a.G, sizeof(T), a.partial_in_smem, a.region_in_smem ? a.region_elems : 0, a.prop_rows);
  c.sW = (T*)(smem + cv.oW);
  c.sb = (T*)(smem + cv.ob);
  c.semb = (T*)(smem + cv.oemb);
  c.swr = (T*)(smem + cv.owr);
  c.sbr = (T*)(smem + cv.obr);
  c.sspin = (int8_t*)(smem + cv.ospin);
  c.sspin2 = c.sspin + a.m.N;
  c.sint = (int*)(smem + cv.oint);
  c.sdbl = (double*)(smem + cv.odbl);
  c.part = a.partial_in_smem ? (double*)(smem + cv.opart) : a.partial + (size_t)blockIdx.x * a.m.P;
  c.region = a.region_in_smem ? (T*)(smem + cv.oregion) : a.gregion + (size_t)blockIdx.x * a.region_elems;
  c.pW = (T*)(smem + cv.oprop);
  c.phi = (T*)(smem + cv.ophi);
  c.h1 = (T*)(smem + cv.oh1);
  c.h2 = (T*)(smem + cv.oh2);
  c.logit = (T*)(smem + cv.ologit);
  c.rows = (int*)(smem + cv.orow);
}

// Weights of GCN layer l (0-based) into shared memory, W with padded row stride F+1.
template <typename T>
__device__ void load_layer(const Ctx<T>& c, int l) {
  const Dims& m = c.a->m;
  const T* W = c.a->theta + m.oW + (size_t)l * m.strideW;
  const T* b = c.a->theta + m.ob + (size_t)l * m.strideW;
  for (int i = threadIdx.x; i < 2 * c.F * c.F; i += blockDim.x) c.sW[(i / c.F) * c.ldw + i % c.F] = W[i];
  for (int i = threadIdx.x; i < c.F; i += blockDim.x) c.sb[i] = b[i];
}

// ReLU then layer norm of one row y[0..F) (the GNA section's f): r = max(y, 0),
// (r - mean r) / sqrt(mean (r - mean r)^2 + eps).  Returns 1/sigma; writes the row when out
// is not NULL (out may alias y).
constexpr double kLnEps = 1e-6;
template <typename T>
__device__ inline T relu_ln_row(const T* y, int F, T* out) {
  T mu = 0;
  for (int f = 0; f < F; ++f) mu += y[f] > (T)0 ? y[f] : (T)0;
  mu /= (T)F;
  T var = 0;
  for (int f = 0; f < F; ++f) {
    const T d = (y[f] > (T)0 ? y[f] : (T)0) - mu;
    var += d * d;
  }
  const T inv = (T)1 / sqrt(var / (T)F + (T)kLnEps);
  if (out)
    for (int f = 0; f < F; ++f) out[f] = ((y[f] > (T)0 ? y[f] : (T)0) - mu) * inv;
  return inv;
}

// Reverse of relu_ln_row for one row: y holds the pre-activation on entry and the cotangent
// of the pre-activation on exit, g the cotangent of the output row h:
// dy = [y > 0] (g - mean g - h mean(g h)) / sigma.
template <typename T>
__device__ inline void ln_vjp_row(T* y, const T* g, const T* h, int F) {
  const T inv = relu_ln_row(y, F, (T*)nullptr);
  T mg = 0, mgh = 0;
  for (int f = 0; f < F; ++f) {
    mg += g[f];
    mgh += g[f] * h[f];
  }
  mg /= (T)F;
  mgh /= (T)F;
  for (int f = 0; f < F; ++f) y[f] = y[f] > (T)0 ? (g[f] - mg - h[f] * mgh) * inv : (T)0;
}

// Embedding rows f(W_e[c] + b_e) for c = 0 (spin +1) and 1 (spin -1), readout weights.
template <typename T>
__device__ void load_fixed(const Ctx<T>& c) {
  const Dims& m = c.a->m;
  const T* th = c.a->theta;
  if (m.act == GNA_ACT_RELU_LN) {
    // each thread computes its row's statistics itself (F <= 64), then keeps one element
    for (int i = threadIdx.x; i < 2 * c.F; i += blockDim.x) {
      const T* we = th + m.oWe + (i / c.F) * c.F;
      const T* be = th + m.obe;
      T mu = 0, var = 0;
      for (int f = 0; f < c.F; ++f) mu += we[f] + be[f] > (T)0 ? we[f] + be[f] : (T)0;
      mu /= (T)c.F;
      for (int f = 0; f < c.F; ++f) {
        const T d = (we[f] + be[f] > (T)0 ? we[f] + be[f] : (T)0) - mu;
        var += d * d;
      }
      const int f0 = i % c.F;
      const T y0 = we[f0] + be[f0];
      c.semb[i] = ((y0 > (T)0 ? y0 : (T)0) - mu) * ((T)1 / sqrt(var / (T)c.F + (T)kLnEps));
    }
  } else {
    for (int i = threadIdx.x; i < 2 * c.F; i += blockDim.x) c.semb[i] = f_tanh(th[m.oWe + i] + th[m.obe + i % c.F]);
  }
  for (int i = threadIdx.x; i < (c.F + 2) * 2; i += blockDim.x) c.swr[i] = th[m.owr + i];
  if (threadIdx.x < 2) c.sbr[threadIdx.x] = th[m.obr + threadIdx.x];
  if (c.L > 0) load_layer(c, 0);
}

// out[r][g] = f(b + X[r] W)[g], r < R, or the pre-activation alone when pre_only.  Four rows
// per thread.  Called by every thread of the block (ReLU + layer norm synchronises it).
template <typename T>
__device__ void rows_gemm_act(const Ctx<T>& c, const T* X, int R, T* out, bool pre_only = false) {
  const int F = c.F, K = 2 * F, ldw = c.ldw;
  const int groups = blockDim.x / F;
  const int g = threadIdx.x % F, rg = threadIdx.x / F;
  const bool ln = c.a->m.act == GNA_ACT_RELU_LN;
  const bool elementwise = !ln && !pre_only;
  const T bias = c.sb[g];
  for (int r0 = rg * 4; rg < groups && r0 < R; r0 += groups * 4) {
    const int r1 = min(r0 + 1, R - 1), r2 = min(r0 + 2, R - 1), r3 = min(r0 + 3, R - 1);
    const T* x0 = X + (size_t)r0 * K;
    const T* x1 = X + (size_t)r1 * K;
    const T* x2 = X + (size_t)r2 * K;
    const T* x3 = X + (size_t)r3 * K;
    T a0 = bias, a1 = bias, a2 = bias, a3 = bias;
#pragma unroll 8
    for (int k = 0; k < K; ++k) {
      const T w = c.sW[k * ldw + g];
      a0 += x0[k] * w;
      a1 += x1[k] * w;
      a2 += x2[k] * w;
      a3 += x3[k] * w;
    }
    if (elementwise) {
      a0 = f_tanh(a0);
      a1 = f_tanh(a1);
      a2 = f_tanh(a2);
      a3 = f_tanh(a3);
    }
    out[(size_t)r0 * F + g] = a0;
    if (r0 + 1 < R) out[(size_t)(r0 + 1) * F + g] = a1;
    if (r0 + 2 < R) out[(size_t)(r0 + 2) * F + g] = a2;
    if (r0 + 3 < R) out[(size_t)(r0 + 3) * F + g] = a3;
  }
  if (ln && !pre_only) {
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) relu_ln_row(out + (size_t)r * F, F, out + (size_t)r * F);
  }
}

// Full forward of configuration sp: layer l written to Hs + l*lstride (lstride = 0 keeps
// only the last layer).  X is N x 2F scratch.
template <typename T>
__device__ void forward_all(const Ctx<T>& c, const int8_t* sp, T* Hs, size_t lstride, T* X) {
  const int N = c.N, F = c.F;
  const DevGraph& g = c.a->g;
  for (int i = threadIdx.x; i < N * F; i += blockDim.x) Hs[i] = c.semb[(sp[i / F] > 0 ? 0 : 1) * F + i % F];
  __syncthreads();
  for (int l = 1; l <= c.L; ++l) {
    const T* Hp = Hs + (size_t)(l - 1) * lstride;
    T* Hn = Hs + (size_t)l * lstride;
    if (!c.a->m.shared && l > 1) load_layer(c, l - 1);
    for (int i = threadIdx.x; i < N * F; i += blockDim.x) {
      const int v = i / F, f = i % F;
      T acc = 0;
      const int k1 = __ldg(g.row_ptr + v + 1);
      for (int k = __ldg(g.row_ptr + v); k < k1; ++k) acc += edge_w<T>(g, k) * Hp[(size_t)__ldg(g.col + k) * F + f];
      X[(size_t)v * 2 * F + f] = acc;
      X[(size_t)v * 2 * F + F + f] = Hp[i];
    }
    __syncthreads();
    rows_gemm_act(c, X, N, Hn);
    __syncthreads();
  }
  if (!c.a->m.shared && c.L > 1) {
    load_layer(c, 0);
    __syncthreads();
  }
}

// log Psi = sum_v [H^L_v ; onehot_v] . w_r + b_r, valid in thread 0.  Deterministic order.
template <typename T>
__device__ void readout(const Ctx<T>& c, const T* HL, const int8_t* sp, double out[2]) {
  const int N = c.N, F = c.F;
  T* red = (T*)(c.sdbl + 16);  // kThreads values of scratch, past the slot results
  const int parts = blockDim.x / F;
  const int f = threadIdx.x % F, part = threadIdx.x / F;
  if (part < parts) {
    T acc = 0;
    for (int v = part; v < N; v += parts) acc += HL[(size_t)v * F + f];
    red[part * F + f] = acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    T re = 0, im = 0;
    for (int ff = threadIdx.x; ff < F; ff += 32) {
      T z = 0;
      for (int p = 0; p < parts; ++p) z += red[p * F + ff];
      re += z * c.swr[ff * 2 + 0];
      im += z * c.swr[ff * 2 + 1];
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (threadIdx.x == 0) {
      int up = 0;
      for (int v = 0; v < N; ++v) up += sp[v] > 0;
      const int dn = N - up;
      re += (T)up * c.swr[F * 2 + 0] + (T)dn * c.swr[(F + 1) * 2 + 0] + c.sbr[0];
      im += (T)up * c.swr[F * 2 + 1] + (T)dn * c.swr[(F + 1) * 2 + 1] + c.sbr[1];
      out[0] = (double)re;
      out[1] = (double)im;
    }
  }
  __syncthreads();
}

// Ordered list of antiparallel bonds (warp 0), and the float64 diagonal energy
// sum_e of bond e's diagonal element (J_e/4 s_i s_j for Heisenberg bonds).  Returns the count in sint[E + G + ...] slot and diag in sdbl.
template <typename T>
__device__ int antiparallel_list(const Ctx<T>& c, const int8_t* sp, int* list, double* diag) {
  const DevGraph& g = c.a->g;
  __shared__ int s_count;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int count = 0;
    double d = 0.0;
    for (int base = 0; base < c.E; base += 32) {
      const int e = base + lane;
      bool anti = false;
      if (e < c.E) {
        const int i = __ldg(g.edges + 2 * e), j = __ldg(g.edges + 2 * e + 1);
        const int si = sp[i], sj = sp[j];
        anti = si != sj;
        d += bond_diag(g, e, si, sj);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, anti);
      if (anti) list[count + __popc(mask & ((1u << lane) - 1u))] = e;
      count += __popc(mask);
    }
    d = warp_sum(d);
    if (lane == 0) {
      s_count = count;
      *diag = d;
    }
  }
  __syncthreads();
  return s_count;
}

// ---------------------------------------------------------------------------------
// incremental bond ratios for a group of bonds
// ---------------------------------------------------------------------------------
template <typename T>
struct IncrLayout {
  T* cache;          // (L+1) x N x F
  T* newl[kMaxL + 1];  // per layer: G * maxball[l] rows x F (group rows, compacted)
  T* X;              // xrows x 2F
};

template <typename T>
__device__ inline IncrLayout<T> incr_layout(const Ctx<T>& c) {
  IncrLayout<T> lay;
  const SimtArgs<T>& a = *c.a;
  const size_t NF = (size_t)c.N * c.F;
  lay.cache = c.region;
  T* p = c.region + (size_t)(c.L + 1) * NF;
  for (int l = 0; l <= c.L; ++l) {
    lay.newl[l] = p;
    p += (size_t)a.G * a.maxball[l] * c.F;
  }
  lay.X = p;
  return lay;
}

// Computes, for the nb bonds in slot_e[0..nb), the new rows of every layer and
// Delta = log Psi(s^e) - log Psi(s) (complex, written to sdbl[2k], sdbl[2k+1]).
// soff is (L+1) x (G+1) ints: row offset of slot k's rows in layer l's group buffer.
template <typename T>
__device__ void incr_group(const Ctx<T>& c, const IncrLayout<T>& lay, const int8_t* sp,
                           const int* slot_e, int nb, int* soff) {
  const DevGraph& g = c.a->g;
  const int F = c.F, N = c.N, L = c.L, Lm = g.Lmax, G = c.a->G;
  const size_t NF = (size_t)N * F;
  // row offsets per layer
  if (threadIdx.x == 0) {
    for (int l = 0; l <= L; ++l) {
      int o = 0;
      for (int k = 0; k < nb; ++k) {
        soff[l * (G + 1) + k] = o;
        o += __ldg(g.ball_size + (size_t)slot_e[k] * (Lm + 1) + l);
      }
      soff[l * (G + 1) + nb] = o;
    }
  }
  __syncthreads();
  // layer 0: the exchanged pair takes each other's embedding rows
  for (int i = threadIdx.x; i < nb * 2 * F; i += blockDim.x) {
    const int k = i / (2 * F), r = (i / F) % 2, f = i % F;
    const int e = slot_e[k];
    const int other = __ldg(g.edges + 2 * e + (1 - r));
    lay.newl[0][(size_t)(soff[k] + r) * F + f] = c.semb[(sp[other] > 0 ? 0 : 1) * F + f];
  }
  __syncthreads();
  for (int l = 1; l <= L; ++l) {
    if (!c.a->m.shared && l > 1) load_layer(c, l - 1);
    const int R = soff[l * (G + 1) + nb];
    const T* cp = lay.cache + (size_t)(l - 1) * NF;
    const T* np = lay.newl[l - 1];
    const int* offp = soff + (l - 1) * (G + 1);
    const int* offl = soff + l * (G + 1);
    for (int i = threadIdx.x; i < R * F; i += blockDim.x) {
      const int q = i / F, f = i % F;
      int k = 0;
      while (k + 1 < nb && offl[k + 1] <= q) ++k;
      const int r = q - offl[k];
      const int e = slot_e[k];
      const int bo = __ldg(g.ball_off + e);
      const int sprev = offp[k + 1] - offp[k];  // |ball_{l-1}(e)|
      const T* nrow = np + (size_t)offp[k] * F;
      const int v = __ldg(g.ball_vert + bo + r);
      const int nb0 = __ldg(g.row_nbr + bo + r);
      const int k0 = __ldg(g.row_ptr + v), k1 = __ldg(g.row_ptr + v + 1);
      T acc = 0;
      for (int kk = k0; kk < k1; ++kk) {
        const int p = __ldg(g.nbr_pos + nb0 + (kk - k0));
        const T val = p < sprev ? nrow[(size_t)p * F + f] : cp[(size_t)__ldg(g.col + kk) * F + f];
        acc += edge_w<T>(g, kk) * val;
      }
      lay.X[(size_t)q * 2 * F + f] = acc;
      lay.X[(size_t)q * 2 * F + F + f] = r < sprev ? nrow[(size_t)r * F + f] : cp[(size_t)v * F + f];
    }
    __syncthreads();
    rows_gemm_act(c, lay.X, R, lay.newl[l]);
    __syncthreads();
  }
  if (!c.a->m.shared && L > 1) load_layer(c, 0);
  // Delta_k = sum_{r in ball_L} (new - old) . w_r[:, k]   (one warp per bond)
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
  const T* cL = lay.cache + (size_t)L * NF;
  const int* offL = soff + L * (G + 1);
  for (int k = warp; k < nb; k += nwarps) {
    const int e = slot_e[k];
    const int bo = __ldg(g.ball_off + e);
    const int R = offL[k + 1] - offL[k];
    const T* nrow = lay.newl[L] + (size_t)offL[k] * F;
    T dre = 0, dim = 0;
    for (int i = lane; i < R * F; i += 32) {
      const int r = i / F, f = i % F;
      const int v = __ldg(g.ball_vert + bo + r);
      const T d = nrow[i] - cL[(size_t)v * F + f];
      dre += d * c.swr[f * 2 + 0];
      dim += d * c.swr[f * 2 + 1];
    }
    dre = warp_sum(dre);
    dim = warp_sum(dim);
    if (lane == 0) {
      c.sdbl[2 * k] = (double)dre;
      c.sdbl[2 * k + 1] = (double)dim;
    }
  }
  __syncthreads();
}


// ---------------------------------------------------------------------------------
// learned exchange proposal inside the sampler
// ---------------------------------------------------------------------------------
// Spin of site v in s, or in s with the pair (a, b) exchanged when a >= 0.
__device__ __forceinline__ int spin_at(const int8_t* sp, int v, int a, int b) {
  return v == a ? sp[b] : (v == b ? sp[a] : sp[v]);
}

template <typename T>
__device__ T nbr_sum(const DevGraph& g, const int8_t* sp, int v, int a, int b) {
  T acc = 0;
  const int k1 = __ldg(g.row_ptr + v + 1);
  for (int k = __ldg(g.row_ptr + v); k < k1; ++k) acc += (T)spin_at(sp, __ldg(g.col + k), a, b);
  return acc;
}

// Logits of the rows c.rows[0..nrows): row (i, j, x) scores the exchange i -> j in s
// (x = 0) or in s with (pi, pj) exchanged (x = 1).  CTA-cooperative.
template <typename T>
__device__ void prop_logits(const Ctx<T>& c, const int8_t* sp, int nrows, int pi, int pj) {
  const DevGraph& g = c.a->g;
  for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
    const int i = c.rows[3 * r], j = c.rows[3 * r + 1];
    const int a = c.rows[3 * r + 2] ? pi : -1, b = c.rows[3 * r + 2] ? pj : -1;
    const int ki0 = __ldg(g.row_ptr + i), ki1 = __ldg(g.row_ptr + i + 1);
    const int kj0 = __ldg(g.row_ptr + j), kj1 = __ldg(g.row_ptr + j + 1);
    const int di = ki1 - ki0, dj = kj1 - kj0;
    const T si = (T)spin_at(sp, i, a, b), sj = (T)spin_at(sp, j, a, b);
    T Jij = 0, bi = 0, bj = 0;
    int ci = 0, cj = 0;
    for (int k = ki0; k < ki1; ++k) {
      const int u = __ldg(g.col + k);
      if (u == j) {
        Jij = (T)__ldg(g.J + __ldg(g.col_edge + k));
        continue;
      }
      bi += nbr_sum<T>(g, sp, u, a, b) / (T)(__ldg(g.row_ptr + u + 1) - __ldg(g.row_ptr + u));
      ++ci;
    }
    for (int k = kj0; k < kj1; ++k) {
      const int u = __ldg(g.col + k);
      if (u == i) continue;
      bj += nbr_sum<T>(g, sp, u, a, b) / (T)(__ldg(g.row_ptr + u + 1) - __ldg(g.row_ptr + u));
      ++cj;
    }
    T* f = c.phi + r * (kPropIn + 1);
    f[0] = si;
    f[1] = sj;
    f[2] = Jij;
    f[3] = (T)1 / (T)di;
    f[4] = (T)1 / (T)dj;
    f[5] = (nbr_sum<T>(g, sp, i, a, b) - sj) / (T)max(di - 1, 1);
    f[6] = (nbr_sum<T>(g, sp, j, a, b) - si) / (T)max(dj - 1, 1);
    f[7] = ci ? bi / (T)ci : (T)0;
    f[8] = cj ? bj / (T)cj : (T)0;
  }
  __syncthreads();
  const T* W1 = c.pW + kPropOW1;
  const T* b1 = c.pW + kPropOb1;
  const T* W2 = c.pW + kPropOW2;
  const T* b2 = c.pW + kPropOb2;
  const T* w3 = c.pW + kPropOw3;
  for (int idx = threadIdx.x; idx < nrows * kPropHid; idx += blockDim.x) {
    const int r = idx / kPropHid, k = idx % kPropHid;
    T z = b1[k];
    for (int f = 0; f < kPropIn; ++f) z += c.phi[r * (kPropIn + 1) + f] * W1[f * kPropHid + k];
    c.h1[r * (kPropHid + 1) + k] = f_tanh(z);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nrows * kPropHid; idx += blockDim.x) {
    const int r = idx / kPropHid, k = idx % kPropHid;
    T z = b2[k];
    for (int mm = 0; mm < kPropHid; ++mm) z += c.h1[r * (kPropHid + 1) + mm] * W2[mm * kPropHid + k];
    c.h2[r * (kPropHid + 1) + k] = f_tanh(z);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < nrows; r += blockDim.x >> 5) {
    T z = c.h2[r * (kPropHid + 1) + lane] * w3[lane] + c.h2[r * (kPropHid + 1) + lane + 32] * w3[lane + 32];
    z = warp_sum(z);
    if (lane == 0) c.logit[r] = z + c.pW[kPropOb3];
  }
  __syncthreads();
}

// Appends the rows (i -> u) for the antiparallel neighbours u of i (in CSR order), in s
// or in the exchanged state; returns the new row count (thread 0 only).
template <typename T>
__device__ int push_candidates(const Ctx<T>& c, const int8_t* sp, int i, int swapped, int pi, int pj, int n) {
  const DevGraph& g = c.a->g;
  const int a = swapped ? pi : -1, b = swapped ? pj : -1;
  const int si = spin_at(sp, i, a, b);
  for (int k = __ldg(g.row_ptr + i); k < __ldg(g.row_ptr + i + 1); ++k) {
    const int u = __ldg(g.col + k);
    if (spin_at(sp, u, a, b) != si) {
      c.rows[3 * n] = i;
      c.rows[3 * n + 1] = u;
      c.rows[3 * n + 2] = swapped;
      ++n;
    }
  }
  return n;
}

// Softmax probability of the row for (i -> target) among the rows [r0, r1) (thread 0).
template <typename T>
__device__ T softmax_prob(const Ctx<T>& c, int r0, int r1, int target) {
  T zmax = c.logit[r0];
  for (int r = r0 + 1; r < r1; ++r) zmax = c.logit[r] > zmax ? c.logit[r] : zmax;
  T sum = 0, pt = 0;
  for (int r = r0; r < r1; ++r) {
    const T w = f_exp(c.logit[r] - zmax);
    sum += w;
    if (c.rows[3 * r + 1] == target) pt = w;
  }
  return pt / sum;
}

// ---------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_forward(const SimtArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Ctx<T> c;
  make_ctx(a, c, smem);
  load_fixed(c);
  const size_t NF = (size_t)c.N * c.F;
  for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    for (int i = threadIdx.x; i < c.N; i += blockDim.x) c.sspin[i] = a.spins[b * c.N + i];
    __syncthreads();
    forward_all(c, c.sspin, c.region, 0, c.region + NF);
    double lp[2];
    readout(c, c.region, c.sspin, lp);
    if (threadIdx.x == 0) {
      a.logpsi[2 * b] = lp[0];
      a.logpsi[2 * b + 1] = lp[1];
    }
  }
}

template <typename T>
__device__ inline void add_ratio(double J, double dre, double dim, double* er, double* ei) {
  // J/2 * exp(dre + i dim), ratio formed in T
  const T amp = f_exp((T)dre);
  T s, co;
  f_sincos((T)dim, &s, &co);
  *er += 0.5 * J * (double)(amp * co);
  *ei += 0.5 * J * (double)(amp * s);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_eloc_full(const SimtArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Ctx<T> c;
  make_ctx(a, c, smem);
  load_fixed(c);
  const size_t NF = (size_t)c.N * c.F;
  int* list = c.sint;
  for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    for (int i = threadIdx.x; i < c.N; i += blockDim.x) c.sspin[i] = a.spins[b * c.N + i];
    __syncthreads();
    double diag;
    const int na = antiparallel_list(c, c.sspin, list, &diag);
    forward_all(c, c.sspin, c.region, 0, c.region + NF);
    double lp0[2];
    readout(c, c.region, c.sspin, lp0);
    __shared__ double s_lp0[2];
    if (threadIdx.x == 0) {
      s_lp0[0] = lp0[0];
      s_lp0[1] = lp0[1];
    }
    double er = diag, ei = 0.0;
    if (a.dlogpsi)
      for (int e = threadIdx.x; e < c.E; e += blockDim.x) a.dlogpsi[b * c.E + e] = 0.f;
    for (int t = 0; t < na; ++t) {
      const int e = list[t];
      const int i = __ldg(a.g.edges + 2 * e), j = __ldg(a.g.edges + 2 * e + 1);
      for (int v = threadIdx.x; v < c.N; v += blockDim.x) {
        int8_t s = c.sspin[v];
        if (v == i) s = c.sspin[j];
        if (v == j) s = c.sspin[i];
        c.sspin2[v] = s;
      }
      __syncthreads();
      forward_all(c, c.sspin2, c.region, 0, c.region + NF);
      double lp1[2];
      readout(c, c.region, c.sspin2, lp1);
      if (threadIdx.x == 0) {
        // the difference of two log Psi values, both in T
        const T dre = (T)lp1[0] - (T)s_lp0[0];
        const T dim = (T)lp1[1] - (T)s_lp0[1];
        add_ratio<T>(__ldg(a.g.J + e), (double)dre, (double)dim, &er, &ei);
        if (a.dlogpsi) a.dlogpsi[b * c.E + e] = (float)dre;
      }
    }
    if (threadIdx.x == 0) {
      a.eloc[2 * b] = er;
      a.eloc[2 * b + 1] = ei;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_eloc_incr(const SimtArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Ctx<T> c;
  make_ctx(a, c, smem);
  load_fixed(c);
  const IncrLayout<T> lay = incr_layout(c);
  const int G = a.G;
  int* list = c.sint;
  int* slot_e = c.sint + c.E;
  int* soff = slot_e + G;
  const size_t NF = (size_t)c.N * c.F;
  for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    for (int i = threadIdx.x; i < c.N; i += blockDim.x) c.sspin[i] = a.spins[b * c.N + i];
    __syncthreads();
    double diag;
    const int na = antiparallel_list(c, c.sspin, list, &diag);
    forward_all(c, c.sspin, lay.cache, NF, lay.X);
    if (a.dlogpsi)
      for (int e = threadIdx.x; e < c.E; e += blockDim.x) a.dlogpsi[b * c.E + e] = 0.f;
    double er = diag, ei = 0.0;
    for (int t0 = 0; t0 < na; t0 += G) {
      const int nb = min(G, na - t0);
      if (threadIdx.x < nb) slot_e[threadIdx.x] = list[t0 + threadIdx.x];
      __syncthreads();
      incr_group(c, lay, c.sspin, slot_e, nb, soff);
      if (threadIdx.x == 0) {
        for (int k = 0; k < nb; ++k) {
          const int e = slot_e[k];
          add_ratio<T>(__ldg(a.g.J + e), c.sdbl[2 * k], c.sdbl[2 * k + 1], &er, &ei);
          if (a.dlogpsi) a.dlogpsi[b * c.E + e] = (float)c.sdbl[2 * k];
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      a.eloc[2 * b] = er;
      a.eloc[2 * b + 1] = ei;
    }
    __syncthreads();
  }
}

template <typename T>
__device__ inline bool metropolis_accept(uint64_t r1, double dre);
template <>
__device__ inline bool metropolis_accept<double>(uint64_t r1, double dre) {
  const double u = (double)(r1 >> 11) * 0x1.0p-53;
  return u < exp(2.0 * dre);
}
template <>
__device__ inline bool metropolis_accept<float>(uint64_t r1, double dre) {
  const float u = (float)(r1 >> 40) * 0x1.0p-24f;
  return u < expf(2.0f * (float)dre);
}

template <typename T>
__device__ inline bool accept_log(uint64_t r1, T log_ratio);
template <>
__device__ inline bool accept_log<double>(uint64_t r1, double log_ratio) {
  return (double)(r1 >> 11) * 0x1.0p-53 < exp(log_ratio);
}
template <>
__device__ inline bool accept_log<float>(uint64_t r1, float log_ratio) {
  return (float)(r1 >> 40) * 0x1.0p-24f < expf(log_ratio);
}

// Metropolis(-Hastings) pair-exchange sweeps, one chain per CTA at a time.  Without a
// proposal network every step proposes a uniform bond; with one, a step is a plain bond
// with probability eps, else site i uniform and its partner drawn from the network's
// softmax over i's antiparallel neighbours, accepted with the exact proposal ratio.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_metropolis(const SimtArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Ctx<T> c;
  make_ctx(a, c, smem);
  load_fixed(c);
  if (a.prop)
    for (int i = threadIdx.x; i < kPropParams; i += blockDim.x) c.pW[i] = (T)a.prop[i];
  const IncrLayout<T> lay = incr_layout(c);
  int* slot_e = c.sint + c.E;
  int* soff = slot_e + a.G;
  const size_t NF = (size_t)c.N * c.F;
  const int64_t n_steps = (int64_t)a.n_sweeps * c.N;
  const int n_rec = a.record_every > 0 ? a.n_sweeps / a.record_every : 0;
  const T eps = (T)a.prop_eps;
  __shared__ int s_acc_flag, s_accepts, s_kind, s_move, s_i, s_j, s_n, s_grp[5];
  __shared__ uint64_t s_r1, s_r3;
  __shared__ T s_pij, s_logq;
  for (int64_t ch = blockIdx.x; ch < a.B; ch += gridDim.x) {
    for (int i = threadIdx.x; i < c.N; i += blockDim.x) c.sspin[i] = a.chain_spins[ch * c.N + i];
    if (threadIdx.x == 0) s_accepts = 0;
    __syncthreads();
    forward_all(c, c.sspin, lay.cache, NF, lay.X);
    for (int64_t k = 0; k < n_steps; ++k) {
      if (threadIdx.x == 0) {
        const U64x4 w = philox4x64_10(a.seed, (uint64_t)ch, U64x4{a.step0 + (uint64_t)k, 0, 0, 0});
        s_r1 = w.y;
        s_r3 = w.w;
        s_acc_flag = 0;
        s_logq = 0;
        bool plain = true;
        if (a.prop) plain = (double)(w.w >> 40) * 0x1.0p-24 < a.prop_eps;
        if (plain) {
          const int e = (int)__umul64hi(w.x, (uint64_t)c.E);
          slot_e[0] = e;
          s_i = __ldg(a.g.edges + 2 * e);
          s_j = __ldg(a.g.edges + 2 * e + 1);
          s_kind = 1;
          s_move = c.sspin[s_i] != c.sspin[s_j];
        } else {
          s_kind = 2;
          s_i = (int)__umul64hi(w.z, (uint64_t)c.N);
          s_j = -1;
          slot_e[0] = -1;
          s_n = push_candidates(c, c.sspin, s_i, 0, -1, -1, 0);
          s_move = s_n > 0;
        }
      }
      __syncthreads();
      if (s_kind == 2 && s_move) {
        // first evaluation: the partner j of i drawn from pi_i(. | s)
        prop_logits(c, c.sspin, s_n, -1, -1);
        if (threadIdx.x == 0) {
          const int n = s_n;
          T zmax = c.logit[0];
          for (int r = 1; r < n; ++r) zmax = c.logit[r] > zmax ? c.logit[r] : zmax;
          T sum = 0;
          for (int r = 0; r < n; ++r) sum += f_exp(c.logit[r] - zmax);
          const T uc = (T)((double)(s_r3 & 0xFFFFFFFFull) * 0x1.0p-32);
          T cum = 0;
          int pick = n - 1;
          for (int r = 0; r < n; ++r) {
            cum += f_exp(c.logit[r] - zmax) / sum;
            if (uc < cum) {
              pick = r;
              break;
            }
          }
          s_j = c.rows[3 * pick + 1];
          s_pij = f_exp(c.logit[pick] - zmax) / sum;
          for (int kk = __ldg(a.g.row_ptr + s_i); kk < __ldg(a.g.row_ptr + s_i + 1); ++kk)
            if (__ldg(a.g.col + kk) == s_j) slot_e[0] = __ldg(a.g.col_edge + kk);
        }
        __syncthreads();
      }
      const int e = slot_e[0];
      const int i = s_i, j = s_j;
      double* tr = a.trace ? a.trace + ((size_t)ch * n_steps + k) * 4 : nullptr;
      if (!s_move) {
        if (tr && threadIdx.x == 0) {
          tr[0] = (double)e;
          tr[1] = 0.0;
          tr[2] = __longlong_as_double(0x7ff8000000000000ll);
          tr[3] = (double)s_kind;
        }
      } else {
        if (a.prop) {
          // the exact mixture proposal density both ways: q(s -> s') and q(s' -> s)
          if (threadIdx.x == 0) {
            int n = 0;
            s_grp[0] = 0;
            if (s_kind == 1) n = push_candidates(c, c.sspin, i, 0, i, j, n);
            s_grp[1] = n;
            n = push_candidates(c, c.sspin, j, 0, i, j, n);
            s_grp[2] = n;
            n = push_candidates(c, c.sspin, i, 1, i, j, n);
            s_grp[3] = n;
            n = push_candidates(c, c.sspin, j, 1, i, j, n);
            s_grp[4] = n;
            s_n = n;
          }
          __syncthreads();
          prop_logits(c, c.sspin, s_n, i, j);
          if (threadIdx.x == 0) {
            const T pij = s_kind == 1 ? softmax_prob(c, s_grp[0], s_grp[1], j) : s_pij;
            const T pji = softmax_prob(c, s_grp[1], s_grp[2], i);
            const T pij2 = softmax_prob(c, s_grp[2], s_grp[3], j);
            const T pji2 = softmax_prob(c, s_grp[3], s_grp[4], i);
            const T w_learn = ((T)1 - eps) / (T)c.N, w_plain = eps / (T)c.E;
            const T qf = w_learn * (pij + pji) + w_plain;
            const T qr = w_learn * (pij2 + pji2) + w_plain;
            s_logq = (T)(log((double)qr) - log((double)qf));
          }
          __syncthreads();
        }
        incr_group(c, lay, c.sspin, slot_e, 1, soff);
        if (threadIdx.x == 0) {
          const double dre = c.sdbl[0];
          int acc;
          double value;
          if (a.prop) {
            const T lr = (T)2 * (T)dre + s_logq;
            acc = accept_log<T>(s_r1, lr) ? 1 : 0;
            value = (double)lr;
          } else {
            acc = metropolis_accept<T>(s_r1, dre) ? 1 : 0;
            value = dre;
          }
          s_acc_flag = acc;
          s_accepts += acc;
          if (tr) {
            tr[0] = (double)e;
            tr[1] = (double)acc;
            tr[2] = value;
            tr[3] = (double)s_kind;
          }
        }
        __syncthreads();
        if (s_acc_flag) {
          // commit: the new rows of every layer replace the cached rows of ball_l(e)
          const int bo = __ldg(a.g.ball_off + e);
          for (int l = 0; l <= c.L; ++l) {
            const int R = soff[l * (a.G + 1) + 1];
            for (int t = threadIdx.x; t < R * c.F; t += blockDim.x) {
              const int r = t / c.F, f = t % c.F;
              const int v = __ldg(a.g.ball_vert + bo + r);
              lay.cache[(size_t)l * NF + (size_t)v * c.F + f] = lay.newl[l][t];
            }
          }
          if (threadIdx.x == 0) {
            const int8_t si = c.sspin[i];
            c.sspin[i] = c.sspin[j];
            c.sspin[j] = si;
          }
        }
      }
      __syncthreads();
      if ((k + 1) % c.N == 0 && a.record_every > 0) {
        const int sweep = (int)((k + 1) / c.N);
        if (sweep % a.record_every == 0) {
          const int rec = sweep / a.record_every - 1;
          if (rec < n_rec) {
            if (a.samples_out)
              for (int v = threadIdx.x; v < c.N; v += blockDim.x)
                a.samples_out[((size_t)rec * a.B + ch) * c.N + v] = c.sspin[v];
            if (a.logpsi_out) {
              double lp[2];
              readout(c, lay.cache + (size_t)c.L * NF, c.sspin, lp);
              if (threadIdx.x == 0) {
                a.logpsi_out[((size_t)rec * a.B + ch) * 2] = lp[0];
                a.logpsi_out[((size_t)rec * a.B + ch) * 2 + 1] = lp[1];
              }
            }
          }
        }
      }
    }
    for (int v = threadIdx.x; v < c.N; v += blockDim.x) a.chain_spins[ch * c.N + v] = c.sspin[v];
    if (threadIdx.x == 0 && a.n_acc) a.n_acc[ch] += s_accepts;
    __syncthreads();
  }
}

// Reverse mode of Eq. (gcn) and the readout; activations recomputed per sample.
constexpr int kThreadsBwd = 512;

template <typename T>
__global__ void __launch_bounds__(kThreadsBwd, 1) k_backward(const SimtArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  Ctx<T> c;
  make_ctx(a, c, smem);
  load_fixed(c);
  const Dims& m = a.m;
  const int N = c.N, F = c.F, L = c.L;
  const size_t NF = (size_t)N * F;
  T* cache = c.region;
  T* Gb = cache + (size_t)(L + 1) * NF;
  T* dY = Gb + NF;
  T* X = dY + NF;  // N x 2F
  const DevGraph& g = a.g;
  double* part = c.part;
  for (int i = threadIdx.x; i < m.P; i += blockDim.x) part[i] = 0.0;
  __syncthreads();
  for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) c.sspin[i] = a.spins[b * N + i];
    __syncthreads();
    const double c0 = a.cot[2 * b], c1 = a.cot[2 * b + 1];
    forward_all(c, c.sspin, cache, NF, X);
    const T* HL = cache + (size_t)L * NF;
    // readout: d w_r[f][k] += cot_k z_f, d b_r[k] += cot_k; z = sum_v [H^L_v ; onehot_v]
    for (int f = threadIdx.x; f < F + 2; f += blockDim.x) {
      double z = 0.0;
      if (f < F) {
        T zz = 0;
        for (int v = 0; v < N; ++v) zz += HL[(size_t)v * F + f];
        z = (double)zz;
      } else {
        int cnt = 0;
        for (int v = 0; v < N; ++v) cnt += (f == F) ? (c.sspin[v] > 0) : (c.sspin[v] < 0);
        z = (double)cnt;
      }
      part[m.owr + 2 * f] += c0 * z;
      part[m.owr + 2 * f + 1] += c1 * z;
    }
    if (threadIdx.x == 0) {
      part[m.obr] += c0;
      part[m.obr + 1] += c1;
    }
    // dL/dH^L_v = w_r[:F] . cot  (same for every site)
    for (int i = threadIdx.x; i < N * F; i += blockDim.x) {
      const int f = i % F;
      Gb[i] = (T)c0 * c.swr[2 * f] + (T)c1 * c.swr[2 * f + 1];
    }
    __syncthreads();
    for (int l = L; l >= 1; --l) {
      if (!m.shared) load_layer(c, l - 1);
      const T* Hp = cache + (size_t)(l - 1) * NF;
      const T* Hl = cache + (size_t)l * NF;
      // X = [A_hat H^{l-1} ; H^{l-1}],  dY = G (1 - H^l^2)
      for (int i = threadIdx.x; i < N * F; i += blockDim.x) {
        const int v = i / F, f = i % F;
        T acc = 0;
        const int k1 = __ldg(g.row_ptr + v + 1);
        for (int k = __ldg(g.row_ptr + v); k < k1; ++k) acc += edge_w<T>(g, k) * Hp[(size_t)__ldg(g.col + k) * F + f];
        X[(size_t)v * 2 * F + f] = acc;
        X[(size_t)v * 2 * F + F + f] = Hp[i];
        if (m.act != GNA_ACT_RELU_LN) dY[i] = Gb[i] * ((T)1 - Hl[i] * Hl[i]);
      }
      __syncthreads();
      if (m.act == GNA_ACT_RELU_LN) {
        // Y = X W + b again, then per row dY = [Y > 0] (G - mean G - H mean(G H)) / sigma
        rows_gemm_act(c, X, N, dY, true);
        __syncthreads();
        for (int v = threadIdx.x; v < N; v += blockDim.x)
          ln_vjp_row(dY + (size_t)v * F, Gb + (size_t)v * F, Hl + (size_t)v * F, F);
        __syncthreads();
      }
      // dW[k][g] += sum_v X[v][k] dY[v][g] (4 k per thread, two v streams);
      // db[g] += sum_v dY[v][g]
      const size_t oW = m.oW + (size_t)(l - 1) * m.strideW;
      const size_t ob = m.ob + (size_t)(l - 1) * m.strideW;
      const int nkb = (2 * F + 3) / 4;  // blocks of 4 input features (the last may be partial)
      for (int i = threadIdx.x; i < nkb * F; i += blockDim.x) {
        const int k0 = (i / F) * 4, gg = i % F;
        const int nq = min(4, 2 * F - k0);
        T a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
        int v = 0;
        for (; v + 1 < N; v += 2) {
          const T* x0 = X + (size_t)v * 2 * F + k0;
          const T* x1 = x0 + 2 * F;
          const T d0 = dY[(size_t)v * F + gg], d1 = dY[(size_t)(v + 1) * F + gg];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < nq) {
              a0[q] += x0[q] * d0;
              a1[q] += x1[q] * d1;
            }
        }
        if (v < N) {
          const T* x0 = X + (size_t)v * 2 * F + k0;
          const T d0 = dY[(size_t)v * F + gg];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < nq) a0[q] += x0[q] * d0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nq) part[oW + (size_t)(k0 + q) * F + gg] += (double)(a0[q] + a1[q]);
      }
      for (int gg = threadIdx.x; gg < F; gg += blockDim.x) {
        T b0 = 0, b1 = 0;
        int v = 0;
        for (; v + 1 < N; v += 2) {
          b0 += dY[(size_t)v * F + gg];
          b1 += dY[(size_t)(v + 1) * F + gg];
        }
        if (v < N) b0 += dY[(size_t)v * F + gg];
        part[ob + gg] += (double)(b0 + b1);
      }
      __syncthreads();
      // dX[v][k] = sum_g dY[v][g] W[k][g]   (into X; 4 rows per thread)
      for (int i = threadIdx.x; i < ((N + 3) / 4) * 2 * F; i += blockDim.x) {
        const int vb = (i / (2 * F)) * 4, k = i % (2 * F);
        const int v1 = min(vb + 1, N - 1), v2 = min(vb + 2, N - 1), v3 = min(vb + 3, N - 1);
        T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        for (int gg = 0; gg < F; ++gg) {
          const T w = c.sW[k * c.ldw + gg];
          s0 += dY[(size_t)vb * F + gg] * w;
          s1 += dY[(size_t)v1 * F + gg] * w;
          s2 += dY[(size_t)v2 * F + gg] * w;
          s3 += dY[(size_t)v3 * F + gg] * w;
        }
        X[(size_t)vb * 2 * F + k] = s0;
        if (vb + 1 < N) X[(size_t)(vb + 1) * 2 * F + k] = s1;
        if (vb + 2 < N) X[(size_t)(vb + 2) * 2 * F + k] = s2;
        if (vb + 3 < N) X[(size_t)(vb + 3) * 2 * F + k] = s3;
      }
      __syncthreads();
      // G^{l-1}_v = sum_u A_hat[v][u] dX[u][:F] + dX[v][F:]
      for (int i = threadIdx.x; i < N * F; i += blockDim.x) {
        const int v = i / F, f = i % F;
        T acc = X[(size_t)v * 2 * F + F + f];
        const int k1 = __ldg(g.row_ptr + v + 1);
        for (int k = __ldg(g.row_ptr + v); k < k1; ++k) acc += edge_w<T>(g, k) * X[(size_t)__ldg(g.col + k) * 2 * F + f];
        Gb[i] = acc;
      }
      __syncthreads();
    }
    if (!m.shared && L > 1) {
      load_layer(c, 0);
    }
    // embedding: dY0 = G f'(Y0); dW_e[c][f] += sum_{v: c_v = c} dY0; db_e[f] += sum_v dY0
    if (m.act == GNA_ACT_RELU_LN) {
      for (int v = threadIdx.x; v < N; v += blockDim.x) {
        const int row = c.sspin[v] > 0 ? 0 : 1;
        T* y = dY + (size_t)v * F;
        for (int f = 0; f < F; ++f) y[f] = a.theta[m.oWe + row * F + f] + a.theta[m.obe + f];
        ln_vjp_row(y, Gb + (size_t)v * F, cache + (size_t)v * F, F);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < 3 * F; i += blockDim.x) {
      const int f = i % F, which = i / F;  // 0: W_e row up, 1: W_e row down, 2: b_e
      T acc = 0;
      for (int v = 0; v < N; ++v) {
        const bool up = c.sspin[v] > 0;
        if (which == 2 || (which == 0) == up) {
          if (m.act == GNA_ACT_RELU_LN) {
            acc += dY[(size_t)v * F + f];
          } else {
            const T h = cache[(size_t)v * F + f];
            acc += Gb[(size_t)v * F + f] * ((T)1 - h * h);
          }
        }
      }
      part[(which < 2 ? m.oWe + which * F : m.obe) + f] += (double)acc;
    }
    __syncthreads();
  }
  if (a.partial_in_smem) {
    for (int i = threadIdx.x; i < m.P; i += blockDim.x) a.partial[(size_t)blockIdx.x * m.P + i] = part[i];
  }
}

// grad[p] = sum_cta partial[cta][p], fixed order, float64.
__global__ void k_reduce_partials(const double* partial, int grid, int P, double* grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double s = 0.0;
  for (int c = 0; c < grid; ++c) s += partial[(size_t)c * P + p];
  grad[p] = s;
}

// ---------------------------------------------------------------------------------
// host side: planning and launch
// ---------------------------------------------------------------------------------
template <typename T>
static const void* kernel_ptr(int op) {
  switch (op) {
    case OP_FWD:
      return (const void*)k_forward<T>;
    case OP_ELOC_FULL:
      return (const void*)k_eloc_full<T>;
    case OP_ELOC_INCR:
      return (const void*)k_eloc_incr<T>;
    case OP_METRO:
    case OP_METRO_LEARNED:
      return (const void*)k_metropolis<T>;
    case OP_BWD:
      return (const void*)k_backward<T>;
  }
  return nullptr;
}

template <typename T>
gna_status simt_plan(const gna_graph* g, const Dims& m, int op, int64_t B, Plan* p) {
  DeviceInfo di;
  gna_status st = device_info(&di);
  if (st != GNA_OK) return st;
  const int* mb = g->max_ball.data();
  int maxball[kMaxL + 1] = {0};
  for (int l = 0; l <= m.L && l <= g->d.Lmax; ++l) maxball[l] = mb[l];
  const int part = (op == OP_BWD);
  const int prop_rows = op == OP_METRO_LEARNED ? 4 * (g->max_deg > 0 ? g->max_deg : 1) : 0;
  p->prop_rows = prop_rows;
  const size_t budget = (size_t)di.smem_optin - 1024;  // room for static shared variables
  int G = 1;
  if (op == OP_ELOC_INCR) {
    // as many bonds per group as fit next to a shared-memory cache (at most 8, one per warp)
    G = 8;
    while (G > 1) {
      Carve cv = carve(m, G, sizeof(T), 0, region_elems(op, m, G, maxball));
      if (cv.total <= budget) break;
      --G;
    }
  }
  const size_t rel = region_elems(op, m, G, maxball);
  int part_smem = 0;
  if (part) {
    Carve cv = carve(m, G, sizeof(T), 1, rel);
    part_smem = cv.total <= budget || carve(m, G, sizeof(T), 1, 0).total <= budget;
  }
  Carve in = carve(m, G, sizeof(T), part_smem, rel, prop_rows);
  p->G = G;
  p->region_elems = rel;
  p->partial_in_smem = part_smem;
  if (in.total <= budget) {
    p->region_in_smem = 1;
    p->smem = (int)in.total;
  } else {
    Carve out = carve(m, G, sizeof(T), part_smem, 0, prop_rows);
    if (out.total > budget) return GNA_ERR_UNSUPPORTED;
    p->region_in_smem = 0;
    p->smem = (int)out.total;
  }
  const void* kp = kernel_ptr<T>(op);
  GNA_CUDA_TRY(cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem));
  int occ = 0;
  GNA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kp, op == OP_BWD ? kThreadsBwd : kThreads, p->smem));
  if (occ < 1) occ = 1;
  int64_t grid = (int64_t)di.sms * occ;
  if (B < grid) grid = B;
  if (grid < 1) grid = 1;
  p->grid = (int)grid;
  size_t ws = 0;
  if (!p->region_in_smem) ws += align_up((size_t)p->grid * rel * sizeof(T));
  if (part) ws += align_up((size_t)p->grid * m.P * sizeof(double));
  p->ws_bytes = ws;
  return GNA_OK;
}



template <typename T>
gna_status simt_launch(const SimtCall& sc, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (sc.B == 0) {
    if (sc.op == OP_BWD) GNA_CUDA_TRY(cudaMemsetAsync(sc.grad, 0, sc.m.P * sizeof(double), stream));
    return GNA_OK;
  }
  Plan p;
  const int plan_op = (sc.op == OP_METRO && sc.prop) ? (int)OP_METRO_LEARNED : sc.op;
  gna_status st = simt_plan<T>(sc.g, sc.m, plan_op, sc.B, &p);
  if (st != GNA_OK) return st;
  if (ws_bytes < p.ws_bytes || (p.ws_bytes > 0 && ws == nullptr)) return GNA_ERR_WORKSPACE;
  SimtArgs<T> a;
  a.g = sc.g->d;
  a.m = sc.m;
  a.op = sc.op;
  a.G = p.G;
  for (int l = 0; l <= kMaxL; ++l) a.maxball[l] = (l <= sc.m.L && l <= sc.g->d.Lmax) ? sc.g->max_ball[l] : 0;
  a.theta = (const T*)sc.theta;
  a.spins = sc.spins;
  a.B = sc.B;
  a.logpsi = sc.logpsi;
  a.eloc = sc.eloc;
  a.dlogpsi = sc.dlogpsi;
  a.cot = sc.cot;
  a.chain_spins = sc.chain_spins;
  a.n_sweeps = sc.n_sweeps;
  a.record_every = sc.record_every;
  a.seed = sc.seed;
  a.step0 = sc.step0;
  a.samples_out = sc.samples_out;
  a.logpsi_out = sc.logpsi_out;
  a.n_acc = sc.n_acc;
  a.trace = sc.trace;
  a.region_elems = p.region_elems;
  a.region_in_smem = p.region_in_smem;
  a.partial_in_smem = p.partial_in_smem;
  a.prop = sc.op == OP_METRO ? sc.prop : nullptr;
  a.prop_eps = sc.prop_eps;
  a.prop_rows = p.prop_rows;
  unsigned char* w = (unsigned char*)ws;
  a.gregion = nullptr;
  if (!p.region_in_smem) {
    a.gregion = (T*)w;
    w += align_up((size_t)p.grid * p.region_elems * sizeof(T));
  }
  a.partial = nullptr;
  if (sc.op == OP_BWD) a.partial = (double*)w;
  switch (sc.op) {
    case OP_FWD:
      k_forward<T><<<p.grid, kThreads, p.smem, stream>>>(a);
      break;
    case OP_ELOC_FULL:
      k_eloc_full<T><<<p.grid, kThreads, p.smem, stream>>>(a);
      break;
    case OP_ELOC_INCR:
      k_eloc_incr<T><<<p.grid, kThreads, p.smem, stream>>>(a);
      break;
    case OP_METRO:
      k_metropolis<T><<<p.grid, kThreads, p.smem, stream>>>(a);
      break;
    case OP_BWD:
      k_backward<T><<<p.grid, kThreadsBwd, p.smem, stream>>>(a);
      GNA_CUDA_TRY(cudaGetLastError());
      k_reduce_partials<<<(sc.m.P + 255) / 256, 256, 0, stream>>>(a.partial, p.grid, sc.m.P, sc.grad);
      break;
    default:
      return GNA_ERR_INVALID_ARG;
  }
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}


// ---------------------------------------------------------------------------------
// Backward with library-owned scratch (gna_backward_static)
// ---------------------------------------------------------------------------------
// The per-block gradient partials -- and the per-block feature region when a sample's
// features do not fit in shared memory -- live in this fixed array instead of a
// caller-supplied workspace.  Every device that loads the library reserves it until
// the process exits.  All calls on a device share it.
constexpr size_t kStaticScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_backward_scratch[kStaticScratchBytes];

// Device address of the array on the current device.  Host code cannot use the
// symbol itself (it names a host-side stand-in), so the address is looked up once per
// device, with that device current, and cached.
static gna_status static_scratch_address(void** out) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  int dev = 0;
  GNA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GNA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    GNA_CUDA_TRY(cudaGetSymbolAddress(&p, g_backward_scratch));
    addr[dev] = p;
  }
  *out = addr[dev];
  return GNA_OK;
}

template <typename T>
static gna_status backward_static_launch(const SimtCall& sc, cudaStream_t stream) {
  if (sc.B == 0) {
    GNA_CUDA_TRY(cudaMemsetAsync(sc.grad, 0, sc.m.P * sizeof(double), stream));
    return GNA_OK;
  }
  Plan p;
  gna_status st = simt_plan<T>(sc.g, sc.m, OP_BWD, sc.B, &p);
  if (st != GNA_OK) return st;
  // Fit the grid to the array: each block needs its partial (and its region when the
  // region is not in shared memory).  A single block that does not fit is an error.
  const size_t region_bytes = p.region_in_smem ? 0 : p.region_elems * sizeof(T);
  const size_t per_block = region_bytes + (size_t)sc.m.P * sizeof(double);
  const size_t usable = kStaticScratchBytes - 512;  // two 256-byte alignment pads
  int64_t grid = (int64_t)(usable / per_block);
  if (grid < 1) return GNA_ERR_WORKSPACE;
  if (grid > p.grid) grid = p.grid;
  void* base = nullptr;
  st = static_scratch_address(&base);
  if (st != GNA_OK) return st;
  SimtArgs<T> a;
  a.g = sc.g->d;
  a.m = sc.m;
  a.op = OP_BWD;
  a.G = p.G;
  for (int l = 0; l <= kMaxL; ++l) a.maxball[l] = (l <= sc.m.L && l <= sc.g->d.Lmax) ? sc.g->max_ball[l] : 0;
  a.theta = (const T*)sc.theta;
  a.spins = sc.spins;
  a.B = sc.B;
  a.logpsi = nullptr;
  a.eloc = nullptr;
  a.dlogpsi = nullptr;
  a.cot = sc.cot;
  a.chain_spins = nullptr;
  a.n_sweeps = 0;
  a.record_every = 0;
  a.seed = 0;
  a.step0 = 0;
  a.samples_out = nullptr;
  a.logpsi_out = nullptr;
  a.n_acc = nullptr;
  a.trace = nullptr;
  a.region_elems = p.region_elems;
  a.region_in_smem = p.region_in_smem;
  a.partial_in_smem = p.partial_in_smem;
  a.prop = nullptr;
  a.prop_eps = 0.0;
  a.prop_rows = 0;
  // Every block zeroes its own partial before accumulating and the reduction reads
  // only what this launch wrote, so nothing left by an earlier call is used.
  unsigned char* w = (unsigned char*)base;
  a.gregion = nullptr;
  if (!p.region_in_smem) {
    a.gregion = (T*)w;
    w += align_up((size_t)grid * region_bytes);
  }
  a.partial = (double*)w;
  k_backward<T><<<(int)grid, kThreadsBwd, p.smem, stream>>>(a);
  GNA_CUDA_TRY(cudaGetLastError());
  k_reduce_partials<<<(sc.m.P + 255) / 256, 256, 0, stream>>>(a.partial, (int)grid, sc.m.P, sc.grad);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

gna_status static_scratch(void** base, size_t* bytes) {
  *bytes = kStaticScratchBytes;
  return static_scratch_address(base);
}

gna_status simt_backward_static(const SimtCall& sc, int prec, cudaStream_t stream) {
  return prec == GNA_PREC_FP64 ? backward_static_launch<double>(sc, stream) : backward_static_launch<float>(sc, stream);
}

gna_status simt_workspace(const gna_graph* g, const Dims& m, int prec, int op, int64_t B, size_t* bytes) {
  Plan p;
  if (B == 0) {
    *bytes = 0;
    return GNA_OK;
  }
  gna_status st = prec == GNA_PREC_FP64 ? simt_plan<double>(g, m, op, B, &p) : simt_plan<float>(g, m, op, B, &p);
  if (st != GNA_OK) return st;
  *bytes = p.ws_bytes;
  return GNA_OK;
}

gna_status simt_run(const SimtCall& sc, int prec, void* ws, size_t ws_bytes, cudaStream_t stream) {
  return prec == GNA_PREC_FP64 ? simt_launch<double>(sc, ws, ws_bytes, stream)
                               : simt_launch<float>(sc, ws, ws_bytes, stream);
}

}  // namespace gna

// Metropolis pair-exchange sweeps with one warp per chain (plain moves).
//
// Sampling P ~ |Psi|^2 (scaling section of arXiv:2011.12453) needs, per proposed exchange
// of an antiparallel pair (i, j), the ratio Psi(s')/Psi(s).  It is computed by propagating
// the change of the node features through the GCN layers of Eq. (gcn), restricted to the
// nested neighbourhoods ball_l(e) of the bond:
//   dH^0 = rows i, j of the embedding difference;
//   dY^l = [A_hat dH^{l-1} ; dH^{l-1}] W   (the bias cancels; zero outside ball_l),
//   dH^l = tanh(Y^l + dY^l) - tanh(Y^l) = t (1 - H^2)/(1 + H t),  t = tanh(dY^l),
//   Delta log Psi = w_r[:F] . sum_v dH^L_v.
// The chain keeps the pre-activations Y^1..Y^L of its current state (in a per-warp slice of
// the workspace, L2-resident); an accepted move adds dY^l to the rows of ball_l.
//
// A warp owns a chain at a time: no block barriers, only warp-synchronous steps, so the
// latency of one chain's step is hidden behind the other warps' chains.  Lanes own
// feature columns (f = lane, lane + 32).  The Philox words of 32 consecutive steps are
// drawn at once, one step per lane, and broadcast by shuffles.
#include <climits>
#include <cmath>

#include "common.cuh"
#include "metro.cuh"
#include "prop.cuh"

namespace gna {

constexpr int kMetroMaxWarps = 16;  // chains per CTA at most (fewer when shared memory is short)

template <typename T>
struct MetroArgs {
  DevGraph g;
  Dims m;
  int maxball[kMaxL + 1];
  int off_dh[kMaxL + 1];  // per-warp smem element offsets (elements of T) of dH^l rows, l < L
  int off_dy[kMaxL + 1];  // workspace element offsets of dY^l rows (l = 1..L) in the warp slot
  int off_x;              // per-warp smem element offset of the 4 staged dX rows (4 x 2F)
  int off_meta;           // per-warp smem byte offset of the row metadata
  int max_rows, max_span; // capacity of the metadata arrays (rows of ball_L, their neighbours)
  int warp_bytes;         // shared-memory bytes per warp
  int prop_rows;          // capacity of the proposal row arrays (4 x max degree, 0 without a network)
  int nwarps;             // warps (chains in flight) per CTA
  const T* theta;
  int8_t* chain_spins;
  int64_t C;
  int32_t n_sweeps, record_every;
  uint64_t seed, step0;
  int8_t* samples_out;
  double* logpsi_out;
  int32_t* n_acc;
  double* trace;
  T* gws;          // per warp slot: Y^1..Y^L [L][N][F], two H scratch layers [2][N][F], dY rows
  size_t ws_elems; // elements per warp slot
  const float* prop;  // learned proposal network or NULL (plain moves)
  double prop_eps;
};

__device__ __forceinline__ double m_tanh(double x) { return tanh(x); }
// float tanh: odd Taylor series through x^13 for |x| < 0.5 (truncation below 5e-7
// relative), else sgn(x) (1 - e)/(1 + e) with e = exp(-2|x|).
__device__ __forceinline__ float m_tanh(float x) {
  const float ax = fabsf(x);
  if (ax < 0.5f) {
    const float x2 = x * x;
    float p = 21844.f / 6081075.f;
    p = fmaf(p, x2, -1382.f / 155925.f);
    p = fmaf(p, x2, 62.f / 2835.f);
    p = fmaf(p, x2, -17.f / 315.f);
    p = fmaf(p, x2, 2.f / 15.f);
    p = fmaf(p, x2, -1.f / 3.f);
    return fmaf(p * x2, x, x);
  }
  const float e = __expf(-2.f * ax);
  return copysignf(__fdividef(1.f - e, 1.f + e), x);
}
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_exp(float x) { return __expf(x); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ float m_div(float a, float b) { return __fdividef(a, b); }

__device__ __forceinline__ void load4(const float* p, float* v) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// dH = tanh(y + dy) - tanh(y), in the stable form t (1 - H^2)/(1 + H t) built from
// e = exp(-2|y|); falls back to the direct difference when 1 + H t is small (a unit
// swinging across saturation, where dH is O(1) and the difference has no cancellation).
template <typename T>
__device__ __forceinline__ T dtanh(T y, T dy) {
  const T e = m_exp((T)-2 * fabs(y));
  const T t = m_tanh(dy);
  const T sg = y < (T)0 ? (T)-1 : (T)1;
  const T ope = (T)1 + e;
  const T den = ope * (ope + sg * ((T)1 - e) * t);
  return den > (T)1e-3 ? m_div((T)4 * e * t, den) : m_tanh(y + dy) - m_tanh(y);
}

template <typename T>
__device__ inline bool m_accept_log(uint64_t r1, T log_ratio);
template <>
__device__ inline bool m_accept_log<double>(uint64_t r1, double log_ratio) {
  return (double)(r1 >> 11) * 0x1.0p-53 < exp(log_ratio);
}
template <>
__device__ inline bool m_accept_log<float>(uint64_t r1, float log_ratio) {
  return (float)(r1 >> 40) * 0x1.0p-24f < expf(log_ratio);
}

// Row index in [r0, r1) whose partner is `other`.
__device__ __forceinline__ int row_of(const int* ro, int r0, int r1, int other) {
  for (int r = r0; r < r1; ++r)
    if (ro[r] == other) return r;
  return r0;
}

template <typename T>
__device__ inline bool m_accept(uint64_t r1, T dre);
template <>
__device__ inline bool m_accept<double>(uint64_t r1, double dre) {
  return (double)(r1 >> 11) * 0x1.0p-53 < exp(2.0 * dre);
}
template <>
__device__ inline bool m_accept<float>(uint64_t r1, float dre) {
  return (float)(r1 >> 40) * 0x1.0p-24f < expf(2.0f * dre);
}


// ---- learned exchange proposal, evaluated by one warp ----------------------------------
__device__ __forceinline__ int spin_x(const int8_t* sp, int v, int a, int b) {
  return v == a ? sp[b] : (v == b ? sp[a] : sp[v]);
}

template <typename T>
__device__ T nsum(const DevGraph& g, const int8_t* sp, int v, int a, int b) {
  T acc = 0;
  const int k1 = __ldg(g.row_ptr + v + 1);
  for (int k = __ldg(g.row_ptr + v); k < k1; ++k) acc += (T)spin_x(sp, __ldg(g.col + k), a, b);
  return acc;
}

// Features of the ordered pair (i, j) in s, or in s with (a, b) exchanged when a >= 0.
template <typename T>
__device__ void pair_phi(const DevGraph& g, const int8_t* sp, int i, int j, int a, int b, T* f) {
  const int ki0 = __ldg(g.row_ptr + i), ki1 = __ldg(g.row_ptr + i + 1);
  const int kj0 = __ldg(g.row_ptr + j), kj1 = __ldg(g.row_ptr + j + 1);
  const int di = ki1 - ki0, dj = kj1 - kj0;
  const T si = (T)spin_x(sp, i, a, b), sj = (T)spin_x(sp, j, a, b);
  T Jij = 0, bi = 0, bj = 0;
  int ci = 0, cj = 0;
  for (int k = ki0; k < ki1; ++k) {
    const int u = __ldg(g.col + k);
    if (u == j) {
      Jij = (T)__ldg(g.J + __ldg(g.col_edge + k));
      continue;
    }
    bi += nsum<T>(g, sp, u, a, b) / (T)(__ldg(g.row_ptr + u + 1) - __ldg(g.row_ptr + u));
    ++ci;
  }
  for (int k = kj0; k < kj1; ++k) {
    const int u = __ldg(g.col + k);
    if (u == i) continue;
    bj += nsum<T>(g, sp, u, a, b) / (T)(__ldg(g.row_ptr + u + 1) - __ldg(g.row_ptr + u));
    ++cj;
  }
  f[0] = si;
  f[1] = sj;
  f[2] = Jij;
  f[3] = (T)1 / (T)di;
  f[4] = (T)1 / (T)dj;
  f[5] = (nsum<T>(g, sp, i, a, b) - sj) / (T)max(di - 1, 1);
  f[6] = (nsum<T>(g, sp, j, a, b) - si) / (T)max(dj - 1, 1);
  f[7] = ci ? bi / (T)ci : (T)0;
  f[8] = cj ? bj / (T)cj : (T)0;
}

// Logits of rows r < n of (rc[r] -> ro[r]) evaluated in the state selected by rx[r]
// (0: s, 1: s with (pa, pb) exchanged).  Returns the logit of row `lane` (and row lane+32).
template <typename T>
__device__ void warp_logits(const DevGraph& g, const int8_t* sp, const T* P, const int* rc, const int* ro,
                            const int* rx, int n, int pa, int pb, T* out0, T* out1) {
  const int lane = threadIdx.x & 31;
  const T* W1 = P + kPropOW1;
  const T* b1 = P + kPropOb1;
  const T* W2 = P + kPropOW2;
  const T* b2 = P + kPropOb2;
  const T* w3 = P + kPropOw3;
  T lg0 = 0, lg1 = 0;
  for (int base = 0; base < n; base += 32) {
    T f[kPropIn];
    const int r = base + lane;
    if (r < n) {
      pair_phi<T>(g, sp, rc[r], ro[r], rx[r] ? pa : -1, rx[r] ? pb : -1, f);
    } else {
#pragma unroll
      for (int q = 0; q < kPropIn; ++q) f[q] = 0;
    }
    const int cnt = min(32, n - base);
    for (int rr = 0; rr < cnt; ++rr) {
      // hidden layer 1 (units lane, lane + 32) of row base + rr
      T z0 = b1[lane], z1 = b1[lane + 32];
#pragma unroll
      for (int q = 0; q < kPropIn; ++q) {
        const T x = __shfl_sync(0xffffffffu, f[q], rr);
        z0 += x * W1[q * kPropHid + lane];
        z1 += x * W1[q * kPropHid + lane + 32];
      }
      const T h0 = m_tanh(z0), h1 = m_tanh(z1);
      // hidden layer 2
      T y0 = b2[lane], y1 = b2[lane + 32];
      for (int q = 0; q < 32; ++q) {
        const T xa = __shfl_sync(0xffffffffu, h0, q);
        const T xb = __shfl_sync(0xffffffffu, h1, q);
        y0 += xa * W2[q * kPropHid + lane] + xb * W2[(q + 32) * kPropHid + lane];
        y1 += xa * W2[q * kPropHid + lane + 32] + xb * W2[(q + 32) * kPropHid + lane + 32];
      }
      T z = m_tanh(y0) * w3[lane] + m_tanh(y1) * w3[lane + 32];
      z = wsum(z) + P[kPropOb3];
      if (lane == rr) {
        if (base == 0)
          lg0 = z;
        else
          lg1 = z;
      }
    }
  }
  *out0 = lg0;
  *out1 = lg1;
}

// Softmax probability of row `target_row` among rows [r0, r1) whose logits sit in lanes.
template <typename T>
__device__ T warp_softmax_prob(T lg0, T lg1, int r0, int r1, int target_row) {
  const int lane = threadIdx.x & 31;
  T zmax = -(T)INFINITY;
  for (int r = r0; r < r1; ++r) {
    const T z = __shfl_sync(0xffffffffu, r < 32 ? lg0 : lg1, r & 31);
    zmax = z > zmax ? z : zmax;
  }
  T sum = 0, pt = 0;
  for (int r = r0; r < r1; ++r) {
    const T z = __shfl_sync(0xffffffffu, r < 32 ? lg0 : lg1, r & 31);
    const T w = m_exp(z - zmax);
    sum += w;
    if (r == target_row) pt = w;
  }
  (void)lane;
  return pt / sum;
}

// Appends the antiparallel neighbours of i (in CSR order) as rows (i -> u, x); all lanes
// write the same values (warp-uniform), returns the new count.
__device__ int push_rows(const DevGraph& g, const int8_t* sp, int i, int x, int pa, int pb, int* rc, int* ro, int* rx,
                         int n) {
  const int a = x ? pa : -1, b = x ? pb : -1;
  const int si = spin_x(sp, i, a, b);
  const int k1 = __ldg(g.row_ptr + i + 1);
  for (int k = __ldg(g.row_ptr + i); k < k1; ++k) {
    const int u = __ldg(g.col + k);
    if (spin_x(sp, u, a, b) != si) {
      rc[n] = i;
      ro[n] = u;
      rx[n] = x;
      ++n;
    }
  }
  return n;
}

template <typename T>
__global__ void __launch_bounds__(32 * kMetroMaxWarps) k_metro_warp(const MetroArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevGraph& g = a.g;
  const Dims& m = a.m;
  const int N = m.N, F = m.F, L = m.L, E = m.E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ldw = F + 1;
  // block-shared parameters: W (2F x F) and its transpose Wt (F x (2F + 4)) for 128-bit row loads
  const int ldt = 2 * F + 4;
  T* sW = (T*)smem;                  // [2F][F+1]
  T* sWt = sW + 2 * F * ldw;         // [F][2F+4]
  T* sb = sWt + F * ldt;             // [F]
  T* semb = sb + F;                  // [2][F]
  T* swr = semb + 2 * F;             // [(F+2)][2]
  T* sbr = swr + (F + 2) * 2;        // [2]
  const size_t param_elems = (size_t)2 * F * ldw + (size_t)F * ldt + F + 2 * F + (F + 2) * 2 + 2;
  const size_t param_pad = (param_elems + 3) / 4 * 4;
  T* sP = (T*)smem + param_pad;  // proposal network (when used)
  const size_t prop_pad = a.prop ? ((size_t)kPropParams + 3) / 4 * 4 : 0;
  T* wbase = sP + prop_pad;
  unsigned char* wb = (unsigned char*)wbase + (size_t)warp * a.warp_bytes;
  T* wsm = (T*)wb;                                   // this warp's dH rows and staged dX rows
  T* sX = wsm + a.off_x;                             // [4][2F]
  int* mv = (int*)(wb + a.off_meta);                 // vertex of ball row r
  int* mdeg = mv + a.max_rows;                       // its degree
  int* mnb = mdeg + a.max_rows;                      // offset of its neighbour entries
  int* npos = mnb + a.max_rows;                      // per neighbour entry: position in the ball
  T* nwt = (T*)(mv + ((3 * a.max_rows + a.max_span + 3) / 4 * 4));  // ... and normalised weight
  int* prc = (int*)(nwt + a.max_span);               // proposal rows: centre, partner, exchanged
  int* pro = prc + a.prop_rows;
  int* prx = pro + a.prop_rows;
  int8_t* spin = (int8_t*)(prx + a.prop_rows);
  const T* th = a.theta;
  for (int i = threadIdx.x; i < 2 * F * F; i += blockDim.x) {
    sW[(i / F) * ldw + i % F] = th[m.oW + i];
    sWt[(i % F) * ldt + i / F] = th[m.oW + i];
  }
  for (int i = threadIdx.x; i < F; i += blockDim.x) sb[i] = th[m.ob + i];
  for (int i = threadIdx.x; i < 2 * F; i += blockDim.x) semb[i] = m_tanh(th[m.oWe + i] + th[m.obe + i % F]);
  for (int i = threadIdx.x; i < (F + 2) * 2; i += blockDim.x) swr[i] = th[m.owr + i];
  if (threadIdx.x < 2) sbr[threadIdx.x] = th[m.obr + threadIdx.x];
  if (a.prop)
    for (int i = threadIdx.x; i < kPropParams; i += blockDim.x) sP[i] = (T)a.prop[i];
  __syncthreads();

  const int64_t gwarp = (int64_t)blockIdx.x * a.nwarps + warp;
  const int64_t nwarps = (int64_t)gridDim.x * a.nwarps;
  T* Ybase = a.gws + (size_t)gwarp * a.ws_elems;  // Y^l at Ybase + (l-1)*N*F
  T* Hs0 = Ybase + (size_t)L * N * F;
  T* Hs1 = Hs0 + (size_t)N * F;
  T* dYg = Ybase;  // dY^l rows at dYg + off_dy[l]
  const int f0 = lane, f1 = lane + 32;
  const bool has0 = f0 < F, has1 = f1 < F;
  const int64_t n_steps = (int64_t)a.n_sweeps * N;
  const int n_rec = a.record_every > 0 ? a.n_sweeps / a.record_every : 0;

  for (int64_t ch = gwarp; ch < a.C; ch += nwarps) {
    for (int v = lane; v < N; v += 32) spin[v] = a.chain_spins[ch * N + v];
    __syncwarp();
    // ---- forward: Y^1..Y^L of the chain's state (H scratch ping-pong) ----
    for (int v = 0; v < N; ++v) {
      const int c = spin[v] > 0 ? 0 : 1;
      if (has0) Hs0[(size_t)v * F + f0] = semb[c * F + f0];
      if (has1) Hs0[(size_t)v * F + f1] = semb[c * F + f1];
    }
    __syncwarp();
    for (int l = 1; l <= L; ++l) {
      const T* Hp = (l & 1) ? Hs0 : Hs1;
      T* Hn = (l & 1) ? Hs1 : Hs0;
      T* Y = Ybase + (size_t)(l - 1) * N * F;
      for (int v = 0; v < N; ++v) {
        T ag0 = 0, ag1 = 0;
        const int k1 = __ldg(g.row_ptr + v + 1);
        for (int k = __ldg(g.row_ptr + v); k < k1; ++k) {
          const T w = (T)__ldg(g.wd + k);
          const T* hu = Hp + (size_t)__ldg(g.col + k) * F;
          if (has0) ag0 += w * hu[f0];
          if (has1) ag1 += w * hu[f1];
        }
        const T sf0 = has0 ? Hp[(size_t)v * F + f0] : (T)0, sf1 = has1 ? Hp[(size_t)v * F + f1] : (T)0;
        T y0 = has0 ? sb[f0] : (T)0, y1 = has1 ? sb[f1] : (T)0;
        for (int kk = 0; kk < F; ++kk) {
          const T av = __shfl_sync(0xffffffffu, kk < 32 ? ag0 : ag1, kk & 31);
          const T sv = __shfl_sync(0xffffffffu, kk < 32 ? sf0 : sf1, kk & 31);
          if (has0) y0 += av * sW[kk * ldw + f0] + sv * sW[(F + kk) * ldw + f0];
          if (has1) y1 += av * sW[kk * ldw + f1] + sv * sW[(F + kk) * ldw + f1];
        }
        if (has0) {
          Y[(size_t)v * F + f0] = y0;
          Hn[(size_t)v * F + f0] = m_tanh(y0);
        }
        if (has1) {
          Y[(size_t)v * F + f1] = y1;
          Hn[(size_t)v * F + f1] = m_tanh(y1);
        }
      }
      __syncwarp();
    }
    int accepts = 0;
    uint64_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;  // Philox words of step (k0 + lane)
    for (int64_t k = 0; k < n_steps; ++k) {
      if ((k & 31) == 0) {
        const U64x4 w = philox4x64_10(a.seed, (uint64_t)ch, U64x4{a.step0 + (uint64_t)(k + lane), 0, 0, 0});
        w0 = w.x;
        w1 = w.y;
        w2 = w.z;
        w3 = w.w;
      }
      const uint64_t r0 = __shfl_sync(0xffffffffu, w0, (int)(k & 31));
      const uint64_t r1 = __shfl_sync(0xffffffffu, w1, (int)(k & 31));
      int e = -1, kind = 1;
      bool move = false;
      T logq = 0;
      if (!a.prop) {
        e = (int)__umul64hi(r0, (uint64_t)E);
        move = spin[__ldg(g.edges + 2 * e)] != spin[__ldg(g.edges + 2 * e + 1)];
      } else {
        const uint64_t r2 = __shfl_sync(0xffffffffu, w2, (int)(k & 31));
        const uint64_t r3 = __shfl_sync(0xffffffffu, w3, (int)(k & 31));
        const T eps = (T)a.prop_eps;
        int pi = -1, pj = -1, n = 0;
        T pij = 0, lg0 = 0, lg1 = 0;
        if ((double)(r3 >> 40) * 0x1.0p-24 < a.prop_eps) {
          e = (int)__umul64hi(r0, (uint64_t)E);
          pi = __ldg(g.edges + 2 * e);
          pj = __ldg(g.edges + 2 * e + 1);
          move = spin[pi] != spin[pj];
          if (move) n = push_rows(g, spin, pi, 0, pi, pj, prc, pro, prx, 0);
        } else {
          kind = 2;
          pi = (int)__umul64hi(r2, (uint64_t)N);
          const int n1 = push_rows(g, spin, pi, 0, -1, -1, prc, pro, prx, 0);
          __syncwarp();
          if (n1 > 0) {
            // the partner j ~ pi_i(. | s), by the categorical uniform (r3 mod 2^32) 2^-32
            warp_logits<T>(g, spin, sP, prc, pro, prx, n1, -1, -1, &lg0, &lg1);
            T zmax = -(T)INFINITY;
            for (int r = 0; r < n1; ++r) {
              const T z = __shfl_sync(0xffffffffu, r < 32 ? lg0 : lg1, r & 31);
              zmax = z > zmax ? z : zmax;
            }
            T sum = 0;
            for (int r = 0; r < n1; ++r) sum += m_exp(__shfl_sync(0xffffffffu, r < 32 ? lg0 : lg1, r & 31) - zmax);
            const T uc = (T)((double)(r3 & 0xFFFFFFFFull) * 0x1.0p-32);
            T cum = 0;
            int pick = n1 - 1;
            for (int r = 0; r < n1; ++r) {
              const T pr = m_exp(__shfl_sync(0xffffffffu, r < 32 ? lg0 : lg1, r & 31) - zmax) / sum;
              cum += pr;
              if (uc < cum) {
                pick = r;
                pij = pr;
                break;
              }
              if (r == n1 - 1) pij = pr;
            }
            pj = pro[pick];
            const int k1 = __ldg(g.row_ptr + pi + 1);
            for (int kk = __ldg(g.row_ptr + pi); kk < k1; ++kk)
              if (__ldg(g.col + kk) == pj) e = __ldg(g.col_edge + kk);
            move = true;
          }
          __syncwarp();
        }
        if (move) {
          // the exact mixture proposal density both ways: q(s -> s') and q(s' -> s)
          int g0 = n;  // rows [0, g0): cand(i, s) (plain moves only)
          n = push_rows(g, spin, pj, 0, pi, pj, prc, pro, prx, n);
          const int g1 = n;
          n = push_rows(g, spin, pi, 1, pi, pj, prc, pro, prx, n);
          const int g2 = n;
          n = push_rows(g, spin, pj, 1, pi, pj, prc, pro, prx, n);
          __syncwarp();
          warp_logits<T>(g, spin, sP, prc, pro, prx, n, pi, pj, &lg0, &lg1);
          const T p_ij = kind == 1 ? warp_softmax_prob<T>(lg0, lg1, 0, g0, row_of(pro, 0, g0, pj)) : pij;
          const T p_ji = warp_softmax_prob<T>(lg0, lg1, g0, g1, row_of(pro, g0, g1, pi));
          const T p_ij2 = warp_softmax_prob<T>(lg0, lg1, g1, g2, row_of(pro, g1, g2, pj));
          const T p_ji2 = warp_softmax_prob<T>(lg0, lg1, g2, n, row_of(pro, g2, n, pi));
          const T wl = ((T)1 - eps) / (T)N, wp = eps / (T)E;
          logq = (T)(log((double)(wl * (p_ij2 + p_ji2) + wp)) - log((double)(wl * (p_ij + p_ji) + wp)));
        }
      }
      double* tr = a.trace ? a.trace + ((size_t)ch * n_steps + k) * 4 : nullptr;
      if (!move) {
        if (tr && lane == 0) {
          tr[0] = (double)e;
          tr[1] = 0.0;
          tr[2] = __longlong_as_double(0x7ff8000000000000ll);
          tr[3] = (double)kind;
        }
      } else {
        const int i = __ldg(g.edges + 2 * e), j = __ldg(g.edges + 2 * e + 1);
        const int bo = __ldg(g.ball_off + e);
        const int* bsz = g.ball_size + (size_t)e * (g.Lmax + 1);
        // layer 0: dH^0 rows (i, j)
        {
          T* d0 = wsm + a.off_dh[0];
          const int ci = spin[i] > 0 ? 0 : 1, cj = spin[j] > 0 ? 0 : 1;
          if (has0) {
            d0[f0] = semb[cj * F + f0] - semb[ci * F + f0];
            d0[F + f0] = semb[ci * F + f0] - semb[cj * F + f0];
          }
          if (has1) {
            d0[f1] = semb[cj * F + f1] - semb[ci * F + f1];
            d0[F + f1] = semb[ci * F + f1] - semb[cj * F + f1];
          }
          __syncwarp();
        }
        // row metadata of ball_L(e): vertex, degree, neighbour positions and weights
        const int RL = __ldg(bsz + L);
        const int nb_base = __ldg(g.row_nbr + bo);
        for (int r = lane; r < RL; r += 32) {
          const int v = __ldg(g.ball_vert + bo + r);
          const int k0 = __ldg(g.row_ptr + v), dg = __ldg(g.row_ptr + v + 1) - k0;
          const int o = __ldg(g.row_nbr + bo + r) - nb_base;
          mv[r] = v;
          mdeg[r] = dg;
          mnb[r] = o;
          for (int t = 0; t < dg; ++t) {
            npos[o + t] = __ldg(g.nbr_pos + nb_base + o + t);
            nwt[o + t] = (T)__ldg(g.wd + k0 + t);
          }
        }
        __syncwarp();
        T pre = 0, pim = 0;
        for (int l = 1; l <= L; ++l) {
          const int sprev = __ldg(bsz + l - 1), R = __ldg(bsz + l);
          const T* dprev = wsm + a.off_dh[l - 1];
          T* dcur = l < L ? wsm + a.off_dh[l] : nullptr;
          T* dyl = dYg + a.off_dy[l];
          const T* Y = Ybase + (size_t)(l - 1) * N * F;
          for (int rb = 0; rb < R; rb += 4) {
            // stage dX = [A_hat dH^{l-1} ; dH^{l-1}] of rows rb..rb+3 (zeros past R)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int r = rb + q;
              T ag0 = 0, ag1 = 0, sf0 = 0, sf1 = 0;
              if (r < R) {
                const int o = mnb[r], dg = mdeg[r];
                for (int t = 0; t < dg; ++t) {
                  const int p = npos[o + t];
                  if (p < sprev) {
                    const T w = nwt[o + t];
                    if (has0) ag0 += w * dprev[(size_t)p * F + f0];
                    if (has1) ag1 += w * dprev[(size_t)p * F + f1];
                  }
                }
                if (r < sprev) {
                  if (has0) sf0 = dprev[(size_t)r * F + f0];
                  if (has1) sf1 = dprev[(size_t)r * F + f1];
                }
              }
              T* x = sX + q * 2 * F;
              if (has0) {
                x[f0] = ag0;
                x[F + f0] = sf0;
              }
              if (has1) {
                x[f1] = ag1;
                x[F + f1] = sf1;
              }
            }
            __syncwarp();
            // prefetch the cached pre-activations of the 4 rows (hidden behind the GEMM)
            T yc0[4], yc1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int r = rb + q < R ? rb + q : R - 1;
              const T* yr = Y + (size_t)mv[r] * F;
              yc0[q] = has0 ? yr[f0] : (T)0;
              yc1[q] = has1 ? yr[f1] : (T)0;
            }
            // dY = dX W for the 4 rows (lane: output columns f0, f1), 4 inputs per load
            T y00 = 0, y10 = 0, y20 = 0, y30 = 0, y01 = 0, y11 = 0, y21 = 0, y31 = 0;
            const T* wt0 = sWt + (size_t)(has0 ? f0 : 0) * ldt;
            const T* wt1 = sWt + (size_t)(has1 ? f1 : 0) * ldt;
#pragma unroll 2
            for (int q = 0; q < 2 * F; q += 4) {
              T xa[4], xb[4], xc[4], xd[4], wa[4], wb[4];
              load4(sX + q, xa);
              load4(sX + 2 * F + q, xb);
              load4(sX + 4 * F + q, xc);
              load4(sX + 6 * F + q, xd);
              load4(wt0 + q, wa);
              if (has1) load4(wt1 + q, wb);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                y00 += xa[u] * wa[u];
                y10 += xb[u] * wa[u];
                y20 += xc[u] * wa[u];
                y30 += xd[u] * wa[u];
                if (has1) {
                  y01 += xa[u] * wb[u];
                  y11 += xb[u] * wb[u];
                  y21 += xc[u] * wb[u];
                  y31 += xd[u] * wb[u];
                }
              }
            }
            __syncwarp();
            const T ys0[4] = {y00, y10, y20, y30};
            const T ys1[4] = {y01, y11, y21, y31};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int r = rb + q;
              if (r >= R) break;
              if (has0) {
                const T d = dtanh(yc0[q], ys0[q]);
                dyl[(size_t)r * F + f0] = ys0[q];
                if (l < L)
                  dcur[(size_t)r * F + f0] = d;
                else {
                  pre += d * swr[2 * f0];
                  pim += d * swr[2 * f0 + 1];
                }
              }
              if (has1) {
                const T d = dtanh(yc1[q], ys1[q]);
                dyl[(size_t)r * F + f1] = ys1[q];
                if (l < L)
                  dcur[(size_t)r * F + f1] = d;
                else {
                  pre += d * swr[2 * f1];
                  pim += d * swr[2 * f1 + 1];
                }
              }
            }
          }
          __syncwarp();
        }
        const T dre = wsum(pre);
        const T dim = wsum(pim);
        (void)dim;
        T value;
        bool acc;
        if (a.prop) {
          value = (T)2 * dre + logq;
          acc = m_accept_log<T>(r1, value);
        } else {
          value = dre;
          acc = m_accept<T>(r1, dre);
        }
        if (tr && lane == 0) {
          tr[0] = (double)e;
          tr[1] = acc ? 1.0 : 0.0;
          tr[2] = (double)value;
          tr[3] = (double)kind;
        }
        if (acc) {
          ++accepts;
          for (int l = 1; l <= L; ++l) {
            const int R = __ldg(bsz + l);
            const T* dy = dYg + a.off_dy[l];
            T* Y = Ybase + (size_t)(l - 1) * N * F;
            for (int r = 0; r < R; ++r) {
              const int v = mv[r];
              if (has0) Y[(size_t)v * F + f0] += dy[(size_t)r * F + f0];
              if (has1) Y[(size_t)v * F + f1] += dy[(size_t)r * F + f1];
            }
          }
          if (lane == 0) {
            const int8_t t = spin[i];
            spin[i] = spin[j];
            spin[j] = t;
          }
        }
        __syncwarp();
      }
      if ((k + 1) % N == 0 && a.record_every > 0) {
        const int sweep = (int)((k + 1) / N);
        if (sweep % a.record_every == 0) {
          const int rec = sweep / a.record_every - 1;
          if (rec < n_rec) {
            if (a.samples_out)
              for (int v = lane; v < N; v += 32) a.samples_out[((size_t)rec * a.C + ch) * N + v] = spin[v];
            if (a.logpsi_out) {
              // log Psi = sum_v [tanh(Y^L_v) ; onehot_v] . w_r + b_r
              const T* YL = Ybase + (size_t)(L - 1) * N * F;
              T z0 = 0, z1 = 0;
              int up = 0;
              for (int v = 0; v < N; ++v) {
                if (has0) z0 += L > 0 ? m_tanh(YL[(size_t)v * F + f0]) : semb[(spin[v] > 0 ? 0 : 1) * F + f0];
                if (has1) z1 += L > 0 ? m_tanh(YL[(size_t)v * F + f1]) : semb[(spin[v] > 0 ? 0 : 1) * F + f1];
                up += spin[v] > 0;
              }
              T re = (has0 ? z0 * swr[2 * f0] : (T)0) + (has1 ? z1 * swr[2 * f1] : (T)0);
              T im = (has0 ? z0 * swr[2 * f0 + 1] : (T)0) + (has1 ? z1 * swr[2 * f1 + 1] : (T)0);
              re = wsum(re);
              im = wsum(im);
              if (lane == 0) {
                const int dn = N - up;
                a.logpsi_out[((size_t)rec * a.C + ch) * 2] =
                    (double)(re + (T)up * swr[2 * F] + (T)dn * swr[2 * (F + 1)] + sbr[0]);
                a.logpsi_out[((size_t)rec * a.C + ch) * 2 + 1] =
                    (double)(im + (T)up * swr[2 * F + 1] + (T)dn * swr[2 * (F + 1) + 1] + sbr[1]);
              }
            }
          }
        }
      }
    }
    for (int v = lane; v < N; v += 32) a.chain_spins[ch * N + v] = spin[v];
    if (lane == 0 && a.n_acc) a.n_acc[ch] += accepts;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------------
struct MetroPlan {
  int grid = 0;
  int smem = 0;
  int nwarps = 0;
  int warp_bytes = 0;
  int off_dh[kMaxL + 1] = {0};
  int off_dy[kMaxL + 1] = {0};
  int off_x = 0, off_meta = 0, max_rows = 0, max_span = 0, prop_rows = 0;
  size_t ws_elems = 0;
  size_t ws_bytes = 0;
};

template <typename T>
static gna_status metro_plan(const gna_graph* g, const Dims& m, int64_t C, int with_prop, MetroPlan* p) {
  if (m.L < 1 || m.F > 64) return GNA_ERR_UNSUPPORTED;
  if (with_prop && g->max_deg > 16) return GNA_ERR_UNSUPPORTED;
  p->prop_rows = with_prop ? 4 * (g->max_deg > 0 ? g->max_deg : 1) : 0;
  DeviceInfo di;
  gna_status st = device_info(&di);
  if (st != GNA_OK) return st;
  const int F = m.F, L = m.L;
  // per-warp shared memory: dH rows (l < L), 4 staged dX rows, row metadata, spins
  int o = 0;
  for (int l = 0; l < L; ++l) {
    p->off_dh[l] = o;
    o += g->max_ball[l] * F;
  }
  p->off_x = o;
  o += 4 * 2 * F;
  size_t bytes = (size_t)o * sizeof(T);
  bytes = (bytes + 15) / 16 * 16;
  p->off_meta = (int)bytes;
  p->max_rows = g->max_ball[L];
  p->max_span = g->max_span[L];
  const int meta_ints = (3 * p->max_rows + p->max_span + 3) / 4 * 4;  // keeps the weights 16-byte aligned
  bytes += (size_t)meta_ints * 4 + (size_t)p->max_span * sizeof(T) + (size_t)3 * p->prop_rows * 4 + (size_t)m.N;
  p->warp_bytes = (int)((bytes + 15) / 16 * 16);
  // per-warp workspace slot: Y^1..Y^L, two H scratch layers, dY^1..dY^L rows
  size_t e = (size_t)(L + 2) * m.N * F;
  for (int l = 1; l <= L; ++l) {
    p->off_dy[l] = (int)e;
    e += (size_t)g->max_ball[l] * F;
  }
  p->ws_elems = (e + 31) / 32 * 32;
  const size_t param_elems = (size_t)2 * F * (F + 1) + (size_t)F * (2 * F + 4) + F + 2 * F + (F + 2) * 2 + 2;
  const size_t param_bytes = ((param_elems + 3) / 4 * 4 + (with_prop ? ((size_t)kPropParams + 3) / 4 * 4 : 0)) * sizeof(T);
  auto smem_for = [&](int nw) { return param_bytes + (size_t)nw * p->warp_bytes; };
  int nw = kMetroMaxWarps;
  while (nw > 0 && smem_for(nw) > (size_t)di.smem_optin - 1024) --nw;
  if (nw < 2) return GNA_ERR_UNSUPPORTED;
  p->nwarps = nw;
  p->smem = (int)smem_for(nw);
  GNA_CUDA_TRY(cudaFuncSetAttribute((const void*)k_metro_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, p->smem));
  int occ = 0;
  GNA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_metro_warp<T>, 32 * nw, p->smem));
  if (occ < 1) occ = 1;
  int64_t grid = (int64_t)di.sms * occ;
  const int64_t need = (C + nw - 1) / nw;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  p->grid = (int)grid;
  p->ws_bytes = align_up((size_t)grid * nw * p->ws_elems * sizeof(T));
  return GNA_OK;
}

gna_status metro_workspace(const gna_graph* g, const Dims& m, int prec, int64_t C, int with_prop, size_t* bytes) {
  if (C == 0) {
    *bytes = 0;
    return GNA_OK;
  }
  MetroPlan p;
  gna_status st = prec == GNA_PREC_FP64 ? metro_plan<double>(g, m, C, with_prop, &p)
                                        : metro_plan<float>(g, m, C, with_prop, &p);
  if (st != GNA_OK) return st;
  *bytes = p.ws_bytes;
  return GNA_OK;
}

template <typename T>
static gna_status metro_launch_t(const MetroCall& mc, void* ws, size_t ws_bytes, cudaStream_t stream) {
  MetroPlan p;
  gna_status st = metro_plan<T>(mc.g, mc.m, mc.C, mc.prop != nullptr, &p);
  if (st != GNA_OK) return st;
  if (ws_bytes < p.ws_bytes || !ws) return GNA_ERR_WORKSPACE;
  MetroArgs<T> a;
  a.g = mc.g->d;
  a.m = mc.m;
  for (int l = 0; l <= kMaxL; ++l) {
    a.maxball[l] = (l <= mc.m.L && l <= mc.g->d.Lmax) ? mc.g->max_ball[l] : 0;
    a.off_dh[l] = p.off_dh[l];
    a.off_dy[l] = p.off_dy[l];
  }
  a.off_x = p.off_x;
  a.off_meta = p.off_meta;
  a.max_rows = p.max_rows;
  a.max_span = p.max_span;
  a.warp_bytes = p.warp_bytes;
  a.prop_rows = p.prop_rows;
  a.prop = mc.prop;
  a.prop_eps = mc.prop_eps;
  a.nwarps = p.nwarps;
  a.theta = (const T*)mc.theta;
  a.chain_spins = mc.chain_spins;
  a.C = mc.C;
  a.n_sweeps = mc.n_sweeps;
  a.record_every = mc.record_every;
  a.seed = mc.seed;
  a.step0 = mc.step0;
  a.samples_out = mc.samples_out;
  a.logpsi_out = mc.logpsi_out;
  a.n_acc = mc.n_acc;
  a.trace = mc.trace;
  a.gws = (T*)ws;
  a.ws_elems = p.ws_elems;
  k_metro_warp<T><<<p.grid, 32 * p.nwarps, p.smem, stream>>>(a);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

gna_status metro_run(const MetroCall& mc, int prec, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (mc.C == 0 || mc.n_sweeps == 0) return GNA_OK;
  return prec == GNA_PREC_FP64 ? metro_launch_t<double>(mc, ws, ws_bytes, stream)
                               : metro_launch_t<float>(mc, ws, ws_bytes, stream);
}

}  // namespace gna

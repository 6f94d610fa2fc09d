// Internal definitions shared by the translation units of libgna.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/gna.h"

namespace gna {

constexpr int kMaxF = 64;
constexpr int kMaxL = 8;
constexpr int kThreads = 256;  // threads per CTA of the SIMT kernels

// Device-resident graph.  All arrays are owned by the handle.
struct DevGraph {
  int n = 0, E = 0, Lmax = 0;
  const int* row_ptr = nullptr;   // [n+1]
  const int* col = nullptr;       // [2E]   neighbour u of v at row_ptr[v]..row_ptr[v+1]
  const int* col_edge = nullptr;  // [2E]   bond index of that CSR entry
  const float* wf = nullptr;      // [2E]   1/sqrt(d_v d_u), float32
  const double* wd = nullptr;     // [2E]   same, float64
  const int* edges = nullptr;     // [E][2]
  const double* J = nullptr;      // [E]    off-diagonal coupling of bond e (J, or Jxy of XXZ bonds)
  const double* Jz = nullptr;     // [E]    diagonal S^z S^z coupling
  const double* hz = nullptr;     // [E]    field on both ends of bond e
  const double* cb = nullptr;     // [E]    constant of bond e
  // Nested neighbourhoods of each bond, for l = 0..Lmax:
  const int* ball_off = nullptr;  // [E+1]  start of bond e's rows in ball_vert / row_nbr
  const int* ball_size = nullptr; // [E][Lmax+1]
  const int* ball_vert = nullptr; // [sum]  vertex of row r (ball_l = first ball_size[l] rows)
  const int* row_nbr = nullptr;   // [sum]  start of row r's entries in nbr_pos
  const int* nbr_pos = nullptr;   // [...]  for neighbour k of the row's vertex (CSR order):
                                  //        its row position in this bond's ball_Lmax, or
                                  //        INT_MAX when outside ball_Lmax
  // Compact forms of the same tables for staging in shared memory (a vertex or a ball
  // position fits 16 bits: n <= 4096):
  const int* ball_span = nullptr;      // [E][Lmax+1] entries (sum of degrees) of the first ball_size rows
  const int* row_pack = nullptr;       // [sum]  v | (start of the row's entries within the bond's << 16)
  const int16_t* nbr_pos16 = nullptr;  // [...]  nbr_pos, 32767 outside ball_Lmax
  const int* bond_ent = nullptr;       // [E]    start of bond e's entries in nbr_pos / nbr_pos16
};

// Diagonal element of bond e's Hamiltonian for S^z eigenvalues s_i/2, s_j/2 (float64):
// Jz/4 s_i s_j + hz/2 (s_i + s_j) + c.  Heisenberg bonds have Jz = J and hz = c = 0.
__device__ inline double bond_diag(const DevGraph& g, int e, int si, int sj) {
  return __ldg(g.Jz + e) * 0.25 * (double)(si * sj) + __ldg(g.hz + e) * 0.5 * (double)(si + sj) +
         __ldg(g.cb + e);
}

}  // namespace gna

struct gna_graph {
  gna::DevGraph d;
  int device = 0;
  std::vector<int> h_row_ptr, h_col, h_edges, h_ball_size, h_ball_off;
  std::vector<double> h_J;  // off-diagonal couplings
  std::vector<int> max_ball;  // [Lmax+1] max over bonds of |ball_l|
  std::vector<int> max_span;  // [Lmax+1] max over bonds of sum of degrees over ball_l rows
  int max_deg = 0;
  bool pack_ok = true;  // every bond's entries fit the 16-bit starts of row_pack
  std::vector<void*> allocations;
};

namespace gna {

// ---- dims ------------------------------------------------------------------------
struct Dims {
  int N, E, F, L, shared, P;
  int act;                         // gna_act: GNA_ACT_TANH or GNA_ACT_RELU_LN
  int oWe, obe, oW, ob, owr, obr;  // parameter offsets (layer l: oW + l*strideW when unshared)
  int strideW;                     // 2F*F + F when unshared, 0 when shared
};

inline Dims make_dims(const gna_graph* g, const gna_model_desc* d) {
  Dims m;
  m.N = g->d.n;
  m.E = g->d.E;
  m.F = d->F;
  m.L = d->L;
  m.shared = d->shared_weights;
  m.act = d->act;
  const int F = d->F;
  m.oWe = 0;
  m.obe = 2 * F;
  m.oW = 3 * F;
  m.ob = m.oW + 2 * F * F;
  const int nl = d->shared_weights ? 1 : d->L;
  m.strideW = d->shared_weights ? 0 : (2 * F * F + F);
  m.owr = 3 * F + nl * (2 * F * F + F);
  m.obr = m.owr + (F + 2) * 2;
  m.P = m.obr + 2;
  return m;
}

// ---- status helpers ---------------------------------------------------------------
#define GNA_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) {                       \
      gna::set_last_cuda_error(_e);                \
      return GNA_ERR_CUDA;                         \
    }                                              \
  } while (0)

void set_last_cuda_error(cudaError_t e);

struct DeviceInfo {
  int sms = 0;
  int smem_optin = 0;  // max dynamic shared memory per block (opt-in), bytes
  int cc = 0;
};
gna_status device_info(DeviceInfo* out);

// Arguments of one SIMT launch (simt.cu).  op: 0 forward, 1 full local energy,
// 2 incremental local energy, 3 Metropolis sweeps, 4 backward.
struct SimtCall {
  const gna_graph* g;
  Dims m;
  int op;
  const void* theta;
  const int8_t* spins;
  int64_t B;
  double* logpsi = nullptr;
  double* eloc = nullptr;
  float* dlogpsi = nullptr;
  const double* cot = nullptr;
  double* grad = nullptr;
  int8_t* chain_spins = nullptr;
  int32_t n_sweeps = 0, record_every = 0;
  uint64_t seed = 0, step0 = 0;
  int8_t* samples_out = nullptr;
  double* logpsi_out = nullptr;
  int32_t* n_acc = nullptr;
  double* trace = nullptr;
  const float* prop = nullptr;  // learned proposal parameters (Metropolis) or NULL
  double prop_eps = 0.0;
};

// Entry points of the translation units.
gna_status simt_workspace(const gna_graph* g, const Dims& m, int prec, int op, int64_t B, size_t* bytes);
gna_status simt_run(const SimtCall& sc, int prec, void* ws, size_t ws_bytes, cudaStream_t stream);
gna_status simt_backward_static(const SimtCall& sc, int prec, cudaStream_t stream);
// Device address and size of the library's fixed backward scratch array on the current device.
gna_status static_scratch(void** base, size_t* bytes);
size_t dedup_workspace(int64_t B, int N);
gna_status dedup_run(int N, const int8_t* spins, const double* logpsi, int64_t B, int8_t* us, double* ul, double* uc,
                     int64_t* n_unique, void* ws, size_t ws_bytes, cudaStream_t st);
size_t isgo_weights_ws(int64_t B);
gna_status isgo_weights_launch(const double* lp, const double* lp0, const double* E, const double* counts, int64_t B,
                               double* cot, double* stats, void* ws, cudaStream_t st);
gna_status sgd_launch(int prec, void* theta, const double* grad, double lr, int P, cudaStream_t st);
gna_status isgo_partials_launch(const double* lp, const double* lp0, const double* E, const double* counts, int64_t B,
                                double* part4, void* ws, cudaStream_t st);
gna_status isgo_finish_launch(const double* lp, const double* lp0, const double* E, const double* counts, int64_t B,
                              const double* global4, double* cot, double* part3, void* ws, cudaStream_t st);
gna_status philox_launch(const uint64_t* keys, const uint64_t* ctrs, int64_t n, uint64_t* out, cudaStream_t st);
gna_status isgo_read_status(int* flags, int clear);

// ---- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------------------
struct U64x4 {
  uint64_t x, y, z, w;
};

__host__ __device__ inline void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
#ifdef __CUDA_ARCH__
  *lo = a * b;
  *hi = __umul64hi(a, b);
#else
  unsigned __int128 p = (unsigned __int128)a * b;
  *lo = (uint64_t)p;
  *hi = (uint64_t)(p >> 64);
#endif
}

__host__ __device__ inline U64x4 philox4x64_10(uint64_t k0, uint64_t k1, U64x4 c) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c.x, &hi0, &lo0);
    mulhilo64(M1, c.z, &hi1, &lo1);
    U64x4 n;
    n.x = hi1 ^ c.y ^ k0;
    n.y = lo1;
    n.z = hi0 ^ c.w ^ k1;
    n.w = lo0;
    c = n;
  }
  return c;
}

// ---- workspace carving --------------------------------------------------------------
inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Launch plan of a per-sample SIMT kernel.
struct Plan {
  int grid = 0;            // CTAs (persistent: each loops over samples)
  int smem = 0;            // dynamic shared memory bytes
  int region_in_smem = 0;  // 1: the per-sample region is in shared memory
  size_t region_elems = 0; // elements of T per CTA in the per-sample region
  size_t ws_bytes = 0;     // workspace bytes for the whole launch
  int G = 1;               // bonds processed together (local energy)
  int partial_in_smem = 0; // backward: per-CTA gradient partial in shared memory
  int prop_rows = 0;       // Metropolis with a proposal network: row buffer capacity
};

}  // namespace gna

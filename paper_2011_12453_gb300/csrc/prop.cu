// Learned exchange proposal: the network 9 -> 64 -> 64 -> 1 (tanh hidden units) that
// scores an exchange of site i with its antiparallel neighbour j from local spin
// features, its training step (mean squared error against the plain exchange's log
// acceptance min(0, 2 Re Delta_e), hand-written reverse mode, Adam), and batched logits.
// Not part of arXiv:2011.12453; it proposes moves for the paper's MCMC step.
//
// Rows are (configuration b, bond e, orientation o): o = 0 scores i -> j, o = 1 scores
// j -> i for e = (i, j); parallel bonds are masked.  One CTA processes tiles of 64 rows:
// features, the two hidden layers and the logit in shared memory, then every parameter's
// gradient contribution summed over the tile by the one thread that owns it (fixed
// order, no atomics).  Per-CTA partials are reduced in float64 by a second kernel.
#include "common.cuh"
#include "prop.cuh"

namespace gna {

constexpr int kPropThreads = 256;
constexpr int kTile = 64;

struct PropArgs {
  DevGraph g;
  const int8_t* spins;     // [B][N]
  const float* dlogpsi;    // [B][E] (training) or NULL
  const float* params;     // [kPropParams]
  int64_t B;
  int mode;                // 0: logits, 1: gradient
  float* logits;           // [B][E][2] (mode 0)
  double* partial;         // [grid][kPropParams + 2] (mode 1): gradient sums, loss sum, row count
};

__device__ __forceinline__ float nbr_spin_sum(const DevGraph& g, const int8_t* s, int v) {
  float acc = 0.f;
  const int k1 = __ldg(g.row_ptr + v + 1);
  for (int k = __ldg(g.row_ptr + v); k < k1; ++k) acc += (float)s[__ldg(g.col + k)];
  return acc;
}

// Features of the ordered pair (i, j) (see the oracle's description): 9 floats.
__device__ void pair_features(const DevGraph& g, const int8_t* s, int i, int j, float J, float* phi) {
  const int di = __ldg(g.row_ptr + i + 1) - __ldg(g.row_ptr + i);
  const int dj = __ldg(g.row_ptr + j + 1) - __ldg(g.row_ptr + j);
  const float si = (float)s[i], sj = (float)s[j];
  const float ni = nbr_spin_sum(g, s, i), nj = nbr_spin_sum(g, s, j);
  float bi = 0.f, bj = 0.f;
  int ci = 0, cj = 0;
  for (int k = __ldg(g.row_ptr + i); k < __ldg(g.row_ptr + i + 1); ++k) {
    const int u = __ldg(g.col + k);
    if (u == j) continue;
    const int du = __ldg(g.row_ptr + u + 1) - __ldg(g.row_ptr + u);
    bi += nbr_spin_sum(g, s, u) / (float)du;
    ++ci;
  }
  for (int k = __ldg(g.row_ptr + j); k < __ldg(g.row_ptr + j + 1); ++k) {
    const int u = __ldg(g.col + k);
    if (u == i) continue;
    const int du = __ldg(g.row_ptr + u + 1) - __ldg(g.row_ptr + u);
    bj += nbr_spin_sum(g, s, u) / (float)du;
    ++cj;
  }
  phi[0] = si;
  phi[1] = sj;
  phi[2] = J;
  phi[3] = 1.f / (float)di;
  phi[4] = 1.f / (float)dj;
  phi[5] = (ni - sj) / (float)max(di - 1, 1);
  phi[6] = (nj - si) / (float)max(dj - 1, 1);
  phi[7] = ci ? bi / (float)ci : 0.f;
  phi[8] = cj ? bj / (float)cj : 0.f;
}

// Dynamic shared memory of k_prop (floats): parameters, features, two hidden layers,
// one gradient buffer, per-row logit gradient and mask.
constexpr int kPropSmemFloats = kPropParams + 3 + kTile * (kPropIn + 1) + 3 * kTile * (kPropHid + 1) + 2 * kTile;

__global__ void __launch_bounds__(kPropThreads) k_prop(const PropArgs a) {
  extern __shared__ __align__(16) float prop_smem[];
  float* sP = prop_smem;
  float(*sPhi)[kPropIn + 1] = reinterpret_cast<float(*)[kPropIn + 1]>(sP + kPropParams + 3);
  float(*sH1)[kPropHid + 1] = reinterpret_cast<float(*)[kPropHid + 1]>(&sPhi[kTile][0]);
  float(*sH2)[kPropHid + 1] = sH1 + kTile;
  float(*sD)[kPropHid + 1] = sH2 + kTile;  // dZ2, then dZ1
  float* sDl = &sD[kTile][0];               // d loss / d logit (masked)
  float* sMask = sDl + kTile;
  const int tid = threadIdx.x;
  const DevGraph& g = a.g;
  const int N = g.n, E = g.E;
  for (int i = tid; i < kPropParams; i += blockDim.x) sP[i] = a.params[i];
  const float* W1 = sP + kPropOW1;
  const float* b1 = sP + kPropOb1;
  const float* W2 = sP + kPropOW2;
  const float* b2 = sP + kPropOb2;
  const float* w3 = sP + kPropOw3;
  // gradient entries owned by this thread: p = tid + k * blockDim.x
  constexpr int kOwn = (kPropParams + kPropThreads - 1) / kPropThreads;
  float acc[kOwn];
#pragma unroll
  for (int k = 0; k < kOwn; ++k) acc[k] = 0.f;
  float loss = 0.f, count = 0.f;
  __syncthreads();
  const int64_t rows = a.B * (int64_t)E * 2;
  const int64_t tiles = (rows + kTile - 1) / kTile;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t r0 = t * kTile;
    if (tid < kTile) {
      const int64_t row = r0 + tid;
      float m = 0.f;
      float phi[kPropIn] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      float tgt = 0.f;
      if (row < rows) {
        const int64_t b = row / (2 * E);
        const int e = (int)((row / 2) % E), o = (int)(row % 2);
        const int8_t* s = a.spins + b * N;
        const int i0 = __ldg(g.edges + 2 * e), j0 = __ldg(g.edges + 2 * e + 1);
        if (s[i0] != s[j0]) {
          m = 1.f;
          const int i = o ? j0 : i0, j = o ? i0 : j0;
          pair_features(g, s, i, j, (float)__ldg(g.J + e), phi);
          if (a.mode == 1) tgt = fminf(0.f, 2.f * a.dlogpsi[b * E + e]);
        }
      }
#pragma unroll
      for (int f = 0; f < kPropIn; ++f) sPhi[tid][f] = phi[f];
      sMask[tid] = m;
      sDl[tid] = tgt;  // target for now
    }
    __syncthreads();
    // hidden layer 1: (row, k)
    for (int idx = tid; idx < kTile * kPropHid; idx += blockDim.x) {
      const int r = idx / kPropHid, k = idx % kPropHid;
      float z = b1[k];
#pragma unroll
      for (int f = 0; f < kPropIn; ++f) z += sPhi[r][f] * W1[f * kPropHid + k];
      sH1[r][k] = tanhf(z);
    }
    __syncthreads();
    for (int idx = tid; idx < kTile * kPropHid; idx += blockDim.x) {
      const int r = idx / kPropHid, k = idx % kPropHid;
      float z = b2[k];
#pragma unroll 8
      for (int mm = 0; mm < kPropHid; ++mm) z += sH1[r][mm] * W2[mm * kPropHid + k];
      sH2[r][k] = tanhf(z);
    }
    __syncthreads();
    // logits: one warp per row group
    {
      const int warp = tid >> 5, lane = tid & 31;
      for (int r = warp; r < kTile; r += blockDim.x >> 5) {
        float z = sH2[r][lane] * w3[lane] + sH2[r][lane + 32] * w3[lane + 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        z += sP[kPropOb3];
        if (lane == 0) {
          const int64_t row = r0 + r;
          if (a.mode == 0) {
            if (row < rows) a.logits[row] = sMask[r] > 0.f ? z : __int_as_float(0x7fc00000);
          } else {
            const float res = sMask[r] * (z - sDl[r]);
            sDl[r] = 2.f * res;             // d (res^2) / d logit
            sH1[r][kPropHid] = res * res;   // padding column: the row's squared residual
          }
        }
      }
    }
    __syncthreads();
    if (a.mode == 0) continue;
    if (tid == 0) {
      for (int r = 0; r < kTile; ++r) {
        loss += sH1[r][kPropHid];
        count += sMask[r];
      }
    }
    // dZ2 = dlogit w3 (1 - H2^2)
    for (int idx = tid; idx < kTile * kPropHid; idx += blockDim.x) {
      const int r = idx / kPropHid, k = idx % kPropHid;
      const float h = sH2[r][k];
      sD[r][k] = sDl[r] * w3[k] * (1.f - h * h);
    }
    __syncthreads();
    // gradient sums of W2, b2, w3, b3 over the tile (owned entries)
#pragma unroll
    for (int kk = 0; kk < kOwn; ++kk) {
      const int p = tid + kk * kPropThreads;
      if (p >= kPropOW2 && p < kPropOW2 + kPropHid * kPropHid) {
        const int mm = (p - kPropOW2) / kPropHid, k = (p - kPropOW2) % kPropHid;
        float s = 0.f;
        for (int r = 0; r < kTile; ++r) s += sH1[r][mm] * sD[r][k];
        acc[kk] += s;
      } else if (p >= kPropOb2 && p < kPropOb2 + kPropHid) {
        const int k = p - kPropOb2;
        float s = 0.f;
        for (int r = 0; r < kTile; ++r) s += sD[r][k];
        acc[kk] += s;
      } else if (p >= kPropOw3 && p < kPropOw3 + kPropHid) {
        const int k = p - kPropOw3;
        float s = 0.f;
        for (int r = 0; r < kTile; ++r) s += sDl[r] * sH2[r][k];
        acc[kk] += s;
      } else if (p == kPropOb3) {
        float s = 0.f;
        for (int r = 0; r < kTile; ++r) s += sDl[r];
        acc[kk] += s;
      }
    }
    __syncthreads();
    // dZ1 = (dZ2 W2^T) (1 - H1^2), written over sH2 (no longer needed)
    for (int idx = tid; idx < kTile * kPropHid; idx += blockDim.x) {
      const int r = idx / kPropHid, mm = idx % kPropHid;
      float s = 0.f;
#pragma unroll 8
      for (int k = 0; k < kPropHid; ++k) s += sD[r][k] * W2[mm * kPropHid + k];
      const float h = sH1[r][mm];
      sH2[r][mm] = s * (1.f - h * h);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kOwn; ++kk) {
      const int p = tid + kk * kPropThreads;
      if (p < kPropOW1 + kPropIn * kPropHid) {
        const int f = p / kPropHid, k = p % kPropHid;
        float s = 0.f;
        for (int r = 0; r < kTile; ++r) s += sPhi[r][f] * sH2[r][k];
        acc[kk] += s;
      } else if (p >= kPropOb1 && p < kPropOb1 + kPropHid) {
        const int k = p - kPropOb1;
        float s = 0.f;
        for (int r = 0; r < kTile; ++r) s += sH2[r][k];
        acc[kk] += s;
      }
    }
    __syncthreads();
  }
  if (a.mode == 1) {
    double* out = a.partial + (size_t)blockIdx.x * (kPropParams + 2);
#pragma unroll
    for (int kk = 0; kk < kOwn; ++kk) {
      const int p = tid + kk * kPropThreads;
      if (p < kPropParams) out[p] = (double)acc[kk];
    }
    if (tid == 0) {
      out[kPropParams] = (double)loss;
      out[kPropParams + 1] = (double)count;
    }
  }
}

// grad = (sum over CTAs of the partials) / count; loss likewise.  Fixed order, float64.
__global__ void k_prop_reduce(const double* partial, int grid, double* grad, double* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kPropParams) return;
  double s = 0.0, n = 0.0;
  for (int c = 0; c < grid; ++c) {
    s += partial[(size_t)c * (kPropParams + 2) + p];
    n += partial[(size_t)c * (kPropParams + 2) + kPropParams + 1];
  }
  const double inv = n > 0.0 ? 1.0 / n : 0.0;
  if (p < kPropParams)
    grad[p] = s * inv;
  else if (loss)
    *loss = s * inv;
}

// Adam (Kingma & Ba 2015), step t >= 1.
__global__ void k_adam(float* params, float* m, float* v, const double* grad, int P, int t, double lr, double b1,
                       double b2, double eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double g = grad[p];
  const double mm = b1 * (double)m[p] + (1.0 - b1) * g;
  const double vv = b2 * (double)v[p] + (1.0 - b2) * g * g;
  m[p] = (float)mm;
  v[p] = (float)vv;
  const double mh = mm / (1.0 - pow(b1, (double)t));
  const double vh = vv / (1.0 - pow(b2, (double)t));
  params[p] = (float)((double)params[p] - lr * mh / (sqrt(vh) + eps));
}

static int prop_grid(int64_t B, int E) {
  DeviceInfo di;
  if (device_info(&di) != GNA_OK) return 1;
  const int64_t tiles = (B * (int64_t)E * 2 + kTile - 1) / kTile;
  int64_t grid = (int64_t)di.sms * 4;
  if (grid > tiles) grid = tiles;
  return grid < 1 ? 1 : (int)grid;
}

size_t prop_workspace(const gna_graph* g, int64_t B) {
  return align_up((size_t)prop_grid(B, g->d.E) * (kPropParams + 2) * sizeof(double));
}

gna_status prop_grad_launch(const gna_graph* g, const int8_t* spins, const float* dlogpsi, int64_t B,
                            const float* params, double* grad, double* loss, void* ws, cudaStream_t st) {
  PropArgs a;
  a.g = g->d;
  a.spins = spins;
  a.dlogpsi = dlogpsi;
  a.params = params;
  a.B = B;
  a.mode = 1;
  a.logits = nullptr;
  a.partial = (double*)ws;
  const int grid = prop_grid(B, g->d.E);
  const int smem = kPropSmemFloats * (int)sizeof(float);
  GNA_CUDA_TRY(cudaFuncSetAttribute((const void*)k_prop, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k_prop<<<grid, kPropThreads, smem, st>>>(a);
  GNA_CUDA_TRY(cudaGetLastError());
  k_prop_reduce<<<(kPropParams + 1 + 255) / 256, 256, 0, st>>>(a.partial, grid, grad, loss);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

gna_status prop_logits_launch(const gna_graph* g, const int8_t* spins, int64_t B, const float* params, float* logits,
                              cudaStream_t st) {
  PropArgs a;
  a.g = g->d;
  a.spins = spins;
  a.dlogpsi = nullptr;
  a.params = params;
  a.B = B;
  a.mode = 0;
  a.logits = logits;
  a.partial = nullptr;
  const int smem = kPropSmemFloats * (int)sizeof(float);
  GNA_CUDA_TRY(cudaFuncSetAttribute((const void*)k_prop, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  k_prop<<<prop_grid(B, g->d.E), kPropThreads, smem, st>>>(a);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

gna_status prop_adam_launch(float* params, float* m, float* v, const double* grad, int t, double lr,
                            cudaStream_t st) {
  k_adam<<<(kPropParams + 255) / 256, 256, 0, st>>>(params, m, v, grad, kPropParams, t, lr, 0.9, 0.999, 1e-8);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

}  // namespace gna

// ISGO importance weights and statistics (Eq. isgo of arXiv:2011.12453, read as the
// covariance gradient), the plain gradient step, and the device Philox used by the
// sampler exposed for bit-exact checks.  All reductions are float64 in a fixed order.
#include <cmath>

#include "common.cuh"

namespace gna {

static __device__ int s_isgo_status;

constexpr int kRedThreads = 256;

// Fixed-order block tree reduction of one double per thread (result in thread 0).
template <bool MAX>
__device__ double block_reduce(double v, double* sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = MAX ? fmax(sm[threadIdx.x], sm[threadIdx.x + s]) : sm[threadIdx.x] + sm[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

__device__ inline double log_weight(const double* lp, const double* lp0, const double* counts, int64_t x) {
  double lw = 2.0 * (lp[2 * x] - lp0[2 * x]);
  if (counts) lw += log(counts[x]);
  return lw;
}

// pass 1: per block (m_b, sum exp(lw - m_b), sum exp(lw - m_b) E)
__global__ void __launch_bounds__(kRedThreads) k_isgo_pass1(const double* lp, const double* lp0, const double* counts,
                                                            const double* E, int64_t B, double* part) {
  __shared__ double sm[kRedThreads];
  double m = -INFINITY;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < B; x += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, log_weight(lp, lp0, counts, x));
  m = block_reduce<true>(m, sm);
  double s = 0.0, sr = 0.0, si = 0.0;
  if (m > -INFINITY) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < B; x += (int64_t)gridDim.x * blockDim.x) {
      const double w = exp(log_weight(lp, lp0, counts, x) - m);
      s += w;
      sr += w * E[2 * x];
      si += w * E[2 * x + 1];
    }
  }
  s = block_reduce<false>(s, sm);
  sr = block_reduce<false>(sr, sm);
  si = block_reduce<false>(si, sm);
  if (threadIdx.x == 0) {
    part[4 * blockIdx.x + 0] = m;
    part[4 * blockIdx.x + 1] = s;
    part[4 * blockIdx.x + 2] = sr;
    part[4 * blockIdx.x + 3] = si;
  }
}

// combine: g = (m, S, Re Ebar, Im Ebar), or with raw = 1 the shard's (m, S, S Re Ebar, S Im Ebar)
__global__ void __launch_bounds__(kRedThreads) k_isgo_combine1(const double* part, int nb, double* gsum, int raw) {
  __shared__ double sm[kRedThreads];
  double m = -INFINITY;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fmax(m, part[4 * b]);
  m = block_reduce<true>(m, sm);
  double s = 0.0, sr = 0.0, si = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double mb = part[4 * b];
    const double f = mb > -INFINITY ? exp(mb - m) : 0.0;
    s += f * part[4 * b + 1];
    sr += f * part[4 * b + 2];
    si += f * part[4 * b + 3];
  }
  s = block_reduce<false>(s, sm);
  sr = block_reduce<false>(sr, sm);
  si = block_reduce<false>(si, sm);
  if (threadIdx.x == 0) {
    gsum[0] = m;
    gsum[1] = s;
    gsum[2] = raw ? sr : sr / s;
    gsum[3] = raw ? si : si / s;
  }
}

// pass 2: p, cotangents, per block sum p |E - Ebar|^2 and sum p^2 / c
__global__ void __launch_bounds__(kRedThreads) k_isgo_pass2(const double* lp, const double* lp0, const double* counts,
                                                            const double* E, int64_t B, const double* gsum,
                                                            double* cot, double* part2) {
  __shared__ double sm[kRedThreads];
  const double m = gsum[0], S = gsum[1], er = gsum[2], ei = gsum[3];
  double v = 0.0, q = 0.0, n = 0.0;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < B; x += (int64_t)gridDim.x * blockDim.x) {
    const double p = exp(log_weight(lp, lp0, counts, x) - m) / S;
    const double dr = E[2 * x] - er, di = E[2 * x + 1] - ei;
    v += p * (dr * dr + di * di);
    q += p * p / (counts ? counts[x] : 1.0);
    n += counts ? counts[x] : 1.0;
    if (cot) {
      cot[2 * x] = 2.0 * p * dr;
      cot[2 * x + 1] = 2.0 * p * di;
    }
  }
  v = block_reduce<false>(v, sm);
  q = block_reduce<false>(q, sm);
  n = block_reduce<false>(n, sm);
  if (threadIdx.x == 0) {
    part2[3 * blockIdx.x] = v;
    part2[3 * blockIdx.x + 1] = q;
    part2[3 * blockIdx.x + 2] = n;
  }
}

// stats = (Re Ebar, Im Ebar, var, ess), or with raw != NULL the shard's sums (var, q, n) only
__global__ void __launch_bounds__(kRedThreads) k_isgo_combine2(const double* part2, int nb, const double* gsum,
                                                               double* stats, double* raw) {
  __shared__ double sm[kRedThreads];
  double v = 0.0, q = 0.0, n = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    v += part2[3 * b];
    q += part2[3 * b + 1];
    n += part2[3 * b + 2];
  }
  v = block_reduce<false>(v, sm);
  q = block_reduce<false>(q, sm);
  n = block_reduce<false>(n, sm);
  if (threadIdx.x == 0 && raw) {
    raw[0] = v;
    raw[1] = q;
    raw[2] = n;
  } else if (threadIdx.x == 0) {
    stats[0] = gsum[2];
    stats[1] = gsum[3];
    stats[2] = v;
    stats[3] = 1.0 / q;
    if (!isfinite(gsum[2]) || !isfinite(gsum[3]) || !isfinite(v) || !isfinite(q)) atomicOr(&s_isgo_status, 2);
    // degenerate reweighting (the failure the paper warns of: a few samples carry the
    // weights and the gradient is dominated by them): IS-ESS below 1% of the copies
    else if (1.0 / q < 0.01 * n) atomicOr(&s_isgo_status, 4);
  }
}

static int isgo_blocks(int64_t B) {
  int64_t nb = (B + 4 * kRedThreads - 1) / (4 * kRedThreads);
  if (nb < 1) nb = 1;
  if (nb > 1024) nb = 1024;
  return (int)nb;
}

size_t isgo_weights_ws(int64_t B) {
  const int nb = isgo_blocks(B);
  return align_up((size_t)nb * 4 * 8) + align_up((size_t)nb * 3 * 8) + align_up(4 * 8);
}

gna_status isgo_weights_launch(const double* lp, const double* lp0, const double* E, const double* counts, int64_t B,
                               double* cot, double* stats, void* ws, cudaStream_t st) {
  const int nb = isgo_blocks(B);
  unsigned char* w = (unsigned char*)ws;
  double* part = (double*)w;
  w += align_up((size_t)nb * 4 * 8);
  double* part2 = (double*)w;
  w += align_up((size_t)nb * 3 * 8);
  double* gsum = (double*)w;
  k_isgo_pass1<<<nb, kRedThreads, 0, st>>>(lp, lp0, counts, E, B, part);
  k_isgo_combine1<<<1, kRedThreads, 0, st>>>(part, nb, gsum, 0);
  k_isgo_pass2<<<nb, kRedThreads, 0, st>>>(lp, lp0, counts, E, B, gsum, cot, part2);
  k_isgo_combine2<<<1, kRedThreads, 0, st>>>(part2, nb, gsum, stats, nullptr);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

// Sample-sharded form: the shard's (m, S, S Re Ebar, S Im Ebar) ...
gna_status isgo_partials_launch(const double* lp, const double* lp0, const double* E, const double* counts, int64_t B,
                                double* part4, void* ws, cudaStream_t st) {
  const int nb = isgo_blocks(B);
  double* part = (double*)ws;
  k_isgo_pass1<<<nb, kRedThreads, 0, st>>>(lp, lp0, counts, E, B, part);
  k_isgo_combine1<<<1, kRedThreads, 0, st>>>(part, nb, part4, 1);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

// ... and, given the global (m, S, Re Ebar, Im Ebar), the shard's cotangents and (var, q, n) sums.
gna_status isgo_finish_launch(const double* lp, const double* lp0, const double* E, const double* counts, int64_t B,
                              const double* global4, double* cot, double* part3, void* ws, cudaStream_t st) {
  const int nb = isgo_blocks(B);
  double* part2 = (double*)ws;
  k_isgo_pass2<<<nb, kRedThreads, 0, st>>>(lp, lp0, counts, E, B, global4, cot, part2);
  k_isgo_combine2<<<1, kRedThreads, 0, st>>>(part2, nb, global4, nullptr, part3);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

template <typename T>
__global__ void k_sgd(T* theta, const double* grad, double lr, int P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) theta[p] = (T)((double)theta[p] - lr * grad[p]);
}

gna_status sgd_launch(int prec, void* theta, const double* grad, double lr, int P, cudaStream_t st) {
  if (prec == GNA_PREC_FP64)
    k_sgd<double><<<(P + 255) / 256, 256, 0, st>>>((double*)theta, grad, lr, P);
  else
    k_sgd<float><<<(P + 255) / 256, 256, 0, st>>>((float*)theta, grad, lr, P);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

__global__ void k_philox(const uint64_t* keys, const uint64_t* ctrs, int64_t n, uint64_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U64x4 r = philox4x64_10(keys[2 * i], keys[2 * i + 1], U64x4{ctrs[4 * i], ctrs[4 * i + 1], ctrs[4 * i + 2], ctrs[4 * i + 3]});
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

gna_status philox_launch(const uint64_t* keys, const uint64_t* ctrs, int64_t n, uint64_t* out, cudaStream_t st) {
  if (n == 0) return GNA_OK;
  k_philox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, ctrs, n, out);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

gna_status isgo_read_status(int* flags, int clear) {
  int v = 0;
  GNA_CUDA_TRY(cudaMemcpyFromSymbol(&v, s_isgo_status, sizeof(int)));
  *flags |= v;
  if (clear) {
    int z = 0;
    GNA_CUDA_TRY(cudaMemcpyToSymbol(s_isgo_status, &z, sizeof(int)));
  }
  return GNA_OK;
}

}  // namespace gna

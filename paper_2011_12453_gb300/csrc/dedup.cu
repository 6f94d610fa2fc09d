// Grouping of duplicated samples into unique states with counts (scaling section of
// arXiv:2011.12453: the sampler's states are grouped before the workers weight them;
// Eq. isgo then carries log count_x).
//
// HBM-bound, five short kernels:
//   1. pack: one warp per sample turns its +-1 bytes into bits with __ballot_sync
//      (W = ceil(N/64) words per sample, coalesced 32-byte reads);
//   2. insert: one thread per sample probes an open-addressing table of 2^k >= 2B slots
//      (hash of the packed words, linear probing, compare-and-swap of index + 1) and, on a
//      slot holding an equal state, lowers it to the smaller sample index (atomicMin) --
//      after the kernel every state's slot holds its first occurrence;
//   3. resolve: each sample finds its slot again, adds one to its representative's count
//      and flags itself when it is the representative;
//   4. scan: exclusive prefix sum of the flags (per-block scans, then the block totals);
//   5. gather: representatives write their state, log Psi^0 and count at their rank.
// Output order = first occurrence, counts exact; the result does not depend on the
// interleaving of the atomics.
#include <cstdint>

#include "common.cuh"

namespace gna {

namespace {

constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  // splitmix64 finaliser
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_pack(const int8_t* spins, int64_t B, int N, int Wd, uint64_t* words) {
  const int lane = threadIdx.x & 31;
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= B) return;
  const int8_t* s = spins + b * N;
  for (int w = 0; w < Wd; ++w) {
    const int v0 = 64 * w + lane, v1 = v0 + 32;
    const unsigned lo = __ballot_sync(0xffffffffu, v0 < N && s[v0 < N ? v0 : 0] > 0);
    const unsigned hi = __ballot_sync(0xffffffffu, v1 < N && s[v1 < N ? v1 : 0] > 0);
    if (lane == 0) words[b * Wd + w] = (uint64_t)lo | ((uint64_t)hi << 32);
  }
}

__device__ __forceinline__ uint64_t hash_words(const uint64_t* w, int Wd) {
  uint64_t h = 0x9e3779b97f4a7c15ull;
  for (int i = 0; i < Wd; ++i) h = mix64(h ^ w[i]);
  return h;
}

__device__ __forceinline__ bool same(const uint64_t* a, const uint64_t* b, int Wd) {
  for (int i = 0; i < Wd; ++i)
    if (a[i] != b[i]) return false;
  return true;
}

__global__ void k_insert(const uint64_t* words, int64_t B, int Wd, int* table, uint64_t mask) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const uint64_t* mine = words + b * Wd;
  uint64_t slot = hash_words(mine, Wd) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    int cur = atomicCAS(table + slot, 0, (int)b + 1);
    if (cur == 0) return;  // a new state (its slot may later be lowered to an earlier copy)
    if (same(words + (int64_t)(cur - 1) * Wd, mine, Wd)) {
      atomicMin(table + slot, (int)b + 1);
      return;
    }
    slot = (slot + 1) & mask;
  }
}

__global__ void k_resolve(const uint64_t* words, int64_t B, int Wd, const int* table, uint64_t mask, int* rep,
                          int* cnt, int* flag) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const uint64_t* mine = words + b * Wd;
  uint64_t slot = hash_words(mine, Wd) & mask;
  int r = (int)b;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const int cur = table[slot];
    if (cur != 0 && same(words + (int64_t)(cur - 1) * Wd, mine, Wd)) {
      r = cur - 1;
      break;
    }
    slot = (slot + 1) & mask;
  }
  rep[b] = r;
  atomicAdd(cnt + r, 1);
  flag[b] = r == (int)b ? 1 : 0;
}

// exclusive scan of flag within blocks of kScanThreads; block totals to tot
__global__ void k_scan_blocks(const int* flag, int64_t B, int* pos, int* tot) {
  __shared__ int sh[kScanThreads];
  const int64_t i = (int64_t)blockIdx.x * kScanThreads + threadIdx.x;
  const int v = i < B ? flag[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < B) pos[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == kScanThreads - 1) tot[blockIdx.x] = sh[threadIdx.x];
}

// exclusive scan of the block totals in place (one block, sequential chunks); the grand
// total to *n_unique
__global__ void k_scan_totals(int* tot, int nblocks, int64_t* n_unique) {
  __shared__ int sh[kScanThreads];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const int v = i < nblocks ? tot[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
      const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nblocks) tot[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry += sh[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_unique = carry;
}

__global__ void k_gather(const int8_t* spins, const double* logpsi, int64_t B, int N, const int* flag,
                         const int* pos, const int* tot, const int* cnt, int8_t* us, double* ul, double* uc) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !flag[b]) return;
  const int64_t o = tot[b / kScanThreads] + pos[b];
  for (int v = 0; v < N; ++v) us[o * N + v] = spins[b * N + v];
  if (logpsi) {
    ul[2 * o] = logpsi[2 * b];
    ul[2 * o + 1] = logpsi[2 * b + 1];
  }
  uc[o] = (double)cnt[b];
}

struct DedupWs {
  uint64_t* words;
  int *table, *rep, *cnt, *flag, *pos, *tot;
  uint64_t cap;
  size_t bytes;
};

DedupWs dedup_carve(int64_t B, int N, unsigned char* base) {
  DedupWs w{};
  const int Wd = (N + 63) / 64;
  uint64_t cap = 1;
  while (cap < (uint64_t)(2 * B)) cap <<= 1;
  w.cap = cap;
  const int64_t nblk = (B + kScanThreads - 1) / kScanThreads;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    o = (o + 255) / 256 * 256;
    size_t r = o;
    o += bytes;
    return base ? base + r : nullptr;
  };
  w.words = (uint64_t*)take((size_t)B * Wd * 8);
  w.table = (int*)take(cap * 4);
  w.rep = (int*)take((size_t)B * 4);
  w.cnt = (int*)take((size_t)B * 4);
  w.flag = (int*)take((size_t)B * 4);
  w.pos = (int*)take((size_t)B * 4);
  w.tot = (int*)take((size_t)(nblk > 0 ? nblk : 1) * 4);
  w.bytes = (o + 255) / 256 * 256;
  return w;
}

}  // namespace

size_t dedup_workspace(int64_t B, int N) { return B > 0 ? dedup_carve(B, N, nullptr).bytes : 0; }

gna_status dedup_run(int N, const int8_t* spins, const double* logpsi, int64_t B, int8_t* us, double* ul, double* uc,
                     int64_t* n_unique, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (B == 0) {
    GNA_CUDA_TRY(cudaMemsetAsync(n_unique, 0, sizeof(int64_t), st));
    return GNA_OK;
  }
  const DedupWs w = dedup_carve(B, N, (unsigned char*)ws);
  if (ws_bytes < w.bytes || !ws) return GNA_ERR_WORKSPACE;
  const int Wd = (N + 63) / 64;
  GNA_CUDA_TRY(cudaMemsetAsync(w.table, 0, w.cap * 4, st));
  GNA_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, (size_t)B * 4, st));
  const int64_t nblk = (B + kScanThreads - 1) / kScanThreads;
  const int t = 256;
  const int64_t g1 = (B * 32 + t - 1) / t, g2 = (B + t - 1) / t;
  k_pack<<<(unsigned)g1, t, 0, st>>>(spins, B, N, Wd, w.words);
  k_insert<<<(unsigned)g2, t, 0, st>>>(w.words, B, Wd, w.table, w.cap - 1);
  k_resolve<<<(unsigned)g2, t, 0, st>>>(w.words, B, Wd, w.table, w.cap - 1, w.rep, w.cnt, w.flag);
  k_scan_blocks<<<(unsigned)nblk, kScanThreads, 0, st>>>(w.flag, B, w.pos, w.tot);
  k_scan_totals<<<1, kScanThreads, 0, st>>>(w.tot, (int)nblk, n_unique);
  k_gather<<<(unsigned)g2, t, 0, st>>>(spins, logpsi, B, N, w.flag, w.pos, w.tot, w.cnt, us, ul, uc);
  GNA_CUDA_TRY(cudaGetLastError());
  return GNA_OK;
}

}  // namespace gna

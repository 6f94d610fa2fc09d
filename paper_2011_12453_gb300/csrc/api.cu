// C ABI entry points of libgna.so: argument validation, workspace carving and dispatch
// to the kernels.  Every check here runs on the host before anything is enqueued.
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "metro.cuh"
#include "prop.cuh"
#include "tc.cuh"

namespace gna {

static thread_local cudaError_t t_last_cuda_error = cudaSuccess;
void set_last_cuda_error(cudaError_t e) { t_last_cuda_error = e; }

gna_status device_info(DeviceInfo* out) {
  static std::mutex mu;
  static DeviceInfo cache[64];
  static bool have[64] = {false};
  int dev = 0;
  GNA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return GNA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (!have[dev]) {
    DeviceInfo di;
    GNA_CUDA_TRY(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev));
    GNA_CUDA_TRY(cudaDeviceGetAttribute(&di.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int major = 0, minor = 0;
    GNA_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    GNA_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    di.cc = major * 10 + minor;
    cache[dev] = di;
    have[dev] = true;
  }
  *out = cache[dev];
  return GNA_OK;
}

// Descriptors whose GEMMs run on the tensor cores: BF16 and BF16X2 (split operands).
static bool tensor_prec(const gna_model_desc* d) { return d->prec == GNA_PREC_BF16 || d->prec == GNA_PREC_BF16X2; }
static int split_prec(const gna_model_desc* d) { return d->prec == GNA_PREC_BF16X2 ? 1 : 0; }

static bool desc_ok(const gna_model_desc* d) {
  if (!d) return false;
  if (d->F < 1 || d->F > kMaxF) return false;
  if (d->L < 0 || d->L > kMaxL) return false;
  if (d->act != GNA_ACT_TANH && d->act != GNA_ACT_RELU_LN) return false;
  if (d->prec < GNA_PREC_FP64 || d->prec > GNA_PREC_BF16X2) return false;
  if (d->shared_weights != 0 && d->shared_weights != 1) return false;
  if (tensor_prec(d) && d->F % 16 != 0) return false;
  return true;
}

static gna_status check_gd(const gna_graph* g, const gna_model_desc* d) {
  if (!g || !desc_ok(d)) return GNA_ERR_INVALID_ARG;
  // ReLU + layer norm runs on the float64 / float32 SIMT kernels only
  if (d->act == GNA_ACT_RELU_LN && tensor_prec(d)) return GNA_ERR_UNSUPPORTED;
  if (d->L > g->d.Lmax) return GNA_ERR_INVALID_ARG;
  int dev = 0;
  GNA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != g->device) return GNA_ERR_INVALID_ARG;
  return GNA_OK;
}

// Arithmetic of the SIMT kernels for a descriptor: BF16 / BF16X2 descriptors run their
// non-tensor-core steps in float32.
static int simt_prec(const gna_model_desc* d) { return d->prec == GNA_PREC_FP64 ? GNA_PREC_FP64 : GNA_PREC_FP32; }

static gna_status op_workspace(const gna_graph* g, const gna_model_desc* d, int op, int64_t B, size_t* bytes);

}  // namespace gna

using namespace gna;

extern "C" int32_t gna_version(void) { return 1; }

extern "C" const char* gna_status_string(gna_status s) {
  switch (s) {
    case GNA_OK:
      return "ok";
    case GNA_ERR_INVALID_ARG:
      return "invalid argument";
    case GNA_ERR_CUDA:
      return cudaGetErrorString(t_last_cuda_error);
    case GNA_ERR_TIMEOUT:
      return "a bounded device-side wait timed out";
    case GNA_ERR_NONFINITE:
      return "non-finite value";
    case GNA_ERR_WORKSPACE:
      return "workspace too small";
    case GNA_ERR_UNSUPPORTED:
      return "unsupported by the library";
    case GNA_WARN_DEGENERATE_WEIGHTS:
      return "degenerate importance weights";
  }
  return "unknown status";
}

extern "C" gna_status gna_model_desc_init(gna_model_desc* d, int32_t F, int32_t L, int32_t act, int32_t prec,
                                          int32_t shared_weights) {
  if (!d) return GNA_ERR_INVALID_ARG;
  gna_model_desc t{F, L, act, prec, shared_weights};
  if (!desc_ok(&t)) return GNA_ERR_INVALID_ARG;
  *d = t;
  return GNA_OK;
}

extern "C" int64_t gna_num_params(const gna_model_desc* d) {
  if (!desc_ok(d)) return -1;
  const int64_t F = d->F;
  const int64_t nl = d->shared_weights ? 1 : d->L;
  return 3 * F + nl * (2 * F * F + F) + (F + 2) * 2 + 2;
}

namespace gna {

static gna_status op_workspace(const gna_graph* g, const gna_model_desc* d, int op, int64_t B, size_t* bytes) {
  const Dims m = make_dims(g, d);
  const int sp = simt_prec(d);
  switch (op) {
    case GNA_OP_FORWARD:
      if (tensor_prec(d)) return tc_workspace(g, m, TC_FWD, B, bytes, split_prec(d));
      return simt_workspace(g, m, sp, 0, B, bytes);
    case GNA_OP_LOCAL_ENERGY_FULL:
      return simt_workspace(g, m, sp, 1, B, bytes);
    case GNA_OP_LOCAL_ENERGY_INCREMENTAL:
      if (tensor_prec(d)) return tc_workspace(g, m, TC_ELOC, B, bytes, split_prec(d));
      return simt_workspace(g, m, sp, 2, B, bytes);
    case GNA_OP_LOCAL_ENERGY_LOGPSI: {
      // the local-energy call (its own forward gives log Psi), or the two calls in turn
      if (tensor_prec(d)) return tc_workspace(g, m, TC_ELOC, B, bytes, split_prec(d));
      size_t a = 0, b = 0;
      gna_status st = simt_workspace(g, m, sp, 0, B, &a);
      if (st != GNA_OK) return st;
      st = simt_workspace(g, m, sp, 2, B, &b);
      if (st != GNA_OK) return st;
      *bytes = a > b ? a : b;
      return GNA_OK;
    }
    case GNA_OP_METROPOLIS: {
      if (tensor_prec(d)) {
        gna_status st = tcm_workspace(g, m, B, bytes);
        if (st != GNA_ERR_UNSUPPORTED) return st;
      }
      // the warp sampler propagates tanh differences; ReLU + layer norm takes one chain per CTA
      if (d->act == GNA_ACT_TANH) {
        gna_status st = metro_workspace(g, m, sp, B, 0, bytes);
        if (st != GNA_ERR_UNSUPPORTED) return st;
      }
      return simt_workspace(g, m, sp, 3, B, bytes);
    }
    case GNA_OP_METROPOLIS_LEARNED: {
      if (g->max_deg > 16) return GNA_ERR_UNSUPPORTED;
      if (d->act == GNA_ACT_TANH) {
        gna_status st = metro_workspace(g, m, sp, B, 1, bytes);
        if (st != GNA_ERR_UNSUPPORTED) return st;
      }
      return simt_workspace(g, m, sp, 5, B, bytes);
    }
    case GNA_OP_BACKWARD:
      if (tensor_prec(d)) {
        gna_status st = tcb_workspace(g, m, B, bytes);
        if (st != GNA_ERR_UNSUPPORTED) return st;
      }
      return simt_workspace(g, m, sp, 4, B, bytes);
    case GNA_OP_ISGO_WEIGHTS:
      *bytes = isgo_weights_ws(B);
      return GNA_OK;
    case GNA_OP_ISGO_GRAD: {
      size_t a = 0, b = 0, c = 0;
      gna_status st = op_workspace(g, d, GNA_OP_FORWARD, B, &a);
      if (st != GNA_OK) return st;
      st = op_workspace(g, d, GNA_OP_LOCAL_ENERGY_LOGPSI, B, &b);
      if (st != GNA_OK) return st;
      st = op_workspace(g, d, GNA_OP_BACKWARD, B, &c);
      if (st != GNA_OK) return st;
      size_t inner = a > b ? a : b;
      inner = inner > c ? inner : c;
      inner = inner > isgo_weights_ws(B) ? inner : isgo_weights_ws(B);
      *bytes = 3 * align_up((size_t)B * 2 * sizeof(double)) + inner;
      return GNA_OK;
    }
  }
  return GNA_ERR_INVALID_ARG;
}

static gna_status check_ws(const gna_graph* g, const gna_model_desc* d, int op, int64_t B, void* ws, size_t bytes) {
  size_t need = 0;
  gna_status st = op_workspace(g, d, op, B, &need);
  if (st != GNA_OK) return st;
  if (bytes < need || (need > 0 && ws == nullptr)) return GNA_ERR_WORKSPACE;
  return GNA_OK;
}

}  // namespace gna

extern "C" gna_status gna_workspace_size(const gna_graph* g, const gna_model_desc* d, int32_t op, int64_t B,
                                         size_t* bytes) {
  gna_status st = check_gd(g, d);
  if (st != GNA_OK) return st;
  if (!bytes || B < 0) return GNA_ERR_INVALID_ARG;
  return op_workspace(g, d, op, B, bytes);
}

extern "C" gna_status gna_forward(const gna_graph* g, const gna_model_desc* d, const void* theta,
                                  const int8_t* spins, int64_t B, double* logpsi, void* workspace,
                                  size_t workspace_bytes, void* stream) {
  gna_status st = check_gd(g, d);
  if (st != GNA_OK) return st;
  if (B < 0 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (B == 0) return GNA_OK;
  if (!theta || !spins || !logpsi) return GNA_ERR_INVALID_ARG;
  st = check_ws(g, d, GNA_OP_FORWARD, B, workspace, workspace_bytes);
  if (st != GNA_OK) return st;
  const Dims m = make_dims(g, d);
  if (tensor_prec(d)) {
    TcCall tc{g, m, TC_FWD, (const float*)theta, spins, B, logpsi, nullptr, nullptr, split_prec(d)};
    return tc_run(tc, workspace, workspace_bytes, (cudaStream_t)stream);
  }
  SimtCall sc{};
  sc.g = g;
  sc.m = m;
  sc.op = 0;
  sc.theta = theta;
  sc.spins = spins;
  sc.B = B;
  sc.logpsi = logpsi;
  return simt_run(sc, simt_prec(d), workspace, workspace_bytes, (cudaStream_t)stream);
}

extern "C" gna_status gna_local_energy(const gna_graph* g, const gna_model_desc* d, const void* theta,
                                       const int8_t* spins, int64_t B, int32_t mode, double* eloc,
                                       float* dlogpsi_bonds, void* workspace, size_t workspace_bytes,
                                       void* stream) {
  gna_status st = check_gd(g, d);
  if (st != GNA_OK) return st;
  if (B < 0 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (mode != GNA_ELOC_FULL && mode != GNA_ELOC_INCREMENTAL) return GNA_ERR_INVALID_ARG;
  if (B == 0) return GNA_OK;
  if (!theta || !spins || !eloc) return GNA_ERR_INVALID_ARG;
  const int op = mode == GNA_ELOC_FULL ? GNA_OP_LOCAL_ENERGY_FULL : GNA_OP_LOCAL_ENERGY_INCREMENTAL;
  st = check_ws(g, d, op, B, workspace, workspace_bytes);
  if (st != GNA_OK) return st;
  const Dims m = make_dims(g, d);
  if (tensor_prec(d) && mode == GNA_ELOC_INCREMENTAL) {
    TcCall tc{g, m, TC_ELOC, (const float*)theta, spins, B, nullptr, eloc, dlogpsi_bonds, split_prec(d)};
    return tc_run(tc, workspace, workspace_bytes, (cudaStream_t)stream);
  }
  SimtCall sc{};
  sc.g = g;
  sc.m = m;
  sc.op = mode == GNA_ELOC_FULL ? 1 : 2;
  sc.theta = theta;
  sc.spins = spins;
  sc.B = B;
  sc.eloc = eloc;
  sc.dlogpsi = dlogpsi_bonds;
  return simt_run(sc, simt_prec(d), workspace, workspace_bytes, (cudaStream_t)stream);
}

extern "C" gna_status gna_local_energy_logpsi(const gna_graph* g, const gna_model_desc* d, const void* theta,
                                              const int8_t* spins, int64_t B, double* eloc, double* logpsi,
                                              void* workspace, size_t workspace_bytes, void* stream) {
  gna_status st = check_gd(g, d);
  if (st != GNA_OK) return st;
  if (B < 0 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (B == 0) return GNA_OK;
  if (!theta || !spins || !eloc || !logpsi) return GNA_ERR_INVALID_ARG;
  st = check_ws(g, d, GNA_OP_LOCAL_ENERGY_LOGPSI, B, workspace, workspace_bytes);
  if (st != GNA_OK) return st;
  if (tensor_prec(d)) {
    TcCall tc{g, make_dims(g, d), TC_ELOC, (const float*)theta, spins, B, logpsi, eloc, nullptr, split_prec(d)};
    return tc_run(tc, workspace, workspace_bytes, (cudaStream_t)stream);
  }
  st = gna_forward(g, d, theta, spins, B, logpsi, workspace, workspace_bytes, stream);
  if (st != GNA_OK) return st;
  return gna_local_energy(g, d, theta, spins, B, GNA_ELOC_INCREMENTAL, eloc, nullptr, workspace, workspace_bytes,
                          stream);
}

extern "C" gna_status gna_metropolis_sweep(const gna_graph* g, const gna_model_desc* d, const void* theta,
                                           int8_t* chain_spins, int64_t C, int32_t n_sweeps, int32_t record_every,
                                           uint64_t seed, uint64_t step0, const float* proposal_params,
                                           double proposal_eps, int8_t* samples_out, double* logpsi_out,
                                           int32_t* n_accepted, double* trace, void* workspace,
                                           size_t workspace_bytes, void* stream) {
  gna_status st = check_gd(g, d);
  if (st != GNA_OK) return st;
  if (C < 0 || C > (int64_t)1 << 31 || n_sweeps < 0 || record_every < 0) return GNA_ERR_INVALID_ARG;
  if (C == 0 || n_sweeps == 0) return GNA_OK;
  if (g->d.E < 1) return GNA_ERR_INVALID_ARG;  // no bond to propose
  if (!theta || !chain_spins) return GNA_ERR_INVALID_ARG;
  if (record_every > 0 && n_sweeps / record_every > 0 && !samples_out && !logpsi_out) return GNA_ERR_INVALID_ARG;
  if (proposal_params && !(proposal_eps >= 0.0 && proposal_eps <= 1.0)) return GNA_ERR_INVALID_ARG;
  st = check_ws(g, d, proposal_params ? GNA_OP_METROPOLIS_LEARNED : GNA_OP_METROPOLIS, C, workspace, workspace_bytes);
  if (st != GNA_OK) return st;
  SimtCall sc{};
  sc.g = g;
  sc.m = make_dims(g, d);
  sc.op = 3;
  sc.theta = theta;
  sc.B = C;
  sc.chain_spins = chain_spins;
  sc.n_sweeps = n_sweeps;
  sc.record_every = record_every;
  sc.seed = seed;
  sc.step0 = step0;
  sc.samples_out = samples_out;
  sc.logpsi_out = logpsi_out;
  sc.n_acc = n_accepted;
  sc.trace = trace;
  sc.prop = proposal_params;
  sc.prop_eps = proposal_eps;
  // BF16 models, plain moves: the tensor-core sampler; otherwise the warp-per-chain sampler
  // when the model fits it, else one chain per CTA
  size_t need = 0;
  if (tensor_prec(d) && !proposal_params && tcm_workspace(g, sc.m, C, &need) == GNA_OK) {
    TcmCall tc{g, sc.m, (const float*)theta, chain_spins, C, n_sweeps, record_every, seed, step0,
               samples_out, logpsi_out, n_accepted, trace};
    return tcm_run(tc, workspace, workspace_bytes, (cudaStream_t)stream);
  }
  if (d->act == GNA_ACT_TANH &&
      metro_workspace(g, sc.m, simt_prec(d), C, proposal_params != nullptr, &need) == GNA_OK) {
    MetroCall mc{g, sc.m, theta, chain_spins, C, n_sweeps, record_every, seed, step0,
                 samples_out, logpsi_out, n_accepted, trace, proposal_params, proposal_eps};
    return metro_run(mc, simt_prec(d), workspace, workspace_bytes, (cudaStream_t)stream);
  }
  return simt_run(sc, simt_prec(d), workspace, workspace_bytes, (cudaStream_t)stream);
}

extern "C" gna_status gna_backward(const gna_graph* g, const gna_model_desc* d, const void* theta,
                                   const int8_t* spins, int64_t B, const double* cot, double* grad, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  gna_status st = check_gd(g, d);
  if (st != GNA_OK) return st;
  if (B < 0 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (!theta || !grad || (B > 0 && (!spins || !cot))) return GNA_ERR_INVALID_ARG;
  st = check_ws(g, d, GNA_OP_BACKWARD, B, workspace, workspace_bytes);
  if (st != GNA_OK) return st;
  // BF16 models: the tensor-core backward when the model fits it
  size_t need = 0;
  if (tensor_prec(d) && tcb_workspace(g, make_dims(g, d), B, &need) == GNA_OK) {
    TcbCall tc{g, make_dims(g, d), (const float*)theta, spins, B, cot, grad};
    return tcb_run(tc, workspace, workspace_bytes, (cudaStream_t)stream);
  }
  SimtCall sc{};
  sc.g = g;
  sc.m = make_dims(g, d);
  sc.op = 4;
  sc.theta = theta;
  sc.spins = spins;
  sc.B = B;
  sc.cot = cot;
  sc.grad = grad;
  return simt_run(sc, simt_prec(d), workspace, workspace_bytes, (cudaStream_t)stream);
}

extern "C" gna_status gna_backward_static(const gna_graph* g, const gna_model_desc* d, const void* theta,
                                          const int8_t* spins, int64_t B, const double* cot, double* grad,
                                          void* stream) {
  gna_status st = check_gd(g, d);
  if (st != GNA_OK) return st;
  if (B < 0 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (!theta || !grad || (B > 0 && (!spins || !cot))) return GNA_ERR_INVALID_ARG;
  // BF16 models: the tensor-core backward of gna_backward, with its scratch in the fixed array
  size_t need = 0;
  if (tensor_prec(d) && tcb_workspace(g, make_dims(g, d), B, &need) == GNA_OK) {
    void* base = nullptr;
    size_t bytes = 0;
    st = static_scratch(&base, &bytes);
    if (st != GNA_OK) return st;
    TcbCall tc{g, make_dims(g, d), (const float*)theta, spins, B, cot, grad};
    return tcb_run_fixed(tc, base, bytes, (cudaStream_t)stream);
  }
  SimtCall sc{};
  sc.g = g;
  sc.m = make_dims(g, d);
  sc.op = 4;
  sc.theta = theta;
  sc.spins = spins;
  sc.B = B;
  sc.cot = cot;
  sc.grad = grad;
  return simt_backward_static(sc, simt_prec(d), (cudaStream_t)stream);
}

extern "C" gna_status gna_dedup_workspace_size(int64_t B, int32_t n_sites, size_t* bytes) {
  if (!bytes || B < 0 || B >= (int64_t)1 << 31 || n_sites < 1 || n_sites > 4096) return GNA_ERR_INVALID_ARG;
  *bytes = dedup_workspace(B, n_sites);
  return GNA_OK;
}

extern "C" gna_status gna_dedup(int32_t n_sites, const int8_t* spins, const double* logpsi, int64_t B,
                                int8_t* u_spins, double* u_logpsi, double* counts, int64_t* n_unique,
                                void* workspace, size_t workspace_bytes, void* stream) {
  if (B < 0 || B >= (int64_t)1 << 31 || n_sites < 1 || n_sites > 4096 || !n_unique) return GNA_ERR_INVALID_ARG;
  if (B > 0 && (!spins || !u_spins || !counts || (logpsi && !u_logpsi))) return GNA_ERR_INVALID_ARG;
  return dedup_run(n_sites, spins, logpsi, B, u_spins, u_logpsi, counts, n_unique, workspace, workspace_bytes,
                   (cudaStream_t)stream);
}

extern "C" gna_status gna_isgo_weights_workspace(int64_t B, size_t* bytes) {
  if (!bytes || B < 1 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  *bytes = isgo_weights_ws(B);
  return GNA_OK;
}

extern "C" gna_status gna_isgo_weights(const double* logpsi, const double* logpsi0, const double* eloc,
                                       const double* counts, int64_t B, double* cot, double* stats, void* workspace,
                                       size_t workspace_bytes, void* stream) {
  if (B < 1 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (!logpsi || !logpsi0 || !eloc || !stats) return GNA_ERR_INVALID_ARG;
  if (workspace_bytes < isgo_weights_ws(B) || !workspace) return GNA_ERR_WORKSPACE;
  return isgo_weights_launch(logpsi, logpsi0, eloc, counts, B, cot, stats, workspace, (cudaStream_t)stream);
}

extern "C" gna_status gna_isgo_partials(const double* logpsi, const double* logpsi0, const double* eloc,
                                        const double* counts, int64_t B, double* part, void* workspace,
                                        size_t workspace_bytes, void* stream) {
  if (B < 1 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (!logpsi || !logpsi0 || !eloc || !part) return GNA_ERR_INVALID_ARG;
  if (workspace_bytes < isgo_weights_ws(B) || !workspace) return GNA_ERR_WORKSPACE;
  return isgo_partials_launch(logpsi, logpsi0, eloc, counts, B, part, workspace, (cudaStream_t)stream);
}

extern "C" gna_status gna_isgo_finish(const double* logpsi, const double* logpsi0, const double* eloc,
                                      const double* counts, int64_t B, const double* global, double* cot,
                                      double* part, void* workspace, size_t workspace_bytes, void* stream) {
  if (B < 1 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (!logpsi || !logpsi0 || !eloc || !global || !part) return GNA_ERR_INVALID_ARG;
  if (workspace_bytes < isgo_weights_ws(B) || !workspace) return GNA_ERR_WORKSPACE;
  return isgo_finish_launch(logpsi, logpsi0, eloc, counts, B, global, cot, part, workspace, (cudaStream_t)stream);
}

extern "C" gna_status isgo_grad(const gna_graph* g, const gna_model_desc* d, const void* theta, const int8_t* spins,
                                const double* logpsi0, const double* counts, int64_t B, double* grad, double* stats,
                                void* workspace, size_t workspace_bytes, void* stream) {
  gna_status st = check_gd(g, d);
  if (st != GNA_OK) return st;
  if (B < 1 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (!theta || !spins || !logpsi0 || !grad || !stats) return GNA_ERR_INVALID_ARG;
  st = check_ws(g, d, GNA_OP_ISGO_GRAD, B, workspace, workspace_bytes);
  if (st != GNA_OK) return st;
  unsigned char* w = (unsigned char*)workspace;
  const size_t vec = align_up((size_t)B * 2 * sizeof(double));
  double* lp = (double*)w;
  double* E = (double*)(w + vec);
  double* cot = (double*)(w + 2 * vec);
  unsigned char* inner = w + 3 * vec;
  const size_t inner_bytes = workspace_bytes - 3 * vec;
  st = gna_local_energy_logpsi(g, d, theta, spins, B, E, lp, inner, inner_bytes, stream);
  if (st != GNA_OK) return st;
  st = isgo_weights_launch(lp, logpsi0, E, counts, B, cot, stats, inner, (cudaStream_t)stream);
  if (st != GNA_OK) return st;
  return gna_backward(g, d, theta, spins, B, cot, grad, inner, inner_bytes, stream);
}

extern "C" gna_status gna_sgd_update(const gna_model_desc* d, void* theta, const double* grad, double lr,
                                     void* stream) {
  if (!desc_ok(d) || !theta || !grad || !std::isfinite(lr)) return GNA_ERR_INVALID_ARG;
  return sgd_launch(d->prec, theta, grad, lr, (int)gna_num_params(d), (cudaStream_t)stream);
}

extern "C" int32_t gna_proposal_num_params(void) { return kPropParams; }

static gna_status check_graph(const gna_graph* g) {
  if (!g) return GNA_ERR_INVALID_ARG;
  int dev = 0;
  GNA_CUDA_TRY(cudaGetDevice(&dev));
  return dev == g->device ? GNA_OK : GNA_ERR_INVALID_ARG;
}

extern "C" gna_status gna_proposal_workspace_size(const gna_graph* g, int64_t B, size_t* bytes) {
  gna_status st = check_graph(g);
  if (st != GNA_OK) return st;
  if (!bytes || B < 0) return GNA_ERR_INVALID_ARG;
  *bytes = B == 0 ? 0 : prop_workspace(g, B);
  return GNA_OK;
}

extern "C" gna_status gna_proposal_logits(const gna_graph* g, const int8_t* spins, int64_t B, const float* params,
                                          float* logits, void* stream) {
  gna_status st = check_graph(g);
  if (st != GNA_OK) return st;
  if (B < 0 || B > (int64_t)1 << 31) return GNA_ERR_INVALID_ARG;
  if (B == 0 || g->d.E == 0) return GNA_OK;
  if (!spins || !params || !logits) return GNA_ERR_INVALID_ARG;
  return prop_logits_launch(g, spins, B, params, logits, (cudaStream_t)stream);
}

extern "C" gna_status gna_proposal_grad(const gna_graph* g, const int8_t* spins, const float* dlogpsi_bonds,
                                        int64_t B, const float* params, double* grad, double* loss, void* workspace,
                                        size_t workspace_bytes, void* stream) {
  gna_status st = check_graph(g);
  if (st != GNA_OK) return st;
  if (B < 1 || B > (int64_t)1 << 31 || g->d.E == 0) return GNA_ERR_INVALID_ARG;
  if (!spins || !dlogpsi_bonds || !params || !grad) return GNA_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < prop_workspace(g, B)) return GNA_ERR_WORKSPACE;
  return prop_grad_launch(g, spins, dlogpsi_bonds, B, params, grad, loss, workspace, (cudaStream_t)stream);
}

extern "C" gna_status gna_proposal_adam(float* params, float* m, float* v, const double* grad, int32_t t, double lr,
                                        void* stream) {
  if (!params || !m || !v || !grad || t < 1 || !std::isfinite(lr)) return GNA_ERR_INVALID_ARG;
  return prop_adam_launch(params, m, v, grad, t, lr, (cudaStream_t)stream);
}

extern "C" gna_status gna_philox4x64_10(const uint64_t* keys, const uint64_t* counters, int64_t n, uint64_t* out,
                                        void* stream) {
  if (n < 0 || (n > 0 && (!keys || !counters || !out))) return GNA_ERR_INVALID_ARG;
  return philox_launch(keys, counters, n, out, (cudaStream_t)stream);
}

extern "C" gna_status gna_device_status(int32_t* flags, int32_t clear) {
  if (!flags) return GNA_ERR_INVALID_ARG;
  GNA_CUDA_TRY(cudaDeviceSynchronize());
  int f = 0;
  gna_status st = isgo_read_status(&f, clear);
  if (st != GNA_OK) return st;
  st = tc_read_status(&f, clear);
  if (st != GNA_OK) return st;
  *flags = f;
  if (f & 1) return GNA_ERR_TIMEOUT;
  if (f & 2) return GNA_ERR_NONFINITE;
  if (f & 4) return GNA_WARN_DEGENERATE_WEIGHTS;
  return GNA_OK;
}

extern "C" gna_status gna_debug_wait_limit(uint32_t iterations) {
  set_wait_limit(iterations);
  return GNA_OK;
}

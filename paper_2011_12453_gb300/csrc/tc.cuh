// Tensor-core (tcgen05, BF16 operands, FP32 accumulation in TMEM) kernels: interface.
#pragma once

#include "common.cuh"

namespace gna {

enum TcOp { TC_FWD = 0, TC_ELOC = 1, TC_BWD = 2 };

struct TcCall {
  const gna_graph* g;
  Dims m;
  int op;
  const float* theta;
  const int8_t* spins;
  int64_t B;
  double* logpsi;  // TC_FWD: [B][2]; TC_ELOC: [B][2] or NULL (log Psi from the call's own forward)
  double* eloc;    // TC_ELOC: [B][2]
  float* dlogpsi;  // TC_ELOC: [B][E] or NULL
  int split = 0;   // 1: operands as hi + lo BF16 pairs (GNA_PREC_BF16X2)
};

// Plain-move Metropolis sweeps of BF16 models on the tensor cores (same move rule and
// outputs as gna_metropolis_sweep's CUDA-core samplers).
struct TcmCall {
  const gna_graph* g;
  Dims m;
  const float* theta;
  int8_t* chain_spins;
  int64_t C;
  int32_t n_sweeps, record_every;
  uint64_t seed, step0;
  int8_t* samples_out;
  double* logpsi_out;
  int32_t* n_acc;
  double* trace;
};

// Backward VJP of BF16 models on the tensor cores: grad = sum_x cot_x . d log Psi_x / d theta.
struct TcbCall {
  const gna_graph* g;
  Dims m;
  const float* theta;
  const int8_t* spins;
  int64_t B;
  const double* cot;  // [B][2]
  double* grad;       // [P]
};

gna_status tc_workspace(const gna_graph* g, const Dims& m, int op, int64_t B, size_t* bytes, int split);
gna_status tcb_workspace(const gna_graph* g, const Dims& m, int64_t B, size_t* bytes);
gna_status tcb_run(const TcbCall& c, void* ws, size_t ws_bytes, cudaStream_t stream);
// Same backward with its scratch in a fixed array of scratch_bytes (the grid is reduced to fit).
gna_status tcb_run_fixed(const TcbCall& c, void* scratch, size_t scratch_bytes, cudaStream_t stream);
gna_status tcm_workspace(const gna_graph* g, const Dims& m, int64_t C, size_t* bytes);
gna_status tcm_run(const TcmCall& c, void* ws, size_t ws_bytes, cudaStream_t stream);
gna_status tc_run(const TcCall& c, void* ws, size_t ws_bytes, cudaStream_t stream);
gna_status tc_read_status(int* flags, int clear);
// Iterations of the bounded MMA waits of tensor-core kernels launched from now on
// (UINT32_MAX: the default).
void set_wait_limit(uint32_t iters);

}  // namespace gna

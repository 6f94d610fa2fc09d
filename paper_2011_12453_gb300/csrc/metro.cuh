// Warp-per-chain Metropolis sampler (metro.cu): interface.
#pragma once

#include "common.cuh"

namespace gna {

struct MetroCall {
  const gna_graph* g;
  Dims m;
  const void* theta;
  int8_t* chain_spins;
  int64_t C;
  int32_t n_sweeps, record_every;
  uint64_t seed, step0;
  int8_t* samples_out;
  double* logpsi_out;
  int32_t* n_acc;
  double* trace;
  const float* prop;  // learned proposal network or NULL
  double prop_eps;
};

// GNA_ERR_UNSUPPORTED when the model or graph does not fit this sampler (the caller then
// uses the CTA-per-chain sampler).
gna_status metro_workspace(const gna_graph* g, const Dims& m, int prec, int64_t C, int with_prop, size_t* bytes);
gna_status metro_run(const MetroCall& mc, int prec, void* ws, size_t ws_bytes, cudaStream_t stream);

}  // namespace gna

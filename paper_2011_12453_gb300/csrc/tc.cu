// Tensor-core BF16 kernels (placeholder until the tcgen05 path lands).
#include "tc.cuh"

namespace gna {

gna_status tc_workspace(const gna_graph*, const Dims&, int, int64_t, size_t*) { return GNA_ERR_UNSUPPORTED; }
gna_status tc_run(const TcCall&, void*, size_t, cudaStream_t) { return GNA_ERR_UNSUPPORTED; }
gna_status tc_read_status(int*, int) { return GNA_OK; }

}  // namespace gna

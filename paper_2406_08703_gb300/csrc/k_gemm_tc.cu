// Tensor-core (tcgen05) form of the MFT contractions -- placeholder until the kernel lands.
#include "dlx_common.cuh"
namespace dlx {
int tc_supported(const dlx_plan *, std::string *why) { *why = "tensor-core form not built yet"; return 0; }
int tc_make_maps(dlx_plan *, std::string *why) { *why = "not built"; return 0; }
cudaError_t tc_forward(dlx_plan *, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_adjoint_chunk(dlx_plan *, const DevParams &, int, int, cudaStream_t) { return cudaErrorNotSupported; }
}

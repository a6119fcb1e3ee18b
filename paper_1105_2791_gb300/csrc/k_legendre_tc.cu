// Tensor-core (tcgen05) Legendre sums: placeholder until the sm_103a kernel lands.
#include "modal_internal.cuh"

namespace modal {

cudaError_t build_tc_tables(Plan& pl, cudaStream_t) {
    (void)pl;
    return cudaErrorNotSupported;
}

void free_tc_tables(Plan& pl) { (void)pl; }

cudaError_t launch_legendre_tc(const Plan&, const float2*, int, float2*, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace modal

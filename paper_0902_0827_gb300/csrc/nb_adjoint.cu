// nb_adjoint.cu - adjoint of the non-bonded forces (placeholder until the
// adjoint kernel lands).
#include "nb_internal.cuh"

namespace acenb {

cudaError_t launch_backward(nb_ctx *, const float *, const float *, const int32_t *, const float *, const double *,
                            float *, float *, double *, double *)
{
    return cudaErrorNotSupported;
}

}  // namespace acenb

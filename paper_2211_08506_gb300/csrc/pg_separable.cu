// Separable tcgen05 contraction (sm_103a) - placeholder until the tensor-core kernel lands.
#include "pg_internal.h"

namespace pgi {

bool separable_supported(const Geometry &, int) { return false; }

cudaError_t separable_plan(const SeparableArgs &, int, const pg_tuning &, int, KernelLaunch *)
{
    return cudaErrorNotSupported;
}

}  // namespace pgi

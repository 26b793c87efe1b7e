// Voxel-integrated (erf) instantiations of the direct kernel (Sec. III-A), compiled apart
// from the point-sampled ones so that the two translation units build in parallel.
#include "direct_kernel.cuh"

namespace pgi {

const void *pick_direct_integral(int dtype, bool vec_ok, int cutoff, int periodic, int hint)
{
    return pick_direct<1>(dtype, vec_ok, cutoff, periodic, hint, false);
}

}  // namespace pgi

// Weighted instantiations of the direct kernel (weighted grids, Sec. III-A), for both voxel
// forms, compiled apart from the unweighted ones so that the translation units build in
// parallel.
#include "direct_kernel.cuh"

namespace pgi {

const void *pick_direct_weighted(int dtype, bool vec_ok, int cutoff, int periodic, int form)
{
    return form == PG_FORM_INTEGRAL ? pick_weighted<1>(dtype, vec_ok, cutoff, periodic)
                                    : pick_weighted<0>(dtype, vec_ok, cutoff, periodic);
}

}  // namespace pgi

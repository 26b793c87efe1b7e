// Launch planning for the direct kernel (sm_103a): the point-sampled instantiations live in
// this translation unit, the voxel-integrated ones in pg_direct_integral.cu, so that the two
// compile in parallel.  The kernel itself is in direct_kernel.cuh.
#include "direct_kernel.cuh"

namespace pgi {

cudaError_t direct_plan(const DirectArgs &a, int dtype, int vec_ok, const pg_tuning &t,
                        int sm_count, KernelLaunch *kl)
{
    const int hint = t.store_hint == 1 ? 1 : 0;
    const bool lanes = a.lane_lists != 0 && a.geo.cutoff != PG_CUTOFF_NONE;
    const int cut = a.geo.cutoff, per = a.geo.periodic;
    const void *f = a.in.weight ? pick_direct_weighted(dtype, vec_ok != 0, cut, per, a.geo.form)
                    : a.geo.form == PG_FORM_INTEGRAL
                        ? pick_direct_integral(dtype, vec_ok != 0, cut, per, hint)
                        : pick_direct<0>(dtype, vec_ok != 0, cut, per, hint, lanes);

    int threads = t.block_threads;
    if (threads != 128 && threads != 256 && threads != 512) threads = 256;
    const size_t per_warp = (size_t)direct_warp_floats(a.erf_tab) * sizeof(float);
    while (threads > 128 && (size_t)(threads / 32) * per_warp > 200 * 1024) threads /= 2;
    const size_t smem = (size_t)(threads / 32) * per_warp;
    int per_sm = 0;
    cudaError_t e = occupancy(f, threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (t.blocks_per_sm > 0 && t.blocks_per_sm < per_sm) per_sm = t.blocks_per_sm;
    const long long items = (long long)a.geo.n_mol * a.geo.C * a.geo.nx;
    const long long need = (items + threads / 32 - 1) / (threads / 32);
    long long blocks = (long long)sm_count * per_sm;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kl->func = f;
    kl->grid = dim3((unsigned)blocks);
    kl->block = dim3((unsigned)threads);
    kl->smem = smem;
    set_args(kl, a);
    return cudaSuccess;
}

}  // namespace pgi

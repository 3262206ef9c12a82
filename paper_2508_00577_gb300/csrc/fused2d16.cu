// Fused single-pass D2Q9 step with FP16 / BF16 deviation storage (dev16.cuh): the kernels
// of fused2d_launch.cuh instantiated for the 16-bit types (no wall columns), in a
// translation unit of their own so that they compile beside the FP32 ones.
#include "fused2d_launch.cuh"

namespace evlbm {

using namespace fused2d_impl;

namespace {

template <typename S>
cudaError_t step16(const KParams &p, const void *f, const void *g, void *fo, void *go, const void *RT_iso,
                   const void *Rin, void *Rout, cudaStream_t st)
{
    FusedArgs A = make_args(p, f, g, fo, go, RT_iso, Rin, Rout);
    int W;
    bool balanced;
    launch_shape(p, A, W, balanced);
    return p.thermal ? launch<true, false, S>(W, A, p.nz, balanced, st) : launch<false, false, S>(W, A, p.nz, balanced, st);
}

}  // namespace

EVLBM_DEFINE_OOB_READER(fused2d16_oob)

cudaError_t fused2d_step16(int prec, const KParams &p, const void *f, const void *g, void *fo, void *go,
                           const void *RT_iso, const void *Rin, void *Rout, cudaStream_t st)
{
    if (prec == 2) return step16<__half>(p, f, g, fo, go, RT_iso, Rin, Rout, st);
    if (prec == 3) return step16<__nv_bfloat16>(p, f, g, fo, go, RT_iso, Rin, Rout, st);
    return cudaErrorNotSupported;
}

}  // namespace evlbm

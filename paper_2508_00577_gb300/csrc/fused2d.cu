// Fused single-pass D2Q9 step with FP32 storage: one launch per time step (kernels in
// fused2d_launch.cuh, tile body in fused2d_tile.cuh); 16-bit storage is instantiated in
// fused2d16.cu.
#include "fused2d_launch.cuh"

namespace evlbm {

using namespace fused2d_impl;

EVLBM_DEFINE_OOB_READER(fused2d_oob)

const int kFusedWidths[kFusedWidthCount] = {64, 96, 128, 192};

bool fused2d_supported(int prec, int Q, const KParams &p)
{
    return prec >= 1 && prec <= 3 && Q == 9 && p.force_form == 0 && (prec == 1 || !p.walls) &&
           (long long)9 * p.N < (1LL << 31);
}

void fused2d_default_tile(const KParams &p, int *W, int *H)
{
    *W = p.nx >= 128 ? 128 : (p.nx > 64 ? 96 : 64);
    const int h = p.ny <= 128 ? p.ny : 128;
    *H = h + (h & 1);
}

cudaError_t fused2d_step(int prec, const KParams &p, const void *f, const void *g, void *fo, void *go,
                         const void *RT_iso, const void *Rin, void *Rout, cudaStream_t st)
{
    if (!fused2d_supported(prec, 9, p)) return cudaErrorNotSupported;
    if (prec != 1) return fused2d_step16(prec, p, f, g, fo, go, RT_iso, Rin, Rout, st);
    FusedArgs A = make_args(p, f, g, fo, go, RT_iso, Rin, Rout);
    int W;
    bool balanced;
    launch_shape(p, A, W, balanced);
    if (p.walls)
        return p.thermal ? launch<true, true, float>(W, A, p.nz, balanced, st)
                         : launch<false, true, float>(W, A, p.nz, balanced, st);
    return p.thermal ? launch<true, false, float>(W, A, p.nz, balanced, st)
                     : launch<false, false, float>(W, A, p.nz, balanced, st);
}

}  // namespace evlbm

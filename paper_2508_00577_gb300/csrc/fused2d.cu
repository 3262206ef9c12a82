// Fused single-pass D2Q9 step: one launch per time step, one CTA per tile
// (strip x chunk x layer).  The tile body is in fused2d_tile.cuh.
#include "fused2d_tile.cuh"

namespace evlbm {

namespace {

using namespace fused;

template <int kW, bool THERMAL>
__global__ void __launch_bounds__(threads_of<kW>(), Shape<kW>::MINB) k_fused2d(FusedArgs A)
{
    extern __shared__ v2 smem[];
    fused_tile<kW, THERMAL, false>(A, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

template <int W, bool THERMAL>
cudaError_t launch_w(const FusedArgs &A, int nz, cudaStream_t st)
{
    static bool attr = false;
    constexpr size_t smem = smem_of<W>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_fused2d<W, THERMAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((A.nx + W - 1) / W, (A.ny + A.H - 1) / A.H, nz);
    k_fused2d<W, THERMAL><<<grid, threads_of<W>(), smem, st>>>(A);
    return cudaGetLastError();
}

template <bool THERMAL>
cudaError_t launch(int W, const FusedArgs &A, int nz, cudaStream_t st)
{
    switch (W) {
    case 64: return launch_w<64, THERMAL>(A, nz, st);
    case 96: return launch_w<96, THERMAL>(A, nz, st);
    case 192: return launch_w<192, THERMAL>(A, nz, st);
    default: return launch_w<128, THERMAL>(A, nz, st);
    }
}

}  // namespace

EVLBM_DEFINE_OOB_READER(fused2d_oob)

const int kFusedWidths[kFusedWidthCount] = {64, 96, 128, 192};

bool fused2d_supported(int prec, int Q, const KParams &p)
{
    return prec == 1 && Q == 9 && p.force_form == 0 && (long long)9 * p.N < (1LL << 31);
}

void fused2d_default_tile(const KParams &p, int *W, int *H)
{
    *W = p.nx >= 128 ? 128 : (p.nx > 64 ? 96 : 64);
    const int h = p.ny <= 128 ? p.ny : 128;
    *H = h + (h & 1);
}

cudaError_t fused2d_step(int prec, const KParams &p, const void *f, const void *g, void *fo, void *go,
                         const void *RT_iso, cudaStream_t st)
{
    if (!fused2d_supported(prec, 9, p)) return cudaErrorNotSupported;
    FusedArgs A;
    A.f = static_cast<const float *>(f);
    A.g = static_cast<const float *>(g);
    A.fo = static_cast<float *>(fo);
    A.go = static_cast<float *>(go);
    A.RT_iso = static_cast<const float *>(RT_iso);
    A.nx = p.nx;
    A.ny = p.ny;
    A.nz = p.nz;
    A.N = (unsigned)p.N;
    A.eos = p.eos;
    A.a = float(p.a);
    A.b = float(p.b);
    A.kappa = float(p.kappa);
    A.lambda = float(p.lambda);
    A.c_eq = float(p.c_eq);
    A.c_star = float(p.c_star);
    int W = p.tile_w, H = p.tile_h;
    if (W <= 0 || H <= 0) fused2d_default_tile(p, &W, &H);
    A.H = H + (H & 1);                 // row pairs: chunks of an even number of rows
    return p.thermal ? launch<true>(W, A, p.nz, st) : launch<false>(W, A, p.nz, st);
}

}  // namespace evlbm

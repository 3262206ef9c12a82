// Fused single-pass D2Q9 step: one launch per time step, one CTA per tile
// (strip x chunk x layer).  The tile body is in fused2d_tile.cuh.
#include "fused2d_tile.cuh"

namespace evlbm {

namespace {

using namespace fused;

template <int kW, bool THERMAL, bool WALLS>
__global__ void __launch_bounds__(threads_of<kW>(), Shape<kW>::MINB) k_fused2d(FusedArgs A)
{
    extern __shared__ v2 smem[];
    const int y0 = blockIdx.y * A.H;                       // H is even
    fused_tile<kW, THERMAL, false, WALLS>(A, blockIdx.x, y0, min(A.H, A.ny - y0), blockIdx.z, smem);
}

// Balanced persistent variant: a grid of S x parts CTAs (S strips, parts = the
// resident CTAs of the GPU / S), CTA b taking strip b % S and the equal share b / S of
// that strip's row pairs over all layers (layer after layer).  Neighbouring strips
// then march over the same rows at the same time, as in the chunked grid, so the
// halo columns they share are re-read from L2 and each row is fetched from DRAM in
// one stretch.  A share that crosses the end of a layer becomes two tiles.
template <int kW, bool THERMAL, bool WALLS>
__global__ void __launch_bounds__(threads_of<kW>(), Shape<kW>::MINB) k_fused2d_bal(FusedArgs A)
{
    extern __shared__ v2 smem[];
    const int S = (A.nx + kW - 1) / kW, P = (A.ny + 1) / 2;
    const int parts = gridDim.x / S, strip = blockIdx.x % S, part = blockIdx.x / S;
    const long long T = (long long)A.nz * P;                 // row pairs of one strip, all layers
    const long long g1 = T * (part + 1) / parts;
    for (long long g = T * part / parts; g < g1;) {
        const int layer = (int)(g / P);
        const int p0 = (int)(g - (long long)layer * P);
        const int p1 = (int)min((long long)P, p0 + (g1 - g));
        const int y0 = 2 * p0;
        fused_tile<kW, THERMAL, false, WALLS>(A, strip, y0, min(2 * p1, A.ny) - y0, layer, smem);
        __syncthreads();
        g += p1 - p0;
    }
}

template <int W, bool THERMAL, bool WALLS>
cudaError_t launch_w(const FusedArgs &A, int nz, bool balanced, cudaStream_t st)
{
    static bool attr = false;
    static int resident = 0;
    constexpr size_t smem = smem_of<W>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_fused2d<W, THERMAL, WALLS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused2d_bal<W, THERMAL, WALLS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        int per_sm = 0, dev = 0, sms = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused2d_bal<W, THERMAL, WALLS>,
                                                              threads_of<W>(), smem);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorLaunchOutOfResources;
        resident = per_sm * sms;
        attr = true;
    }
    if (balanced) {
        const int S = (A.nx + W - 1) / W;
        const long long parts = min((long long)max(resident / S, 1), (long long)nz * ((A.ny + 1) / 2));
        k_fused2d_bal<W, THERMAL, WALLS><<<(unsigned)(S * parts), threads_of<W>(), smem, st>>>(A);
    } else {
        const dim3 grid((A.nx + W - 1) / W, (A.ny + A.H - 1) / A.H, nz);
        k_fused2d<W, THERMAL, WALLS><<<grid, threads_of<W>(), smem, st>>>(A);
    }
    return cudaGetLastError();
}

template <bool THERMAL, bool WALLS>
cudaError_t launch(int W, const FusedArgs &A, int nz, bool balanced, cudaStream_t st)
{
    switch (W) {
    case 64: return launch_w<64, THERMAL, WALLS>(A, nz, balanced, st);
    case 96: return launch_w<96, THERMAL, WALLS>(A, nz, balanced, st);
    case 192: return launch_w<192, THERMAL, WALLS>(A, nz, balanced, st);
    default: return launch_w<128, THERMAL, WALLS>(A, nz, balanced, st);
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
    A.walls = p.walls;
    A.wall_uy[0] = float(p.wall_u[0][1]);
    A.wall_uy[1] = float(p.wall_u[1][1]);
    A.wall_RT = float(p.wall_RT);
    int W = p.tile_w, H = p.tile_h;
    const bool balanced = W > 0 && H == kTileBalanced;
    if (W <= 0 || (H <= 0 && !balanced)) fused2d_default_tile(p, &W, &H);
    A.H = balanced ? 0 : H + (H & 1);  // row pairs: chunks of an even number of rows
    if (p.walls)
        return p.thermal ? launch<true, true>(W, A, p.nz, balanced, st) : launch<false, true>(W, A, p.nz, balanced, st);
    return p.thermal ? launch<true, false>(W, A, p.nz, balanced, st) : launch<false, false>(W, A, p.nz, balanced, st);
}

}  // namespace evlbm

// Kernels and launch of the fused single-pass D2Q9 step, templated on the storage type
// ST (float, or __half / __nv_bfloat16 deviations): one launch per time step, one CTA per
// tile (strip x chunk x layer) or the balanced persistent grid.  Included by fused2d.cu
// (FP32 storage) and fused2d16.cu (16-bit storage), which instantiate it.
#pragma once

#include "fused2d_tile.cuh"

namespace evlbm {
namespace fused2d_impl {

using namespace fused;

template <int kW, bool THERMAL, bool WALLS, typename ST>
__global__ void __launch_bounds__(threads_of<kW>(), Shape<kW>::MINB) k_fused2d(FusedArgs A)
{
    extern __shared__ v2 smem[];
    const int y0 = blockIdx.y * A.H;                       // H is even
    fused_tile<kW, THERMAL, false, WALLS, ST>(A, blockIdx.x, y0, min(A.H, A.ny - y0), blockIdx.z, smem);
}

// Balanced persistent variant: a grid of S x parts CTAs (S strips, parts = the
// resident CTAs of the GPU / S), CTA b taking strip b % S and the equal share b / S of
// that strip's row pairs over all layers (layer after layer).  Neighbouring strips
// then march over the same rows at the same time, as in the chunked grid, so the
// halo columns they share are re-read from L2 and each row is fetched from DRAM in
// one stretch.  A share that crosses the end of a layer becomes two tiles.
template <int kW, bool THERMAL, bool WALLS, typename ST>
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
        fused_tile<kW, THERMAL, false, WALLS, ST>(A, strip, y0, min(2 * p1, A.ny) - y0, layer, smem);
        __syncthreads();
        g += p1 - p0;
    }
}

template <int W, bool THERMAL, bool WALLS, typename ST>
cudaError_t launch_w(const FusedArgs &A, int nz, bool balanced, cudaStream_t st)
{
    static bool attr = false;
    static int resident = 0;
    constexpr size_t smem = smem_of<W>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_fused2d<W, THERMAL, WALLS, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fused2d_bal<W, THERMAL, WALLS, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        int per_sm = 0, dev = 0, sms = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused2d_bal<W, THERMAL, WALLS, ST>,
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
        k_fused2d_bal<W, THERMAL, WALLS, ST><<<(unsigned)(S * parts), threads_of<W>(), smem, st>>>(A);
    } else {
        const dim3 grid((A.nx + W - 1) / W, (A.ny + A.H - 1) / A.H, nz);
        k_fused2d<W, THERMAL, WALLS, ST><<<grid, threads_of<W>(), smem, st>>>(A);
    }
    return cudaGetLastError();
}

template <bool THERMAL, bool WALLS, typename ST>
cudaError_t launch(int W, const FusedArgs &A, int nz, bool balanced, cudaStream_t st)
{
    switch (W) {
    case 64: return launch_w<64, THERMAL, WALLS, ST>(A, nz, balanced, st);
    case 96: return launch_w<96, THERMAL, WALLS, ST>(A, nz, balanced, st);
    case 192: return launch_w<192, THERMAL, WALLS, ST>(A, nz, balanced, st);
    default: return launch_w<128, THERMAL, WALLS, ST>(A, nz, balanced, st);
    }
}


// Kernel arguments of a lattice (populations, records and the T field as passed by the caller).
inline FusedArgs make_args(const KParams &p, const void *f, const void *g, void *fo, void *go, const void *RT_iso,
                           const void *Rin, void *Rout)
{
    FusedArgs A;
    A.f = static_cast<const float *>(f);
    A.g = static_cast<const float *>(g);
    A.fo = static_cast<float *>(fo);
    A.go = static_cast<float *>(go);
    A.Rin = static_cast<const float *>(Rin);
    A.Rout = static_cast<float *>(Rout);
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
    return A;
}

// Launch shape of a step: strip width W and chunk height (A.H); balanced persistent grid.
inline void launch_shape(const KParams &p, FusedArgs &A, int &W, bool &balanced)
{
    int H = p.tile_h;
    W = p.tile_w;
    balanced = W > 0 && H == kTileBalanced;
    if (W <= 0 || (H <= 0 && !balanced)) fused2d_default_tile(p, &W, &H);
    A.H = balanced ? 0 : H + (H & 1);  // row pairs: chunks of an even number of rows
}

}  // namespace fused2d_impl
}  // namespace evlbm

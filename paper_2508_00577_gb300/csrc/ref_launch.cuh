// Host-side launchers of the stage kernels; included by one translation unit per
// arithmetic precision (the FP64 one is compiled without multiply-add contraction).
#pragma once

#include "ref_kernels.cuh"
#include "dispatch.h"

namespace evlbm {

template <typename real>
inline RefFields<real> ref_fields(void *scratch, long long N, const void *RT_iso)
{
    real *b = static_cast<real *>(scratch);
    RefFields<real> w;
    w.rho = b;          b += N;
    w.j = b;            b += 3 * N;
    w.Gam = b;          b += N;
    w.Pi = b;           b += 9 * N;
    w.lap = b;          b += N;
    w.A = b;            b += N;
    w.F = b;            b += 3 * N;
    w.u = b;            b += 3 * N;
    w.RT = b;           b += N;
    w.theta0 = b;       b += N;
    w.P0 = b;           b += N;
    w.gamma0 = b;       b += N;
    w.flux = b;         b += 3 * N;
    w.wq = b;           b += N;
    w.m_in = b;         b += N;
    w.RT_iso = static_cast<const real *>(RT_iso);
    return w;
}

inline dim3 node_grid(long long N, int block) { return dim3((unsigned)((N + block - 1) / block)); }

template <typename real, typename S, int Q>
cudaError_t ref_init_t(const KParams &p, const void *rho, const void *u, const void *RT, void *f, void *g,
                       void *Rout, cudaStream_t st)
{
    const int B = 256;
    k_init<real, S, Q><<<node_grid(p.N, B), B, 0, st>>>(p, static_cast<const real *>(rho),
                                                        static_cast<const real *>(u),
                                                        static_cast<const real *>(RT), static_cast<S *>(f),
                                                        static_cast<S *>(g), static_cast<float *>(Rout));
    return cudaGetLastError();
}

template <typename real, typename S, int Q>
cudaError_t ref_macro_t(const KParams &p, void *scratch, const void *RT_iso, const void *f, const void *g,
                        const void *Rin, cudaStream_t st)
{
    const int B = 256;
    const dim3 G = node_grid(p.N, B);
    RefFields<real> w = ref_fields<real>(scratch, p.N, RT_iso);
    k_moments<real, S, Q><<<G, B, 0, st>>>(p, static_cast<const S *>(f), static_cast<const S *>(g),
                                           static_cast<const float *>(Rin), w);
    k_stress<real, Q><<<G, B, 0, st>>>(p, w);
    k_macro<real, Q><<<G, B, 0, st>>>(p, w);
    return cudaGetLastError();
}

template <typename real, typename S, int Q>
cudaError_t ref_step_t(const KParams &p, void *scratch, const void *RT_iso, const void *f, const void *g, void *fo,
                       void *go, const void *Rin, void *Rout, cudaStream_t st)
{
    cudaError_t e = ref_macro_t<real, S, Q>(p, scratch, RT_iso, f, g, Rin, st);
    if (e != cudaSuccess) return e;
    const int B = 256;
    RefFields<real> w = ref_fields<real>(scratch, p.N, RT_iso);
    k_collide<real, S, Q><<<node_grid(p.N, B), B, 0, st>>>(p, w, static_cast<const S *>(f),
                                                           static_cast<const S *>(g), static_cast<S *>(fo),
                                                           static_cast<S *>(go), static_cast<const float *>(Rin),
                                                           static_cast<float *>(Rout));
    if constexpr (!Store<S>::dev) {
        if (p.walls) {
            const long long nw = 2LL * p.ny * p.nz;
            k_walls<real, S, Q><<<(unsigned)((nw + B - 1) / B), B, 0, st>>>(p, w, static_cast<S *>(fo),
                                                                             static_cast<S *>(go));
        }
    }
    return cudaGetLastError();
}

template <typename real, int Q>
cudaError_t ref_export_t(const KParams &p, void *scratch, double R, float *rho, float *u, float *T, cudaStream_t st)
{
    const int B = 256;
    RefFields<real> w = ref_fields<real>(scratch, p.N, nullptr);
    k_export_f32<real, Q><<<node_grid(p.N, B), B, 0, st>>>(p, w, R, rho, u, T);
    return cudaGetLastError();
}

template <typename S, int Q>
cudaError_t expand_t(const KParams &p, const void *src, const void *R, double *dst, int which, cudaStream_t st)
{
    const int B = 256;
    k_expand<S, Q><<<node_grid(p.N, B), B, 0, st>>>(p, static_cast<const S *>(src), static_cast<const float *>(R), dst,
                                                    which);
    return cudaGetLastError();
}

}  // namespace evlbm

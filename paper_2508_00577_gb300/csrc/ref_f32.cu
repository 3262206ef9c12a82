// FP32 instantiations of the stage kernels, with FP32, FP16-deviation and
// BF16-deviation population storage.
#include "ref_launch.cuh"

namespace evlbm {

#define EVLBM_PREC_Q(prec, Q, FN, ...)                                                       \
    ((prec) == 1 ? ((Q) == 9 ? FN<float, float, 9>(__VA_ARGS__) : FN<float, float, 27>(__VA_ARGS__))        \
     : (prec) == 2 ? ((Q) == 9 ? FN<float, __half, 9>(__VA_ARGS__) : FN<float, __half, 27>(__VA_ARGS__)) \
                   : ((Q) == 9 ? FN<float, __nv_bfloat16, 9>(__VA_ARGS__)                              \
                               : FN<float, __nv_bfloat16, 27>(__VA_ARGS__)))

cudaError_t ref_init_f32(int prec, int Q, const KParams &p, const void *rho, const void *u, const void *RT, void *f,
                         void *g, void *Rout, cudaStream_t st)
{
    return EVLBM_PREC_Q(prec, Q, ref_init_t, p, rho, u, RT, f, g, Rout, st);
}

cudaError_t ref_macro_f32(int prec, int Q, const KParams &p, void *scratch, const void *RT_iso, const void *f,
                          const void *g, const void *Rin, cudaStream_t st)
{
    return EVLBM_PREC_Q(prec, Q, ref_macro_t, p, scratch, RT_iso, f, g, Rin, st);
}

cudaError_t ref_step_f32(int prec, int Q, const KParams &p, void *scratch, const void *RT_iso, const void *f,
                         const void *g, void *fo, void *go, const void *Rin, void *Rout, cudaStream_t st)
{
    return EVLBM_PREC_Q(prec, Q, ref_step_t, p, scratch, RT_iso, f, g, fo, go, Rin, Rout, st);
}

cudaError_t ref_export_f32(int Q, const KParams &p, void *scratch, double R, float *rho, float *u, float *T,
                           cudaStream_t st)
{
    return Q == 9 ? ref_export_t<float, 9>(p, scratch, R, rho, u, T, st)
                  : ref_export_t<float, 27>(p, scratch, R, rho, u, T, st);
}

cudaError_t expand_f32(int prec, int Q, const KParams &p, const void *src, const void *R, double *dst, int which,
                       cudaStream_t st)
{
    if (prec == 1)
        return Q == 9 ? expand_t<float, 9>(p, src, R, dst, which, st) : expand_t<float, 27>(p, src, R, dst, which, st);
    if (prec == 2)
        return Q == 9 ? expand_t<__half, 9>(p, src, R, dst, which, st) : expand_t<__half, 27>(p, src, R, dst, which, st);
    return Q == 9 ? expand_t<__nv_bfloat16, 9>(p, src, R, dst, which, st)
                  : expand_t<__nv_bfloat16, 27>(p, src, R, dst, which, st);
}

}  // namespace evlbm

// FP64 instantiation of the stage kernels.  This translation unit is compiled
// with --fmad=false so that every multiply and add is rounded separately, as in
// the reference evaluation order of the step.
#include "ref_launch.cuh"

namespace evlbm {

#define EVLBM_Q_SWITCH(Q, CALL9, CALL27) ((Q) == 9 ? (CALL9) : (CALL27))

cudaError_t ref_init_f64(int Q, const KParams &p, const void *rho, const void *u, const void *RT, void *f, void *g,
                         cudaStream_t st)
{
    return EVLBM_Q_SWITCH(Q, (ref_init_t<double, double, 9>(p, rho, u, RT, f, g, nullptr, st)),
                          (ref_init_t<double, double, 27>(p, rho, u, RT, f, g, nullptr, st)));
}

cudaError_t ref_macro_f64(int Q, const KParams &p, void *scratch, const void *RT_iso, const void *f, const void *g,
                          cudaStream_t st)
{
    return EVLBM_Q_SWITCH(Q, (ref_macro_t<double, double, 9>(p, scratch, RT_iso, f, g, nullptr, st)),
                          (ref_macro_t<double, double, 27>(p, scratch, RT_iso, f, g, nullptr, st)));
}

cudaError_t ref_step_f64(int Q, const KParams &p, void *scratch, const void *RT_iso, const void *f, const void *g,
                         void *fo, void *go, cudaStream_t st)
{
    return EVLBM_Q_SWITCH(Q, (ref_step_t<double, double, 9>(p, scratch, RT_iso, f, g, fo, go, nullptr, nullptr, st)),
                          (ref_step_t<double, double, 27>(p, scratch, RT_iso, f, g, fo, go, nullptr, nullptr, st)));
}

cudaError_t ref_export_f64(int Q, const KParams &p, void *scratch, double R, float *rho, float *u, float *T,
                           cudaStream_t st)
{
    return EVLBM_Q_SWITCH(Q, (ref_export_t<double, 9>(p, scratch, R, rho, u, T, st)),
                          (ref_export_t<double, 27>(p, scratch, R, rho, u, T, st)));
}

cudaError_t expand_f64(int Q, const KParams &p, const void *src, double *dst, int which, cudaStream_t st)
{
    return EVLBM_Q_SWITCH(Q, (expand_t<double, 9>(p, src, nullptr, dst, which, st)),
                          (expand_t<double, 27>(p, src, nullptr, dst, which, st)));
}

}  // namespace evlbm

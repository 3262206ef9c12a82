// Internal interface between the surrogate kernels and the U-Net runtime.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/evsur.h"

namespace evsur {

typedef __nv_bfloat16 bf16;

int gemm(const sur_gemm_args &a, int *status, cudaStream_t st);

cudaError_t silu_bwd(const bf16 *dY, int ldd, const bf16 *Z, long long M, int C, bf16 *dZ, cudaStream_t st);
cudaError_t colsum(const bf16 *X, int ldx, long long M, int C, float *out, cudaStream_t st);
cudaError_t pool2(const bf16 *X, int ldx, long long Mc, int lh, int lw, int C, bf16 *Y, cudaStream_t st);
cudaError_t unpool2_acc(const bf16 *dY, long long Mc, int lh, int lw, int C, bf16 *dX, int ldx, cudaStream_t st);
cudaError_t pack_in(const float *x, long long M, const float *norm, bf16 *X, cudaStream_t st);
cudaError_t head(const bf16 *Y, long long M, const float *Wh, const float *bh, const float *norm, const float *x,
                 const float *yt, int mode, float *dO, float *loss, float *xn, cudaStream_t st);
cudaError_t head_bwd(const bf16 *Y, long long M, const float *Wh, const float *dO, bf16 *dY, float *dWh, float *dbh,
                     cudaStream_t st);
cudaError_t adam(float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t st);
cudaError_t conv_weights(const float *Wt, int Cin, int Cout, int Kp, int Kpo, bf16 *Wb, bf16 *Wf, cudaStream_t st);
cudaError_t up_weights(const float *Wm, int Cin, int Cout, bf16 *Wb, bf16 *Wt, cudaStream_t st);
cudaError_t indicators(const float *F, int batch, long long Mb, float rho_mid, double *out, int *nonfinite,
                       cudaStream_t st);

}  // namespace evsur

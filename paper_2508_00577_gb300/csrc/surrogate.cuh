// Internal interface between the surrogate kernels and the U-Net runtime.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/evsur.h"

namespace evsur {

typedef __nv_bfloat16 bf16;

// Halo-padded NHWC storage: a tensor of an H x W grid (H, W powers of two) is
// stored as [B][H+2][W+2][ld]; rows 0, H+1 and columns 0, W+1 hold the periodic
// copies of rows H-1, 0 and columns W-1, 0.  Interior pixel q = (b*H + y)*W + x.
// Stored (padded) position of interior pixel q of a 2^lh x 2^lw grid.
static __device__ __forceinline__ long long pad_pix(long long q, int lh, int lw)
{
    const int H = 1 << lh, W = 1 << lw;
    const long long b = q >> (lh + lw);
    const int y = (int)((q >> lw) & (H - 1)), x = (int)(q & (W - 1));
    return (b * (H + 2) + y + 1) * (W + 2) + x + 1;
}

// Stored position of child (0, 0) of coarse interior pixel q on the padded
// 2H x 2W grid; child (di, dj) is di*(2W+2) + dj further.
static __device__ __forceinline__ long long child0(long long q, int lh, int lw)
{
    const int H = 1 << lh, W = 1 << lw;
    const long long b = q >> (lh + lw);
    const int y = (int)((q >> lw) & (H - 1)), x = (int)(q & (W - 1));
    return (b * (2 * H + 2) + 2 * y + 1) * (2 * W + 2) + 2 * x + 1;
}

// Stored positions (main and periodic halo copies, up to 4) of interior pixel q.
static __device__ __forceinline__ int halo_targets(long long q, int lh, int lw, long long *out)
{
    const int H = 1 << lh, W = 1 << lw;
    const long long b = q >> (lh + lw);
    const int y = (int)((q >> lw) & (H - 1)), x = (int)(q & (W - 1));
    int ys[2] = {y + 1, -1}, xs[2] = {x + 1, -1};
    if (y == 0) ys[1] = H + 1;
    else if (y == H - 1) ys[1] = 0;
    if (x == 0) xs[1] = W + 1;
    else if (x == W - 1) xs[1] = 0;
    int n = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            if (ys[i] >= 0 && xs[j] >= 0) out[n++] = (b * (H + 2) + ys[i]) * (W + 2) + xs[j];
    return n;
}

static __device__ __forceinline__ uint4 pack8(const float *v)
{
    uint4 r;
    uint32_t *w = reinterpret_cast<uint32_t *>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    return r;
}

static __device__ __forceinline__ void store32_bf16(bf16 *dst, const float *v)
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = pack8(v + 8 * i);
}


int gemm(const sur_gemm_args &a, int *status, cudaStream_t st);
void set_tma(bool on);

cudaError_t silu_bwd(const bf16 *dY, int ldd, const bf16 *Z, long long M, int lh, int lw, int C, bf16 *dZ,
                     float *dbias, cudaStream_t st);
cudaError_t colsum(const bf16 *X, int ldx, long long M, int lh, int lw, int C, float *out, cudaStream_t st);
cudaError_t pool2(const bf16 *X, int ldx, long long Mc, int lh, int lw, int C, bf16 *Y, cudaStream_t st);
cudaError_t unpool2_acc(const bf16 *dY, long long Mc, int lh, int lw, int C, bf16 *dX, int ldx, cudaStream_t st);
cudaError_t pack_in(const float *x, long long M, int lh, int lw, const float *norm, bf16 *X, cudaStream_t st);
cudaError_t head(const bf16 *Y, long long M, int lh, int lw, const float *Wh, const float *bh, const float *norm,
                 const float *x, const float *yt, int mode, float *dO, float *loss, float *xn, cudaStream_t st);
cudaError_t head_bwd(const bf16 *Y, long long M, int lh, int lw, const float *Wh, const float *dO, bf16 *dY,
                     float *dWh, float *dbh, cudaStream_t st);
cudaError_t unroll_term(const float *xp, const float *yt, long long M, const float *norm, float inv, float *G, float *dO,
                        float *loss, cudaStream_t st);
cudaError_t conv0_dx(const bf16 *dZ, const bf16 *Wb, int Kp, long long M, int lh, int lw, const float *norm, float *G,
                     cudaStream_t st);
cudaError_t adam(float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t st);
cudaError_t conv_weights(const float *Wt, int Cin, int Cout, int Kp, int Kpo, bf16 *Wb, bf16 *Wf, cudaStream_t st);
cudaError_t up_weights(const float *Wm, int Cin, int Cout, bf16 *Wb, bf16 *Wt, cudaStream_t st);
cudaError_t indicators(const float *F, int batch, long long Mb, float rho_mid, double *out, int *invalid,
                       cudaStream_t st);
cudaError_t phase_flips(const float *A, const float *B, int batch, long long Mb, float rho_mid, double *out,
                        cudaStream_t st);
cudaError_t shift_rho(float *rho, int batch, long long Mb, const float *delta, cudaStream_t st);

}  // namespace evsur

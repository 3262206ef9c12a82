// Elementwise and reduction kernels of the learned surrogate on halo-padded
// NHWC tensors (see surrogate.cuh): SiLU backward, bias gradients, 2x2 average
// pooling and its adjoint, input packing, the 1x1 head with the loss or the
// state update, the loss terms and first-layer input gradient of unrolled
// training, Adam, the BF16 operand copies of the weights, and the per-domain
// fallback indicators.
#include <stdint.h>

#include "surrogate.cuh"

namespace evsur {

namespace {

inline int grid_1d(long long n)
{
    long long g = (n + 255) / 256;
    return (int)(g > 8192 ? 8192 : (g < 1 ? 1 : g));
}

// Kernels that end in per-channel atomics (block_colsum8): at most 512 blocks, so that
// each channel's accumulator takes at most 512 atomic additions per call.
inline int grid_red(long long n)
{
    const int g = grid_1d(n);
    return g > 512 ? 512 : g;
}

#define GRID_STRIDE(e, total)                                                                    \
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)(total); \
         e += (long long)gridDim.x * blockDim.x)

// Sum over the block of each thread's 8-channel partial sums into out[c] (atomic).  Every
// thread of a block keeps one channel group, threadIdx.x % C8: the grid stride and the
// block size (256) are multiples of C8 = C / 8 <= 32.
__device__ __forceinline__ void block_colsum8(const float acc[8], int C8, float *out)
{
    __shared__ float red[256][9];
#pragma unroll
    for (int j = 0; j < 8; ++j) red[threadIdx.x][j] = acc[j];
    __syncthreads();
    if ((int)threadIdx.x < C8) {
        for (int j = 0; j < 8; ++j) {
            float s = 0.f;
            for (int k = threadIdx.x; k < 256; k += C8) s += red[k][j];
            atomicAdd(out + threadIdx.x * 8 + j, s);
        }
    }
}

// dZ = dY * silu'(Z), silu'(z) = s (1 + z (1 - s)) with s = 1 / (1 + e^-z);
// 8 channels per thread; dZ gets its halo copies (it is gathered by the adjoint
// convolution).  dbias (may be NULL) += the column sums of the stored (BF16) dZ over
// the interior pixels: the bias gradient, without a second pass over dZ.
__global__ void __launch_bounds__(256) k_silu_bwd(const bf16 *dY, int ldd, const bf16 *Z, long long M, int lh,
                                                  int lw, int C, bf16 *dZ, float *dbias)
{
    const int C8 = C >> 3;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    GRID_STRIDE(e, M * C8)
    {
        const long long m = e / C8;
        const int c = (int)(e - m * C8) << 3;
        const long long p = pad_pix(m, lh, lw);
        const uint4 dv = *reinterpret_cast<const uint4 *>(dY + p * ldd + c);
        const uint4 zv = *reinterpret_cast<const uint4 *>(Z + p * C + c);
        const bf16 *dh = reinterpret_cast<const bf16 *>(&dv), *zh = reinterpret_cast<const bf16 *>(&zv);
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float z = __bfloat162float(zh[j]);
            const float s = 1.f / (1.f + __expf(-z));
            o[j] = __bfloat162float(dh[j]) * s * (1.f + z * (1.f - s));
        }
        const uint4 ov = pack8(o);
        const bf16 *oh = reinterpret_cast<const bf16 *>(&ov);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(oh[j]);
        long long tg[4];
        const int n = halo_targets(m, lh, lw, tg);
        for (int i = 0; i < n; ++i) *reinterpret_cast<uint4 *>(dZ + tg[i] * C + c) = ov;
    }
    if (dbias) block_colsum8(acc, C8, dbias);
}

// out[c] += sum over interior pixels of X[pix*ldx + c], c < C (bias gradients), 8
// channels (16 bytes) per load.
__global__ void __launch_bounds__(256) k_colsum(const bf16 *X, int ldx, long long M, int lh, int lw, int C,
                                                float *out)
{
    const int C8 = C >> 3;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    GRID_STRIDE(e, M * C8)
    {
        const long long m = e / C8;
        const int c = (int)(e - m * C8) << 3;
        const uint4 v = *reinterpret_cast<const uint4 *>(X + pad_pix(m, lh, lw) * ldx + c);
        const bf16 *h = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(h[j]);
    }
    block_colsum8(acc, C8, out);
}

// 2x2 average pooling: X (fine grid, ld ldx, first C channels) -> Y (coarse grid
// 2^lh x 2^lw, ld C) with halo copies.
__global__ void k_pool2(const bf16 *X, int ldx, long long Mc, int lh, int lw, int C, bf16 *Y)
{
    const int Wf2 = 2 * (1 << lw) + 2;
    GRID_STRIDE(e, Mc * C)
    {
        const long long q = e / C;
        const int c = (int)(e - q * C);
        const long long f = child0(q, lh, lw);
        const float s = __bfloat162float(X[f * ldx + c]) + __bfloat162float(X[(f + 1) * ldx + c]) +
                        __bfloat162float(X[(f + Wf2) * ldx + c]) + __bfloat162float(X[(f + Wf2 + 1) * ldx + c]);
        const bf16 v = __float2bfloat16_rn(0.25f * s);
        long long tg[4];
        const int n = halo_targets(q, lh, lw, tg);
        for (int i = 0; i < n; ++i) Y[tg[i] * C + c] = v;
    }
}

// Adjoint of the pooling, accumulated into the interior: dX[child] += dY[q] / 4.
__global__ void k_unpool2_acc(const bf16 *dY, long long Mc, int lh, int lw, int C, bf16 *dX, int ldx)
{
    const int Wf2 = 2 * (1 << lw) + 2;
    GRID_STRIDE(e, Mc * C)
    {
        const long long q = e / C;
        const int c = (int)(e - q * C);
        const float d = 0.25f * __bfloat162float(dY[pad_pix(q, lh, lw) * C + c]);
        const long long f = child0(q, lh, lw);
        const long long fs[4] = {f, f + 1, f + Wf2, f + Wf2 + 1};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            bf16 *p = dX + fs[s] * ldx + c;
            *p = __float2bfloat16_rn(__bfloat162float(*p) + d);
        }
    }
}

// Input packing: x fields [4][M] FP32 -> X (8 channels, halo-padded) BF16,
// channels 4..7 zero.
__global__ void k_pack_in(const float *x, long long M, int lh, int lw, const float *norm, bf16 *X)
{
    GRID_STRIDE(m, M)
    {
        float v[8];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = (x[c * M + m] - norm[c]) / norm[4 + c];
#pragma unroll
        for (int c = 4; c < 8; ++c) v[c] = 0.f;
        const uint4 pv = pack8(v);
        long long tg[4];
        const int n = halo_targets(m, lh, lw, tg);
        for (int i = 0; i < n; ++i) *reinterpret_cast<uint4 *>(X + tg[i] * 8) = pv;
    }
}

// 1x1 head (C -> 4) and its use: mode 0 = loss against targets, mode 1 = next state.
//   o[m][k] = bh[k] + sum_c Y[m][c] Wh[k][c]
//   mode 0: r = o - (y - x)/out_scale; loss += r^2 / (4M); dO[m][k] = 2 r / (4M)
//   mode 1: xn[k][m] = x[k][m] + out_scale[k] o[m][k]
template <int C>
__global__ void k_head(const bf16 *Y, long long M, int lh, int lw, const float *Wh, const float *bh,
                       const float *norm, const float *x, const float *yt, int mode, float *dO, float *loss,
                       float *xn)
{
    __shared__ float w[4 * C + 4];
    __shared__ float red[256];
    for (int i = threadIdx.x; i < 4 * C; i += blockDim.x) w[i] = Wh[i];
    if (threadIdx.x < 4) w[4 * C + threadIdx.x] = bh[threadIdx.x];
    __syncthreads();
    const float inv = 1.f / (4.f * (float)M);
    float acc = 0.f;
    GRID_STRIDE(m, M)
    {
        float o[4] = {w[4 * C], w[4 * C + 1], w[4 * C + 2], w[4 * C + 3]};
        const bf16 *yr = Y + pad_pix(m, lh, lw) * C;
#pragma unroll
        for (int c8 = 0; c8 < C; c8 += 8) {
            const uint4 v = *reinterpret_cast<const uint4 *>(yr + c8);
            const bf16 *h = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float yv = __bfloat162float(h[j]);
#pragma unroll
                for (int k = 0; k < 4; ++k) o[k] += yv * w[k * C + c8 + j];
            }
        }
        if (mode == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float r = o[k] - (yt[k * M + m] - x[k * M + m]) / norm[8 + k];
                acc += r * r;
                dO[m * 4 + k] = 2.f * r * inv;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) xn[k * M + m] = x[k * M + m] + norm[8 + k] * o[k];
        }
    }
    if (mode != 0) return;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv);
}

// Head backward (C = 32): dY[m][c] = sum_k dO[m][k] Wh[k][c]; dWh[k][c] += sum_m dO[m][k] Y[m][c];
// dbh[k] += sum_m dO[m][k].  One warp per pixel at a time, lane = channel.
// Unrolled training (k windows, each applied to the previous prediction): the loss
// term of a prediction x'_j against its target y_j, r = (x'_j - y_j) / out_scale, added
// to the planar field gradient G = dL/dx'_j as 2 r / out_scale * inv (inv = 1 / (4 M k)),
// and the output gradient of the window that produced x'_j, dO = out_scale * G
// (x'_j = x'_{j-1} + out_scale o).  loss += sum r^2 * inv.
__global__ void k_unroll_term(const float *xp, const float *yt, long long M, const float *norm, float inv, float *G,
                              float *dO, float *loss)
{
    __shared__ float red[256];
    float acc = 0.f;
    GRID_STRIDE(m, M)
    {
        float d[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float s = norm[8 + c];
            const float r = (xp[c * M + m] - yt[c * M + m]) / s;
            acc += r * r;
            const float g = G[c * M + m] + 2.f * r / s * inv;
            G[c * M + m] = g;
            d[c] = s * g;
        }
        *reinterpret_cast<float4 *>(dO + m * 4) = make_float4(d[0], d[1], d[2], d[3]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv);
}

// Input gradient of the first convolution (8 -> 32 channels) in its 4 field channels,
// dxin[p][c] = sum_tap sum_co W[tap * 8 + c][co] dZ[p - s_tap][co] (s_tap = (dy, dx); the
// periodic neighbours come from the halo of dZ), added to the planar field gradient:
// G[c][m] += dxin[m][c] / in_scale[c].  Wb is the forward BF16 copy [32][Kp].
__global__ void k_conv0_dx(const bf16 *dZ, const bf16 *Wb, int Kp, long long M, int lh, int lw, const float *norm,
                           float *G)
{
    __shared__ float w[9][32][4];
    for (int e = threadIdx.x; e < 9 * 32 * 4; e += blockDim.x) {
        const int tap = e / 128, co = (e / 4) % 32, c = e % 4;
        w[tap][co][c] = __bfloat162float(Wb[co * Kp + tap * 8 + c]);
    }
    __syncthreads();
    const long long Wp = (1 << lw) + 2;
    GRID_STRIDE(m, M)
    {
        const long long p = pad_pix(m, lh, lw);
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            const bf16 *z = dZ + (p - dy * Wp - dx) * 32;
#pragma unroll
            for (int c8 = 0; c8 < 32; c8 += 8) {
                const uint4 v = *reinterpret_cast<const uint4 *>(z + c8);
                const bf16 *h = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float zv = __bfloat162float(h[j]);
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[c] += w[tap][c8 + j][c] * zv;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) G[c * M + m] += acc[c] / norm[4 + c];
    }
}

__global__ void k_head_bwd(const bf16 *Y, long long M, int lh, int lw, const float *Wh, const float *dO, bf16 *dY,
                           float *dWh, float *dbh)
{
    __shared__ float red[8][4 * 32 + 4];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = Wh[k * 32 + lane];
    float gw[4] = {0, 0, 0, 0}, gb = 0.f;
    for (long long m = (long long)blockIdx.x * 8 + wi; m < M; m += (long long)gridDim.x * 8) {
        const float4 d = *reinterpret_cast<const float4 *>(dO + m * 4);
        const long long p = pad_pix(m, lh, lw) * 32 + lane;
        const float yv = __bfloat162float(Y[p]);
        dY[p] = __float2bfloat16_rn(d.x * w[0] + d.y * w[1] + d.z * w[2] + d.w * w[3]);
        gw[0] += d.x * yv;
        gw[1] += d.y * yv;
        gw[2] += d.z * yv;
        gw[3] += d.w * yv;
        if (lane < 4) gb += lane == 0 ? d.x : (lane == 1 ? d.y : (lane == 2 ? d.z : d.w));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[wi][k * 32 + lane] = gw[k];
    if (lane < 4) red[wi][128 + lane] = gb;
    __syncthreads();
    if (wi == 0) {
        for (int k = 0; k < 4; ++k) {
            float s = 0.f;
            for (int j = 0; j < 8; ++j) s += red[j][k * 32 + lane];
            atomicAdd(dWh + k * 32 + lane, s);
        }
        if (lane < 4) {
            float s = 0.f;
            for (int j = 0; j < 8; ++j) s += red[j][128 + lane];
            atomicAdd(dbh + lane, s);
        }
    }
}

// Adam with bias correction on FP32 masters (c1 = 1 - b1^t, c2 = 1 - b2^t).
__global__ void k_adam(float *w, const float *gr, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    GRID_STRIDE(i, n)
    {
        const float g = gr[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 operand copies of a 3x3 convolution from its master Wt [Kp][Cout]:
//   Wb [Cout][Kp]   (forward B operand, K = tap*Cin + ci)
//   Wf [Cin][Kpo]   (adjoint B operand, K = tap*Cout + co, taken at the mirrored tap 8 - tap)
__global__ void k_conv_weights(const float *Wt, int Cin, int Cout, int Kp, int Kpo, bf16 *Wb, bf16 *Wf)
{
    GRID_STRIDE(e, (long long)Cout * Kp)
    {
        const int co = (int)(e / Kp), k = (int)(e % Kp);
        Wb[e] = __float2bfloat16_rn(Wt[(long long)k * Cout + co]);
    }
    if (!Wf) return;
    GRID_STRIDE(e, (long long)Cin * Kpo)
    {
        const int ci = (int)(e / Kpo), k = (int)(e % Kpo);
        float v = 0.f;
        if (k < 9 * Cout) {
            const int tap = k / Cout, co = k % Cout;
            v = Wt[(long long)((8 - tap) * Cin + ci) * Cout + co];
        }
        Wf[e] = __float2bfloat16_rn(v);
    }
}

// BF16 copies of a transposed convolution from its master W [4 Cout][Cin]:
//   Wb [4 Cout][Cin] (forward B operand), Wt [Cin][4 Cout] (adjoint B operand).
__global__ void k_up_weights(const float *Wm, int Cin, int Cout, bf16 *Wb, bf16 *Wt)
{
    GRID_STRIDE(e, 4LL * Cout * Cin)
    {
        const int r = (int)(e / Cin), ci = (int)(e % Cin);
        const bf16 v = __float2bfloat16_rn(Wm[e]);
        Wb[e] = v;
        Wt[(long long)ci * 4 * Cout + r] = v;
    }
}

// Per-domain FP64 sums of rho and of the liquid count (rho > rho_mid): out[2b],
// out[2b+1]; invalid[0] |= 1 if any field is not finite or rho or T is not > 0.
// Interface-position indicator: per domain, the number of nodes whose phase (rho above or
// below rho_mid) differs between the density fields A and B (out[b] += count).
__global__ void k_phase_flips(const float *A, const float *B, long long Mb, float rho_mid, double *out)
{
    __shared__ double s1[256];
    const long long b = blockIdx.y;
    double a = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Mb; i += (long long)gridDim.x * blockDim.x) {
        const long long n = b * Mb + i;
        a += ((A[n] > rho_mid) != (B[n] > rho_mid)) ? 1.0 : 0.0;
    }
    s1[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) s1[threadIdx.x] += s1[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out + b, s1[0]);
}

__global__ void k_indicators(const float *F, long long M, long long Mb, float rho_mid, double *out, int *invalid)
{
    __shared__ double s1[256], s2[256];
    const long long b = blockIdx.y;
    double a1 = 0.0, a2 = 0.0;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Mb; i += (long long)gridDim.x * blockDim.x) {
        const long long n = b * Mb + i;
        const float r = F[n];
        a1 += r;
        a2 += r > rho_mid ? 1.0 : 0.0;
        if (invalid) {
            for (int c = 0; c < 4; ++c) bad |= !isfinite(F[c * M + n]);
            bad |= !(r > 0.f) || !(F[3 * M + n] > 0.f);
        }
    }
    if (bad) atomicOr(invalid, 1);
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            s1[threadIdx.x] += s1[threadIdx.x + s];
            s2[threadIdx.x] += s2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(out + 2 * b, s1[0]);
        atomicAdd(out + 2 * b + 1, s2[0]);
    }
}

// rho[b*Mb + i] -= delta[b]: restores each domain's mass (the lattice Boltzmann
// step conserves it exactly).
__global__ void k_shift_rho(float *rho, long long Mb, const float *delta)
{
    const long long b = blockIdx.y;
    const float d = delta[b];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Mb; i += (long long)gridDim.x * blockDim.x)
        rho[b * Mb + i] -= d;
}

}  // namespace

cudaError_t shift_rho(float *rho, int batch, long long Mb, const float *delta, cudaStream_t st)
{
    long long gx = (Mb + 255) / 256;
    if (gx > 64) gx = 64;
    k_shift_rho<<<dim3((unsigned)gx, (unsigned)batch), 256, 0, st>>>(rho, Mb, delta);
    return cudaGetLastError();
}

cudaError_t silu_bwd(const bf16 *dY, int ldd, const bf16 *Z, long long M, int lh, int lw, int C, bf16 *dZ,
                     float *dbias, cudaStream_t st)
{
    if (C % 8 || C / 8 > 32) return cudaErrorInvalidValue;
    k_silu_bwd<<<grid_red(M * C / 8), 256, 0, st>>>(dY, ldd, Z, M, lh, lw, C, dZ, dbias);
    return cudaGetLastError();
}

cudaError_t colsum(const bf16 *X, int ldx, long long M, int lh, int lw, int C, float *out, cudaStream_t st)
{
    if (C % 8 || C / 8 > 32 || ldx % 8 || (reinterpret_cast<uintptr_t>(X) & 15)) return cudaErrorInvalidValue;
    k_colsum<<<grid_red(M * C / 8), 256, 0, st>>>(X, ldx, M, lh, lw, C, out);
    return cudaGetLastError();
}

cudaError_t pool2(const bf16 *X, int ldx, long long Mc, int lh, int lw, int C, bf16 *Y, cudaStream_t st)
{
    k_pool2<<<grid_1d(Mc * C), 256, 0, st>>>(X, ldx, Mc, lh, lw, C, Y);
    return cudaGetLastError();
}

cudaError_t unpool2_acc(const bf16 *dY, long long Mc, int lh, int lw, int C, bf16 *dX, int ldx, cudaStream_t st)
{
    k_unpool2_acc<<<grid_1d(Mc * C), 256, 0, st>>>(dY, Mc, lh, lw, C, dX, ldx);
    return cudaGetLastError();
}

cudaError_t pack_in(const float *x, long long M, int lh, int lw, const float *norm, bf16 *X, cudaStream_t st)
{
    k_pack_in<<<grid_1d(M), 256, 0, st>>>(x, M, lh, lw, norm, X);
    return cudaGetLastError();
}

cudaError_t head(const bf16 *Y, long long M, int lh, int lw, const float *Wh, const float *bh, const float *norm,
                 const float *x, const float *yt, int mode, float *dO, float *loss, float *xn, cudaStream_t st)
{
    k_head<32><<<grid_1d(M), 256, 0, st>>>(Y, M, lh, lw, Wh, bh, norm, x, yt, mode, dO, loss, xn);
    return cudaGetLastError();
}

cudaError_t head_bwd(const bf16 *Y, long long M, int lh, int lw, const float *Wh, const float *dO, bf16 *dY,
                     float *dWh, float *dbh, cudaStream_t st)
{
    long long g = (M + 8 * 32 - 1) / (8 * 32);
    if (g > 2048) g = 2048;
    k_head_bwd<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(Y, M, lh, lw, Wh, dO, dY, dWh, dbh);
    return cudaGetLastError();
}

cudaError_t unroll_term(const float *xp, const float *yt, long long M, const float *norm, float inv, float *G, float *dO,
                        float *loss, cudaStream_t st)
{
    k_unroll_term<<<grid_1d(M), 256, 0, st>>>(xp, yt, M, norm, inv, G, dO, loss);
    return cudaGetLastError();
}

cudaError_t conv0_dx(const bf16 *dZ, const bf16 *Wb, int Kp, long long M, int lh, int lw, const float *norm, float *G,
                     cudaStream_t st)
{
    if (Kp < 72 || (reinterpret_cast<uintptr_t>(dZ) & 15)) return cudaErrorInvalidValue;
    k_conv0_dx<<<grid_1d(M), 256, 0, st>>>(dZ, Wb, Kp, M, lh, lw, norm, G);
    return cudaGetLastError();
}

cudaError_t adam(float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t st)
{
    k_adam<<<grid_1d(n), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t conv_weights(const float *Wt, int Cin, int Cout, int Kp, int Kpo, bf16 *Wb, bf16 *Wf, cudaStream_t st)
{
    k_conv_weights<<<grid_1d((long long)Cout * Kp), 256, 0, st>>>(Wt, Cin, Cout, Kp, Kpo, Wb, Wf);
    return cudaGetLastError();
}

cudaError_t up_weights(const float *Wm, int Cin, int Cout, bf16 *Wb, bf16 *Wt, cudaStream_t st)
{
    k_up_weights<<<grid_1d(4LL * Cout * Cin), 256, 0, st>>>(Wm, Cin, Cout, Wb, Wt);
    return cudaGetLastError();
}

cudaError_t indicators(const float *F, int batch, long long Mb, float rho_mid, double *out, int *invalid,
                       cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 2 * batch, st);
    if (e != cudaSuccess) return e;
    long long gx = (Mb + 255) / 256;
    if (gx > 64) gx = 64;
    const dim3 grid((unsigned)gx, (unsigned)batch);
    k_indicators<<<grid, 256, 0, st>>>(F, (long long)batch * Mb, Mb, rho_mid, out, invalid);
    return cudaGetLastError();
}

cudaError_t phase_flips(const float *A, const float *B, int batch, long long Mb, float rho_mid, double *out,
                        cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * batch, st);
    if (e != cudaSuccess) return e;
    long long gx = (Mb + 255) / 256;
    if (gx > 64) gx = 64;
    const dim3 grid((unsigned)gx, (unsigned)batch);
    k_phase_flips<<<grid, 256, 0, st>>>(A, B, Mb, rho_mid, out);
    return cudaGetLastError();
}

}  // namespace evsur

extern "C" int sur_indicators(const float *d_fields, int batch, int H, int W, float rho_mid, double *d_out,
                              void *stream)
{
    if (!d_fields || !d_out || batch < 1 || H < 1 || W < 1) return SUR_EINVAL;
    const cudaError_t e = evsur::indicators(d_fields, batch, (long long)H * W, rho_mid, d_out, nullptr,
                                            static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SUR_OK : SUR_ECUDA;
}

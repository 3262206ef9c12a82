/* Learned surrogate for the Enskog-Vlasov lattice Boltzmann step: C ABI.
 *
 * A 4-level convolutional U-Net maps the macroscopic fields (rho, u_x, u_y, T)
 * of 2-D periodic domains to their state one window of lattice Boltzmann steps
 * later (it predicts the increment).  The lattice Boltzmann method of the paper
 * (Sec. 3, Eqs. for the moments, the shifted equilibria and the relaxation,
 * implemented in evlbm.h) generates its training data, is its fallback and
 * is the reference its error is measured against; the paper itself has no learned
 * component, so nothing in this header restates a passage of it beyond that.
 *
 * Arithmetic: BF16 weights and activations, FP32 accumulation on the tensor
 * cores (tcgen05.mma kind::f16), FP32 master weights, gradients and Adam
 * moments.  Activations are NHWC matrices [pixels][channels] with pixels
 * ordered (sample, y, x), x fastest.
 *
 * Pointers named d_* are device pointers owned by the caller; host arrays are
 * named h_* or documented as host.  All calls run on the stream given at
 * creation (NULL = a stream the model creates) and are asynchronous unless
 * they return a host value.  Errors: SUR_EINVAL for invalid sizes, layouts or
 * NULL arguments (nothing is launched), SUR_ECUDA for a CUDA runtime error,
 * SUR_ETIMEOUT when a tensor-core wait gave up (the result is then invalid;
 * the context stays usable), SUR_ENOMEM for a failed allocation.
 */
#ifndef EVSUR_H
#define EVSUR_H

#include <stdint.h>

#include "evlbm.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { SUR_OK = 0, SUR_EINVAL = 1, SUR_ECUDA = 2, SUR_ENOMEM = 3, SUR_ETIMEOUT = 4, SUR_EUNPHYSICAL = 5 };

/* ---------------------------------------------------------------------------
 * Layer primitives (exposed for testing and for callers that build their own
 * networks).  All matrices are BF16 unless stated.
 * ------------------------------------------------------------------------- */

/* Halo-padded NHWC storage.  A tensor of B images on an H x W periodic grid
 * (H, W powers of two) is stored as [B][H+2][W+2][ld] BF16: interior pixel
 * (b, y, x) at [b][y+1][x+1]; rows 0 and H+1 and columns 0 and W+1 hold the
 * periodic copies of rows H-1, 0 and columns W-1, 0.  Pixel index
 * q = (b*H + y)*W + x counts interior pixels; pix(q) is its stored position.
 *
 * Operand kinds of the tensor-core GEMM C[m][n] = sum_k A(m, k) B(n, k):
 *
 *  SUR_OP_DENSE   X(r, k) = p[r*ld + c0 + k]                   (row-major matrix)
 *  SUR_OP_PIX     X(r, k) = p[pix(r)*ld + c0 + k],  k < C       (pixel rows)
 *  SUR_OP_CONV3   X(r, k) = p[(pix(r) + dy*(W+2) + dx)*ld + c0 + c]  with
 *                 k = tap*C + c, tap = (dy+1)*3 + (dx+1); k >= 9C reads 0
 *                 (implicit im2col of a periodic 3x3 convolution)
 *  SUR_OP_UPADJ   X(r, k) = p[fine(r, s)*ld + c0 + c]  with k = s*C + c, r an
 *                 interior pixel of the coarse H x W grid, fine(r, s) the stored
 *                 position of its child (2y + s/2, 2x + s%2) on the padded
 *                 2H x 2W grid; k >= 4C reads 0
 *  SUR_OP_TPIX    X(r, k) = p[pix(k)*ld + c0 + r]               (pixels along K)
 *  SUR_OP_TCONV3  X(r, k) = p[(pix(k) + dy*(W+2) + dx)*ld + c0 + c],  r = tap*C + c
 *  SUR_OP_TUP     X(r, k) = p[fine(k, s)*ld + c0 + c],  r = s*C + c
 *
 * Rows r >= rows and K indices k >= K read zero.  C >= 8 is a power of two; ld
 * and c0 are multiples of 8 elements and p is 16-byte aligned.  Memory is read
 * in 8-element chunks: a DENSE operand needs c0 + K rounded up to 8 <= ld, a
 * TPIX operand c0 + rows rounded up to 8 <= ld, and the other kinds
 * c0 + C <= ld (SUR_EINVAL otherwise). */
enum {
    SUR_OP_DENSE = 0, SUR_OP_PIX = 1, SUR_OP_CONV3 = 2, SUR_OP_UPADJ = 3,
    SUR_OP_TPIX = 4, SUR_OP_TCONV3 = 5, SUR_OP_TUP = 6
};

typedef struct sur_operand {
    const void *p; /* device, BF16 */
    int kind;      /* SUR_OP_* */
    int ld, c0;    /* row stride and first column, elements */
    int C;         /* channels of the gathered tensor (gather kinds) */
    int rows;      /* valid rows of the operand */
    int H, W;      /* pixel grid of the gather kinds (coarse grid for UPADJ/TUP) */
} sur_operand;

/* Epilogues.  acc is the FP32 accumulator of C[m][n]; bias (FP32, may be NULL
 * except for SUR_EPI_CONV and SUR_EPI_SHUF) is indexed by n (by n % cout for SHUF).
 * When A's rows are pixels (PIX, CONV3, UPADJ) the output rows are pixels of
 * A's grid and row m is stored at pix(m) of a halo-padded output; otherwise at m.
 *  SUR_EPI_BF16        out[row(m)*ldo + co0 + n] = bf16(acc + bias)
 *  SUR_EPI_F32         out[row(m)*ldo + co0 + n] = acc + bias        (FP32 out)
 *  SUR_EPI_F32_ATOMIC  out[m*ldo + co0 + n] += acc                   (FP32 out, split-K)
 *  SUR_EPI_CONV        z = acc + bias; out[row(m)...] = bf16(z) (skipped when out is
 *                      NULL); y[...*ldy + cy0 + n] = bf16(silu(z)), silu(z) = z/(1+e^-z),
 *                      written at pix(m) and at its periodic halo copies
 *  SUR_EPI_SHUF        2x2 stride-2 transposed convolution (A's rows are pixels of
 *                      the coarse grid): n = s*cout + c, y at the child s of m on
 *                      the padded 2H x 2W grid (and its halo copies):
 *                      bf16(acc + bias[c]). */
enum { SUR_EPI_BF16 = 0, SUR_EPI_F32 = 1, SUR_EPI_F32_ATOMIC = 2, SUR_EPI_CONV = 3, SUR_EPI_SHUF = 4 };

typedef struct sur_gemm_args {
    sur_operand a, b;
    int M, N, K;       /* output rows (any >= 1), columns (multiple of 32), reduction length (>= 1) */
    int splits;        /* K split across CTAs (>= 1; > 1 only with SUR_EPI_F32_ATOMIC) */
    int epi;           /* SUR_EPI_* */
    const float *bias;
    void *out;         /* BF16 or FP32 per epi */
    int ldo, co0;
    void *y;           /* BF16, SUR_EPI_CONV / SUR_EPI_SHUF */
    int ldy, cy0;
    int shuf_cout;
} sur_gemm_args;

/* One GEMM on the tensor cores (128 x {32,64,128} CTA tiles, 64-deep K blocks,
 * one thread issuing tcgen05.mma into a TMEM accumulator).  A CONV3 or PIX A
 * operand with a DENSE B operand and no split is fed by TMA (swizzled
 * cp.async.bulk.tensor boxes); every other form by a cp.async pipeline.
 * d_status (device int) is set to 1 if a wait gave up. */
int sur_gemm(const sur_gemm_args *g, int *d_status, void *stream);

/* 0 routes every GEMM through the cp.async pipeline (for testing both paths);
 * 1 (the default) lets eligible GEMMs use TMA.  Process-wide. */
int sur_set_tma(int enable);

/* ---------------------------------------------------------------------------
 * The model.
 * ------------------------------------------------------------------------- */
typedef struct sur_model sur_model;

/* Architecture (fixed): input 4 channels zero-padded to 8; levels of widths
 * base, 2 base, 4 base, 8 base (base = 32); two 3x3 periodic convolutions with
 * bias and SiLU per level; 2x2 average pooling down; 2x2 stride-2 transposed
 * convolutions with bias up, concatenated after the skip tensor; a 1x1 head to
 * 4 channels.  H and W are powers of two >= 16.
 *
 * Parameters (FP32, canonical order, packed without gaps):
 *   14 convolutions in execution order c00 c01 c10 c11 c20 c21 c30 c31 c22 c23
 *   c12 c13 c02 c03, each W [Kp][Cout] with row tap*Cin + ci (Kp = 9 Cin rounded
 *   up to a multiple of 64, rows >= 9 Cin zero) followed by bias [Cout];
 *   3 transposed convolutions u2 u1 u0, each W [4 Cout][Cin] with row s*Cout + co,
 *   s = 2 di + dj the child offset, followed by bias [Cout];
 *   the head W [4][base] and bias [4].
 * Initialised with uniform(-sqrt(6/fan_in), sqrt(6/fan_in)) weights from a
 * splitmix64 stream of seed, zero biases, and zero weights on padded inputs. */
int sur_init(int H, int W, int base_ch, uint64_t seed, void *stream, sur_model **out);
int sur_free(sur_model *m);                                      /* NULL-safe */
long long sur_num_params(const sur_model *m);
int sur_get_params(sur_model *m, float *h_params, long long n);  /* synchronises */
int sur_set_params(sur_model *m, const float *h_params, long long n);
int sur_get_grads(sur_model *m, float *h_grads, long long n);    /* gradients of the last forward_backward */

/* Normalisation: the network sees (x_c - in_mean[c]) / in_scale[c] and its
 * output o_c means an increment out_scale[c] * o_c of field c (host arrays of 4). */
int sur_set_norm(sur_model *m, const float *in_mean, const float *in_scale, const float *out_scale);

/* Fields are FP32 planar device arrays [4][batch*H*W]: rho, u_x, u_y, T.
 * forward_backward: loss = mean over pixels and channels of
 * (o - (y - x)/out_scale)^2; gradients of it (overwritten) into the model.
 * train_step: forward_backward then one Adam step (lr, beta1 0.9, beta2 0.999,
 * eps 1e-8, bias-corrected).  loss (host, may be NULL) synchronises. */
int sur_forward_backward(sur_model *m, const float *d_x, const float *d_y, int batch, float *loss);
int sur_train_step(sur_model *m, const float *d_x, const float *d_y, int batch, float lr, float *loss);
/* Unrolled training over `windows` = k consecutive windows: the network is applied to
 * its own prediction, x'_0 = d_x0, x'_{j+1} = x'_j + out_scale * o(x'_j), and
 *   loss = (1/k) sum_{j=1..k} mean over pixels and channels of ((x'_j - y_j)/out_scale)^2
 * with the targets y_j = d_targets + (j - 1) * 4 * batch*H*W (planar [k][4][batch*H*W]);
 * k = 1 is the loss of sur_forward_backward.  Gradients (overwritten) flow through the
 * whole chain, predictions included.  The predictions are kept (an internal buffer of
 * (k + 1) * 4 * batch*H*W floats, grown as needed), the activations of one window at a
 * time: each window's forward pass runs twice.  1 <= k <= 64.  train_step_unrolled adds
 * the Adam step of sur_train_step.  loss (host, may be NULL) synchronises. */
int sur_forward_backward_unrolled(sur_model *m, const float *d_x0, const float *d_targets, int windows, int batch,
                                  float *loss);
int sur_train_step_unrolled(sur_model *m, const float *d_x0, const float *d_targets, int windows, int batch, float lr,
                            float *loss);
/* d_y = x + out_scale * o (d_y may equal d_x). */
int sur_infer(sur_model *m, const float *d_x, float *d_y, int batch);

/* Per-domain indicators (FP64 sums over each H x W domain of a planar field
 * array): d_out[2 b] = sum rho, d_out[2 b + 1] = number of nodes with
 * rho > rho_mid. */
int sur_indicators(const float *d_fields, int batch, int H, int W, float rho_mid, double *d_out, void *stream);

/* Rollout of `windows` windows of `steps` lattice steps each on the fields
 * d_fields (in/out).  Each window the surrogate proposes the next state.  With
 * project_mass != 0 the proposal's density is shifted per domain so that each
 * domain keeps the mass it had at the start of the rollout (the lattice
 * Boltzmann step conserves mass exactly).  The proposal is discarded if, for
 * any domain, a field is not finite or rho or T is not positive, the mass
 * differs from the start by more than max_mass_drift (relative), or the liquid
 * node count (rho > rho_mid) differs from the previous window's by more than
 * max_area_change (relative), or more than a fraction max_interface_shift of the
 * domain's nodes change phase (rho above / below rho_mid) against the current
 * fields -- an interface-position indicator, which also sees interfaces that move
 * without changing the liquid count (1 or more: off); the window is then advanced
 * by the lattice
 * Boltzmann context lb instead (nz = batch layers of H x W, D2Q9, not FP64).
 * The first fallback window and every fallback window that follows an accepted
 * surrogate window restart lb from the local equilibrium of the current fields
 * (lbm_reset_device); consecutive fallback windows continue the lattice
 * Boltzmann state, so a rollout in which every window falls back is exactly a
 * plain lattice Boltzmann run from the equilibrium of the start fields.
 * h_used_lb (host, windows entries, may be NULL) records 1 for fallback
 * windows; *n_fallback (host) counts them.  SUR_EUNPHYSICAL if a lattice
 * Boltzmann window itself ends non-finite or non-positive (the fields then hold
 * that state).  Synchronises once or twice per window. */
typedef struct sur_rollout_cfg {
    int windows, steps;
    float rho_mid, max_mass_drift, max_area_change;
    int project_mass;
    float max_interface_shift;
} sur_rollout_cfg;
int sur_rollout(sur_model *m, lbm_ctx *lb, float *d_fields, int batch, const sur_rollout_cfg *cfg,
                unsigned char *h_used_lb, int *n_fallback);

/* Description of the last error of this model (static string storage). */
const char *sur_last_error(const sur_model *m);

#ifdef __cplusplus
}
#endif

#endif

// U-Net runtime of the learned surrogate: parameters, activation arena,
// forward, backward, Adam, inference and the rollout with lattice Boltzmann
// fallback.  Every arithmetic step runs in the kernels of surrogate.cu (and,
// for the fallback, in the lattice Boltzmann library).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "surrogate.cuh"
#include "trace.h"

using evsur::bf16;

namespace {

constexpr int kConvs = 14, kUps = 3, kBase = 32;
// Execution order c00 c01 c10 c11 c20 c21 c30 c31 c22 c23 c12 c13 c02 c03 (in, out channels).
constexpr int kConvIO[kConvs][2] = {{8, 32},   {32, 32},   {32, 64},   {64, 64},   {64, 128},
                                    {128, 128}, {128, 256}, {256, 256}, {256, 128}, {128, 128},
                                    {128, 64},  {64, 64},   {64, 32},   {32, 32}};
constexpr int kConvLevel[kConvs] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0};
// u2 u1 u0: (in, out channels); coarse level of the input.
constexpr int kUpIO[kUps][2] = {{256, 128}, {128, 64}, {64, 32}};
constexpr int kUpLevel[kUps] = {3, 2, 1};

struct ConvL {
    int cin, cout, kp, kpo;
    long long w, b;   // offsets into the parameter arrays
    bf16 *wb, *wf;
};
struct UpL {
    int cin, cout;
    long long w, b;
    bf16 *wb, *wt;
};

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

struct sur_model {
    int H, W, lh, lw;
    cudaStream_t stream;
    bool own_stream;
    ConvL conv[kConvs];
    UpL up[kUps];
    long long head_w, head_b, nparam;
    float *P, *G, *Mo, *Vo;   // FP32 master weights, gradients, Adam moments
    bf16 *wpool;
    float *norm;              // in_mean[4], in_scale[4], out_scale[4]
    int *status;              // [0] tensor-core wait status, [1] non-finite flag
    float *loss;
    double *ind;              // indicators, 2 per domain
    float *ubuf;              // unrolled training: field gradient and the k predicted states
    long long ucap;           // floats in ubuf
    int adam_t;
    // Activation arena for `cap` samples.
    int cap;
    void *arena;
    bool train_buffers;
    bf16 *xin, *Z[kConvs];
    bf16 *Y00, *cat0, *p0, *Y10, *cat1, *p1, *Y20, *cat2, *p2, *Y30, *Y31, *Y22, *Y23, *Y12, *Y13, *Y02, *Y03;
    float *dO, *next;
    bf16 *dZ, *dY03, *dY02, *dcat0, *dY13, *dY12, *dcat1, *dY23, *dY22, *dcat2, *dY31, *dY30, *dp2, *dY20, *dp1, *dY10,
        *dp0, *dY00;
    char err[256];
};

namespace {

int fail(sur_model *m, int code, const char *fmt, ...)
{
    if (m) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(m->err, sizeof(m->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(sur_model *m, cudaError_t e, const char *where)
{
    return fail(m, SUR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(expr)                                                    \
    do {                                                            \
        cudaError_t e_ = (expr);                                    \
        if (e_ != cudaSuccess) return cuda_fail(m, e_, #expr);      \
    } while (0)
#define CKS(expr)                                                   \
    do {                                                            \
        int r_ = (expr);                                            \
        if (r_ != SUR_OK) return fail(m, r_, "%s failed (%d)", #expr, r_); \
    } while (0)

int lvl_h(const sur_model *m, int l) { return m->H >> l; }
int lvl_w(const sur_model *m, int l) { return m->W >> l; }
long long lvl_pix(const sur_model *m, int l, int B) { return (long long)B * lvl_h(m, l) * lvl_w(m, l); }
// Stored (halo-padded) pixel count of level l.
long long lvl_pad(const sur_model *m, int l, int B) { return (long long)B * (lvl_h(m, l) + 2) * (lvl_w(m, l) + 2); }
int lvl_lh(const sur_model *m, int l) { return m->lh - l; }
int lvl_lw(const sur_model *m, int l) { return m->lw - l; }

sur_operand dense(const void *p, int ld, int c0, long long rows)
{
    sur_operand o{};
    o.p = p;
    o.kind = SUR_OP_DENSE;
    o.ld = ld;
    o.c0 = c0;
    o.rows = (int)rows;
    return o;
}

sur_operand gather(int kind, const void *p, int ld, int c0, int C, long long rows, int H, int W)
{
    sur_operand o{};
    o.p = p;
    o.kind = kind;
    o.ld = ld;
    o.c0 = c0;
    o.C = C;
    o.rows = (int)rows;
    o.H = H;
    o.W = W;
    return o;
}

// Split-K count for a weight-gradient GEMM: about four CTAs per SM in total,
// at least 8 K blocks of 64 per split.
int pick_splits(long long mrows, int n, long long K)
{
    const int bn = n % 128 == 0 ? 128 : (n % 64 == 0 ? 64 : 32);
    const long long tiles = ((mrows + 127) / 128) * (n / bn);
    long long s = (4 * 152 + tiles - 1) / tiles;
    const long long kb = (K + 63) / 64;
    if (s > kb / 8) s = kb / 8;
    if (s < 1) s = 1;
    return (int)s;
}

int conv_fwd(sur_model *m, int i, int B, const bf16 *X, int ldx, bf16 *Y, int ldy, int cy0, bool train)
{
    const ConvL &L = m->conv[i];
    const int l = kConvLevel[i];
    const long long M = lvl_pix(m, l, B);
    sur_gemm_args g{};
    g.a = gather(SUR_OP_CONV3, X, ldx, 0, L.cin, M, lvl_h(m, l), lvl_w(m, l));
    g.b = dense(L.wb, L.kp, 0, L.cout);
    g.M = (int)M;
    g.N = L.cout;
    g.K = L.kp;
    g.splits = 1;
    g.epi = SUR_EPI_CONV;
    g.bias = m->P + L.b;
    g.out = train ? m->Z[i] : nullptr;
    g.ldo = L.cout;
    g.y = Y;
    g.ldy = ldy;
    g.cy0 = cy0;
    return evsur::gemm(g, m->status, m->stream);
}

int up_fwd(sur_model *m, int j, int B, const bf16 *Xc, bf16 *cat)
{
    const UpL &U = m->up[j];
    const int l = kUpLevel[j];
    const long long Mc = lvl_pix(m, l, B);
    sur_gemm_args g{};
    g.a = gather(SUR_OP_PIX, Xc, U.cin, 0, U.cin, Mc, lvl_h(m, l), lvl_w(m, l));
    g.b = dense(U.wb, U.cin, 0, 4 * U.cout);
    g.M = (int)Mc;
    g.N = 4 * U.cout;
    g.K = U.cin;
    g.splits = 1;
    g.epi = SUR_EPI_SHUF;
    g.bias = m->P + U.b;
    g.y = cat;
    g.ldy = 2 * U.cout;
    g.cy0 = U.cout;
    g.shuf_cout = U.cout;
    return evsur::gemm(g, m->status, m->stream);
}

// dY (ld ldd) -> dZ; bias and weight gradients; dX (ld ldx, may be NULL).
int conv_bwd(sur_model *m, int i, int B, const bf16 *X, int ldx, const bf16 *dY, int ldd, bf16 *dX, int ldxo)
{
    const ConvL &L = m->conv[i];
    const int l = kConvLevel[i];
    const long long M = lvl_pix(m, l, B);
    const int H = lvl_h(m, l), W = lvl_w(m, l);
    // dZ and, in the same pass, the bias gradient (its column sums).
    CK(evsur::silu_bwd(dY, ldd, m->Z[i], M, lvl_lh(m, l), lvl_lw(m, l), L.cout, m->dZ, m->G + L.b, m->stream));
    sur_gemm_args g{};
    g.a = gather(SUR_OP_TCONV3, X, ldx, 0, L.cin, 9LL * L.cin, H, W);
    g.b = gather(SUR_OP_TPIX, m->dZ, L.cout, 0, 0, L.cout, H, W);
    g.M = L.kp;
    g.N = L.cout;
    g.K = (int)M;
    g.splits = pick_splits(L.kp, L.cout, M);
    g.epi = SUR_EPI_F32_ATOMIC;
    g.out = m->G + L.w;
    g.ldo = L.cout;
    int rc = evsur::gemm(g, m->status, m->stream);
    if (rc) return fail(m, rc, "weight-gradient GEMM of convolution %d", i);
    if (!dX) return SUR_OK;
    sur_gemm_args d{};
    d.a = gather(SUR_OP_CONV3, m->dZ, L.cout, 0, L.cout, M, H, W);
    d.b = dense(L.wf, L.kpo, 0, L.cin);
    d.M = (int)M;
    d.N = L.cin;
    d.K = L.kpo;
    d.splits = 1;
    d.epi = SUR_EPI_BF16;
    d.out = dX;
    d.ldo = ldxo;
    rc = evsur::gemm(d, m->status, m->stream);
    if (rc) return fail(m, rc, "input-gradient GEMM of convolution %d", i);
    return SUR_OK;
}

// Transposed convolution j: coarse input Xc [Mc][cin]; gradient of the fine
// output in dcat (ld 2 cout, columns cout..2cout-1); dXc [Mc][cin].
int up_bwd(sur_model *m, int j, int B, const bf16 *Xc, const bf16 *dcat, bf16 *dXc)
{
    const UpL &U = m->up[j];
    const int l = kUpLevel[j];
    const long long Mc = lvl_pix(m, l, B);
    const int H = lvl_h(m, l), W = lvl_w(m, l);
    CK(evsur::colsum(dcat + U.cout, 2 * U.cout, 4 * Mc, lvl_lh(m, l - 1), lvl_lw(m, l - 1), U.cout, m->G + U.b,
                     m->stream));
    sur_gemm_args g{};
    g.a = gather(SUR_OP_TUP, dcat, 2 * U.cout, U.cout, U.cout, 4LL * U.cout, H, W);
    g.b = gather(SUR_OP_TPIX, Xc, U.cin, 0, 0, U.cin, H, W);
    g.M = 4 * U.cout;
    g.N = U.cin;
    g.K = (int)Mc;
    g.splits = pick_splits(4 * U.cout, U.cin, Mc);
    g.epi = SUR_EPI_F32_ATOMIC;
    g.out = m->G + U.w;
    g.ldo = U.cin;
    int rc = evsur::gemm(g, m->status, m->stream);
    if (rc) return fail(m, rc, "weight-gradient GEMM of transposed convolution %d", j);
    sur_gemm_args d{};
    d.a = gather(SUR_OP_UPADJ, dcat, 2 * U.cout, U.cout, U.cout, Mc, H, W);
    d.b = dense(U.wt, 4 * U.cout, 0, U.cin);
    d.M = (int)Mc;
    d.N = U.cin;
    d.K = 4 * U.cout;
    d.splits = 1;
    d.epi = SUR_EPI_BF16;
    d.out = dXc;
    d.ldo = U.cin;
    rc = evsur::gemm(d, m->status, m->stream);
    if (rc) return fail(m, rc, "input-gradient GEMM of transposed convolution %d", j);
    return SUR_OK;
}

int refresh_weights(sur_model *m)
{
    for (int i = 0; i < kConvs; ++i) {
        const ConvL &L = m->conv[i];
        CK(evsur::conv_weights(m->P + L.w, L.cin, L.cout, L.kp, L.kpo, L.wb, L.wf, m->stream));
    }
    for (int j = 0; j < kUps; ++j) {
        const UpL &U = m->up[j];
        CK(evsur::up_weights(m->P + U.w, U.cin, U.cout, U.wb, U.wt, m->stream));
    }
    return SUR_OK;
}

// Carve the activation arena for B samples (train adds the saved pre-activations
// and the gradient buffers).
int ensure_batch(sur_model *m, int B, bool train)
{
    if (B <= m->cap && (!train || m->train_buffers)) return SUR_OK;
    if (m->arena) {
        CK(cudaStreamSynchronize(m->stream));
        cudaFree(m->arena);
        m->arena = nullptr;
        m->cap = 0;
    }
    // NHWC tensors are stored halo-padded; the planar FP32 fields are not.
    const long long M0 = lvl_pad(m, 0, B), M1 = lvl_pad(m, 1, B), M2 = lvl_pad(m, 2, B), M3 = lvl_pad(m, 3, B);
    const long long F0 = lvl_pix(m, 0, B);
    struct Req {
        void **dst;
        long long bytes;
    };
    std::vector<Req> req;
    auto bf = [&](bf16 **p, long long elems) { req.push_back({reinterpret_cast<void **>(p), 2 * elems}); };
    auto fl = [&](float **p, long long elems) { req.push_back({reinterpret_cast<void **>(p), 4 * elems}); };
    bf(&m->xin, M0 * 8);
    bf(&m->Y00, M0 * 32);
    bf(&m->cat0, M0 * 64);
    bf(&m->p0, M1 * 32);
    bf(&m->Y10, M1 * 64);
    bf(&m->cat1, M1 * 128);
    bf(&m->p1, M2 * 64);
    bf(&m->Y20, M2 * 128);
    bf(&m->cat2, M2 * 256);
    bf(&m->p2, M3 * 128);
    bf(&m->Y30, M3 * 256);
    bf(&m->Y31, M3 * 256);
    bf(&m->Y22, M2 * 128);
    bf(&m->Y23, M2 * 128);
    bf(&m->Y12, M1 * 64);
    bf(&m->Y13, M1 * 64);
    bf(&m->Y02, M0 * 32);
    bf(&m->Y03, M0 * 32);
    fl(&m->next, 4 * F0);
    if (train) {
        for (int i = 0; i < kConvs; ++i) bf(&m->Z[i], lvl_pad(m, kConvLevel[i], B) * m->conv[i].cout);
        fl(&m->dO, 4 * F0);
        bf(&m->dZ, M0 * 32);
        bf(&m->dY03, M0 * 32);
        bf(&m->dY02, M0 * 32);
        bf(&m->dcat0, M0 * 64);
        bf(&m->dY13, M1 * 64);
        bf(&m->dY12, M1 * 64);
        bf(&m->dcat1, M1 * 128);
        bf(&m->dY23, M2 * 128);
        bf(&m->dY22, M2 * 128);
        bf(&m->dcat2, M2 * 256);
        bf(&m->dY31, M3 * 256);
        bf(&m->dY30, M3 * 256);
        bf(&m->dp2, M3 * 128);
        bf(&m->dY20, M2 * 128);
        bf(&m->dp1, M2 * 64);
        bf(&m->dY10, M1 * 64);
        bf(&m->dp0, M1 * 32);
        bf(&m->dY00, M0 * 32);
    }
    long long total = 0;
    for (const Req &r : req) total += round_up(r.bytes, 256);
    void *arena = nullptr;
    cudaError_t e = cudaMalloc(&arena, (size_t)total);
    if (e != cudaSuccess) return fail(m, SUR_ENOMEM, "activation arena of %lld bytes: %s", total, cudaGetErrorString(e));
    char *p = static_cast<char *>(arena);
    for (const Req &r : req) {
        *r.dst = p;
        p += round_up(r.bytes, 256);
    }
    m->arena = arena;
    m->cap = B;
    m->train_buffers = train;
    return SUR_OK;
}

int forward(sur_model *m, const float *d_x, int B, bool train)
{
    const long long M0 = lvl_pix(m, 0, B);
    CK(evsur::pack_in(d_x, M0, m->lh, m->lw, m->norm, m->xin, m->stream));
    int rc;
#define F(expr)                  \
    if ((rc = (expr)) != SUR_OK) \
        return fail(m, rc, "forward: %s", #expr);
    F(conv_fwd(m, 0, B, m->xin, 8, m->Y00, 32, 0, train));
    F(conv_fwd(m, 1, B, m->Y00, 32, m->cat0, 64, 0, train));
    CK(evsur::pool2(m->cat0, 64, lvl_pix(m, 1, B), m->lh - 1, m->lw - 1, 32, m->p0, m->stream));
    F(conv_fwd(m, 2, B, m->p0, 32, m->Y10, 64, 0, train));
    F(conv_fwd(m, 3, B, m->Y10, 64, m->cat1, 128, 0, train));
    CK(evsur::pool2(m->cat1, 128, lvl_pix(m, 2, B), m->lh - 2, m->lw - 2, 64, m->p1, m->stream));
    F(conv_fwd(m, 4, B, m->p1, 64, m->Y20, 128, 0, train));
    F(conv_fwd(m, 5, B, m->Y20, 128, m->cat2, 256, 0, train));
    CK(evsur::pool2(m->cat2, 256, lvl_pix(m, 3, B), m->lh - 3, m->lw - 3, 128, m->p2, m->stream));
    F(conv_fwd(m, 6, B, m->p2, 128, m->Y30, 256, 0, train));
    F(conv_fwd(m, 7, B, m->Y30, 256, m->Y31, 256, 0, train));
    F(up_fwd(m, 0, B, m->Y31, m->cat2));
    F(conv_fwd(m, 8, B, m->cat2, 256, m->Y22, 128, 0, train));
    F(conv_fwd(m, 9, B, m->Y22, 128, m->Y23, 128, 0, train));
    F(up_fwd(m, 1, B, m->Y23, m->cat1));
    F(conv_fwd(m, 10, B, m->cat1, 128, m->Y12, 64, 0, train));
    F(conv_fwd(m, 11, B, m->Y12, 64, m->Y13, 64, 0, train));
    F(up_fwd(m, 2, B, m->Y13, m->cat0));
    F(conv_fwd(m, 12, B, m->cat0, 64, m->Y02, 32, 0, train));
    F(conv_fwd(m, 13, B, m->Y02, 32, m->Y03, 32, 0, train));
#undef F
    (void)M0;
    return SUR_OK;
}

int backward(sur_model *m, int B)
{
    const long long M0 = lvl_pix(m, 0, B);
    CK(evsur::head_bwd(m->Y03, M0, m->lh, m->lw, m->P + m->head_w, m->dO, m->dY03, m->G + m->head_w, m->G + m->head_b, m->stream));
    int rc;
#define BW(expr)                 \
    if ((rc = (expr)) != SUR_OK) \
        return rc;
    BW(conv_bwd(m, 13, B, m->Y02, 32, m->dY03, 32, m->dY02, 32));
    BW(conv_bwd(m, 12, B, m->cat0, 64, m->dY02, 32, m->dcat0, 64));
    BW(up_bwd(m, 2, B, m->Y13, m->dcat0, m->dY13));
    BW(conv_bwd(m, 11, B, m->Y12, 64, m->dY13, 64, m->dY12, 64));
    BW(conv_bwd(m, 10, B, m->cat1, 128, m->dY12, 64, m->dcat1, 128));
    BW(up_bwd(m, 1, B, m->Y23, m->dcat1, m->dY23));
    BW(conv_bwd(m, 9, B, m->Y22, 128, m->dY23, 128, m->dY22, 128));
    BW(conv_bwd(m, 8, B, m->cat2, 256, m->dY22, 128, m->dcat2, 256));
    BW(up_bwd(m, 0, B, m->Y31, m->dcat2, m->dY31));
    BW(conv_bwd(m, 7, B, m->Y30, 256, m->dY31, 256, m->dY30, 256));
    BW(conv_bwd(m, 6, B, m->p2, 128, m->dY30, 256, m->dp2, 128));
    CK(evsur::unpool2_acc(m->dp2, lvl_pix(m, 3, B), m->lh - 3, m->lw - 3, 128, m->dcat2, 256, m->stream));
    BW(conv_bwd(m, 5, B, m->Y20, 128, m->dcat2, 256, m->dY20, 128));
    BW(conv_bwd(m, 4, B, m->p1, 64, m->dY20, 128, m->dp1, 64));
    CK(evsur::unpool2_acc(m->dp1, lvl_pix(m, 2, B), m->lh - 2, m->lw - 2, 64, m->dcat1, 128, m->stream));
    BW(conv_bwd(m, 3, B, m->Y10, 64, m->dcat1, 128, m->dY10, 64));
    BW(conv_bwd(m, 2, B, m->p0, 32, m->dY10, 64, m->dp0, 32));
    CK(evsur::unpool2_acc(m->dp0, lvl_pix(m, 1, B), m->lh - 1, m->lw - 1, 32, m->dcat0, 64, m->stream));
    BW(conv_bwd(m, 1, B, m->Y00, 32, m->dcat0, 64, m->dY00, 32));
    BW(conv_bwd(m, 0, B, m->xin, 8, m->dY00, 32, nullptr, 0));
#undef BW
    return SUR_OK;
}

// Read and clear the status words; SUR_ETIMEOUT if a tensor-core wait gave up.
int check_status(sur_model *m, int *nonfinite)
{
    int h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, m->status, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    if (h[0] || h[1]) CK(cudaMemsetAsync(m->status, 0, sizeof(h), m->stream));
    if (nonfinite) *nonfinite = h[1];
    if (h[0]) return fail(m, SUR_ETIMEOUT, "a tensor-core wait gave up; results of this call are invalid");
    return SUR_OK;
}

int fwd_bwd(sur_model *m, const float *d_x, const float *d_y, int B, float *loss)
{
    if (!m || !d_x || !d_y || B < 1) return fail(m, SUR_EINVAL, "invalid arguments");
    int rc = ensure_batch(m, B, true);
    if (rc) return rc;
    CK(cudaMemsetAsync(m->G, 0, sizeof(float) * m->nparam, m->stream));
    CK(cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
    if ((rc = forward(m, d_x, B, true))) return rc;
    const long long M0 = lvl_pix(m, 0, B);
    CK(evsur::head(m->Y03, M0, m->lh, m->lw, m->P + m->head_w, m->P + m->head_b, m->norm, d_x, d_y, 0, m->dO, m->loss, nullptr,
                   m->stream));
    if ((rc = backward(m, B))) return rc;
    if (loss) {
        CK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        return check_status(m, nullptr);
    }
    return SUR_OK;
}

// Loss and gradients of `k` windows chained through the network (unrolled training):
// x'_0 = d_x0, x'_{j+1} = x'_j + out_scale o(x'_j), L = (1/k) sum_j mean ((x'_j - y_j) /
// out_scale)^2 with the targets y_j = d_targets[j - 1].  The predictions are kept, the
// activations are not: the backward pass runs j = k .. 1, each time recomputing the
// forward pass of window j - 1, and carries dL/dx'_j (loss term + identity path + the
// network path through the first convolution's input gradient) down the chain.
int fwd_bwd_unrolled(sur_model *m, const float *d_x0, const float *d_targets, int k, int B, float *loss)
{
    if (!m || !d_x0 || !d_targets || B < 1 || k < 1 || k > 64) return fail(m, SUR_EINVAL, "invalid arguments");
    int rc = ensure_batch(m, B, true);
    if (rc) return rc;
    const long long M0 = lvl_pix(m, 0, B), F = 4 * M0;
    const long long need = (long long)(k + 1) * F;
    if (need > m->ucap) {
        if (m->ubuf) {
            CK(cudaStreamSynchronize(m->stream));
            cudaFree(m->ubuf);
            m->ubuf = nullptr;
            m->ucap = 0;
        }
        cudaError_t e = cudaMalloc(&m->ubuf, sizeof(float) * need);
        if (e != cudaSuccess) return fail(m, SUR_ENOMEM, "unrolled buffers of %lld floats: %s", need, cudaGetErrorString(e));
        m->ucap = need;
    }
    float *Gx = m->ubuf;
    auto state = [&](int j) { return j == 0 ? const_cast<float *>(d_x0) : m->ubuf + (long long)j * F; };
    CK(cudaMemsetAsync(m->G, 0, sizeof(float) * m->nparam, m->stream));
    CK(cudaMemsetAsync(m->loss, 0, sizeof(float), m->stream));
    CK(cudaMemsetAsync(Gx, 0, sizeof(float) * F, m->stream));
    for (int j = 0; j < k; ++j) {
        if ((rc = forward(m, state(j), B, false))) return rc;
        CK(evsur::head(m->Y03, M0, m->lh, m->lw, m->P + m->head_w, m->P + m->head_b, m->norm, state(j), nullptr, 1,
                       nullptr, nullptr, state(j + 1), m->stream));
    }
    const float inv = 1.f / (4.f * (float)M0 * (float)k);
    for (int j = k; j >= 1; --j) {
        CK(evsur::unroll_term(state(j), d_targets + (long long)(j - 1) * F, M0, m->norm, inv, Gx, m->dO, m->loss,
                              m->stream));
        if ((rc = forward(m, state(j - 1), B, true))) return rc;
        if ((rc = backward(m, B))) return rc;
        // backward() leaves the first convolution's dZ in m->dZ.
        if (j > 1)
            CK(evsur::conv0_dx(m->dZ, m->conv[0].wb, m->conv[0].kp, M0, m->lh, m->lw, m->norm, Gx, m->stream));
    }
    if (loss) {
        CK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        return check_status(m, nullptr);
    }
    return SUR_OK;
}

// One bias-corrected Adam step on the gradients in m->G, then the BF16 weight copies.
int adam_update(sur_model *m, float lr)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m->adam_t++;
    const double c1 = 1.0 - pow((double)b1, (double)m->adam_t), c2 = 1.0 - pow((double)b2, (double)m->adam_t);
    CK(evsur::adam(m->P, m->G, m->Mo, m->Vo, m->nparam, lr, b1, b2, eps, (float)c1, (float)c2, m->stream));
    return refresh_weights(m);
}

}  // namespace

extern "C" {

int sur_init(int H, int W, int base_ch, uint64_t seed, void *stream, sur_model **out)
{
    if (!out) return SUR_EINVAL;
    *out = nullptr;
    if (base_ch != kBase) return SUR_EINVAL;
    int lh = 0, lw = 0;
    while ((1 << lh) < H && lh < 30) ++lh;
    while ((1 << lw) < W && lw < 30) ++lw;
    if ((1 << lh) != H || (1 << lw) != W || H < 16 || W < 16) return SUR_EINVAL;
    sur_model *m = new (std::nothrow) sur_model();
    if (!m) return SUR_ENOMEM;
    m->H = H;
    m->W = W;
    m->lh = lh;
    m->lw = lw;
    m->stream = static_cast<cudaStream_t>(stream);
    if (!m->stream) {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete m;
            return SUR_ECUDA;
        }
        m->own_stream = true;
    }
    // Parameter layout (canonical order).
    long long off = 0;
    long long wb_elems = 0;
    for (int i = 0; i < kConvs; ++i) {
        ConvL &L = m->conv[i];
        L.cin = kConvIO[i][0];
        L.cout = kConvIO[i][1];
        L.kp = (int)round_up(9LL * L.cin, 64);
        L.kpo = (int)round_up(9LL * L.cout, 64);
        L.w = off;
        off += (long long)L.kp * L.cout;
        L.b = off;
        off += L.cout;
        wb_elems += round_up((long long)L.cout * L.kp, 128) + round_up((long long)L.cin * L.kpo, 128);
    }
    for (int j = 0; j < kUps; ++j) {
        UpL &U = m->up[j];
        U.cin = kUpIO[j][0];
        U.cout = kUpIO[j][1];
        U.w = off;
        off += 4LL * U.cout * U.cin;
        U.b = off;
        off += U.cout;
        wb_elems += 2 * round_up(4LL * U.cout * U.cin, 128);
    }
    m->head_w = off;
    off += 4 * kBase;
    m->head_b = off;
    off += 4;
    m->nparam = off;

    // Host initialisation: uniform(-sqrt(6/fan_in), sqrt(6/fan_in)); padded inputs
    // of c00 (channels 4..7) and the padded rows stay zero; the head is scaled by 0.1
    // so that the first predictions are small increments.
    std::vector<float> h((size_t)off, 0.f);
    uint64_t s = seed;
    auto uni = [&](float bound) { return (float)((double)(splitmix64(s) >> 11) * 0x1.0p-53 * 2.0 - 1.0) * bound; };
    for (int i = 0; i < kConvs; ++i) {
        const ConvL &L = m->conv[i];
        const int cin_eff = i == 0 ? 4 : L.cin;
        const float bound = sqrtf(6.f / (9.f * cin_eff));
        for (int tap = 0; tap < 9; ++tap)
            for (int ci = 0; ci < cin_eff; ++ci)
                for (int co = 0; co < L.cout; ++co) h[L.w + (long long)(tap * L.cin + ci) * L.cout + co] = uni(bound);
    }
    for (int j = 0; j < kUps; ++j) {
        const UpL &U = m->up[j];
        const float bound = sqrtf(6.f / U.cin);
        for (long long e = 0; e < 4LL * U.cout * U.cin; ++e) h[U.w + e] = uni(bound);
    }
    {
        const float bound = 0.1f * sqrtf(6.f / kBase);
        for (int e = 0; e < 4 * kBase; ++e) h[m->head_w + e] = uni(bound);
    }

    cudaError_t e = cudaSuccess;
    const size_t pb = sizeof(float) * (size_t)off;
    if (e == cudaSuccess) e = cudaMalloc(&m->P, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->G, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->Mo, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->Vo, pb);
    if (e == cudaSuccess) e = cudaMalloc(&m->wpool, 2 * (size_t)wb_elems);
    if (e == cudaSuccess) e = cudaMalloc(&m->norm, sizeof(float) * 12);
    if (e == cudaSuccess) e = cudaMalloc(&m->status, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->P, h.data(), pb, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->G, 0, pb, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->Mo, 0, pb, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->Vo, 0, pb, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(int) * 2, m->stream);
    if (e == cudaSuccess) {
        const float nrm[12] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1};
        e = cudaMemcpyAsync(m->norm, nrm, sizeof(nrm), cudaMemcpyHostToDevice, m->stream);
    }
    if (e == cudaSuccess) {
        bf16 *p = m->wpool;
        for (int i = 0; i < kConvs; ++i) {
            ConvL &L = m->conv[i];
            L.wb = p;
            p += round_up((long long)L.cout * L.kp, 128);
            L.wf = p;
            p += round_up((long long)L.cin * L.kpo, 128);
        }
        for (int j = 0; j < kUps; ++j) {
            UpL &U = m->up[j];
            U.wb = p;
            p += round_up(4LL * U.cout * U.cin, 128);
            U.wt = p;
            p += round_up(4LL * U.cout * U.cin, 128);
        }
        if (refresh_weights(m) != SUR_OK) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        sur_free(m);
        return SUR_ECUDA;
    }
    *out = m;
    return SUR_OK;
}

int sur_free(sur_model *m)
{
    if (!m) return SUR_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->P);
    cudaFree(m->G);
    cudaFree(m->Mo);
    cudaFree(m->Vo);
    cudaFree(m->wpool);
    cudaFree(m->norm);
    cudaFree(m->status);
    cudaFree(m->loss);
    cudaFree(m->ind);
    cudaFree(m->ubuf);
    cudaFree(m->arena);
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
    return SUR_OK;
}

long long sur_num_params(const sur_model *m) { return m ? m->nparam : -1; }

int sur_get_params(sur_model *m, float *h_params, long long n)
{
    if (!m || !h_params || n != m->nparam) return fail(m, SUR_EINVAL, "expected %lld parameters", m ? m->nparam : 0);
    CK(cudaMemcpyAsync(h_params, m->P, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return SUR_OK;
}

int sur_set_params(sur_model *m, const float *h_params, long long n)
{
    if (!m || !h_params || n != m->nparam) return fail(m, SUR_EINVAL, "expected %lld parameters", m ? m->nparam : 0);
    CK(cudaMemcpyAsync(m->P, h_params, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream));
    int rc = refresh_weights(m);
    if (rc) return rc;
    CK(cudaStreamSynchronize(m->stream));
    return SUR_OK;
}

int sur_get_grads(sur_model *m, float *h_grads, long long n)
{
    if (!m || !h_grads || n != m->nparam) return fail(m, SUR_EINVAL, "expected %lld parameters", m ? m->nparam : 0);
    CK(cudaMemcpyAsync(h_grads, m->G, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return SUR_OK;
}

int sur_set_norm(sur_model *m, const float *in_mean, const float *in_scale, const float *out_scale)
{
    if (!m || !in_mean || !in_scale || !out_scale) return fail(m, SUR_EINVAL, "NULL normalisation array");
    float h[12];
    for (int c = 0; c < 4; ++c) {
        if (!(in_scale[c] > 0.f) || !(out_scale[c] > 0.f) || !isfinite(in_mean[c]))
            return fail(m, SUR_EINVAL, "scales must be positive and finite");
        h[c] = in_mean[c];
        h[4 + c] = in_scale[c];
        h[8 + c] = out_scale[c];
    }
    CK(cudaMemcpyAsync(m->norm, h, sizeof(h), cudaMemcpyHostToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return SUR_OK;
}

int sur_forward_backward(sur_model *m, const float *d_x, const float *d_y, int batch, float *loss)
{
    evtrace::Range trace_("sur_forward_backward");
    return fwd_bwd(m, d_x, d_y, batch, loss);
}

int sur_train_step(sur_model *m, const float *d_x, const float *d_y, int batch, float lr, float *loss)
{
    evtrace::Range trace_("sur_train_step");
    if (!m || !(lr >= 0.f)) return fail(m, SUR_EINVAL, "invalid arguments");
    int rc = fwd_bwd(m, d_x, d_y, batch, nullptr);
    if (rc) return rc;
    if ((rc = adam_update(m, lr))) return rc;
    if (loss) {
        CK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        return check_status(m, nullptr);
    }
    return SUR_OK;
}

int sur_forward_backward_unrolled(sur_model *m, const float *d_x0, const float *d_targets, int windows, int batch,
                                  float *loss)
{
    evtrace::Range trace_("sur_forward_backward_unrolled");
    return fwd_bwd_unrolled(m, d_x0, d_targets, windows, batch, loss);
}

int sur_train_step_unrolled(sur_model *m, const float *d_x0, const float *d_targets, int windows, int batch, float lr,
                            float *loss)
{
    evtrace::Range trace_("sur_train_step_unrolled");
    if (!m || !(lr >= 0.f)) return fail(m, SUR_EINVAL, "invalid arguments");
    int rc = fwd_bwd_unrolled(m, d_x0, d_targets, windows, batch, nullptr);
    if (rc) return rc;
    if ((rc = adam_update(m, lr))) return rc;
    if (loss) {
        CK(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        return check_status(m, nullptr);
    }
    return SUR_OK;
}

int sur_infer(sur_model *m, const float *d_x, float *d_y, int batch)
{
    evtrace::Range trace_("sur_infer");
    if (!m || !d_x || !d_y || batch < 1) return fail(m, SUR_EINVAL, "invalid arguments");
    int rc = ensure_batch(m, batch, m->train_buffers);
    if (rc) return rc;
    if ((rc = forward(m, d_x, batch, false))) return rc;
    const long long M0 = lvl_pix(m, 0, batch);
    CK(evsur::head(m->Y03, M0, m->lh, m->lw, m->P + m->head_w, m->P + m->head_b, m->norm, d_x, nullptr, 1, nullptr, nullptr, d_y,
                   m->stream));
    return SUR_OK;
}

int sur_rollout(sur_model *m, lbm_ctx *lb, float *d_fields, int batch, const sur_rollout_cfg *cfg,
                unsigned char *h_used_lb, int *n_fallback)
{
    evtrace::Range trace_("sur_rollout");
    if (!m || !lb || !d_fields || !cfg || batch < 1 || cfg->windows < 0 || cfg->steps < 1)
        return fail(m, SUR_EINVAL, "invalid arguments");
    if (batch > 4096) return fail(m, SUR_EINVAL, "at most 4096 domains per rollout");
    const long long Mb = (long long)m->H * m->W, N = Mb * batch;
    int rc = ensure_batch(m, batch, m->train_buffers);
    if (rc) return rc;
    if (!m->ind) CK(cudaMalloc(&m->ind, sizeof(double) * 3 * 4096 + sizeof(float) * 4096));
    double *d_flips = m->ind + 2 * 4096;
    float *d_delta = reinterpret_cast<float *>(m->ind + 3 * 4096);
    std::vector<double> cur(2 * batch), nxt(2 * batch), mass0(batch), flips(batch);
    const bool use_shift = cfg->max_interface_shift < 1.f;
    std::vector<float> delta(batch);
    // Indicators of d_fields into host (v); *invalid = the invalid flag.
    auto measure = [&](const float *F, std::vector<double> &v, int *invalid) -> int {
        CK(evsur::indicators(F, batch, Mb, cfg->rho_mid, m->ind, m->status + 1, m->stream));
        CK(cudaMemcpyAsync(v.data(), m->ind, sizeof(double) * 2 * batch, cudaMemcpyDeviceToHost, m->stream));
        return check_status(m, invalid);
    };
    int bad = 0;
    if ((rc = measure(d_fields, cur, &bad))) return rc;
    if (bad) return fail(m, SUR_EUNPHYSICAL, "the start fields are not finite and positive");
    for (int b = 0; b < batch; ++b) mass0[b] = cur[2 * b];
    int fallbacks = 0;
    // lb_current: the context's populations are the lattice Boltzmann state of
    // d_fields (true after a fallback window), so the next fallback window
    // continues from them instead of restarting from the local equilibrium.
    bool lb_current = false;
    for (int w = 0; w < cfg->windows; ++w) {
        if ((rc = forward(m, d_fields, batch, false))) return rc;
        CK(evsur::head(m->Y03, N, m->lh, m->lw, m->P + m->head_w, m->P + m->head_b, m->norm, d_fields, nullptr, 1,
                       nullptr, nullptr, m->next, m->stream));
        if ((rc = measure(m->next, nxt, &bad))) return rc;
        if (cfg->project_mass && !bad) {
            for (int b = 0; b < batch; ++b) delta[b] = (float)((nxt[2 * b] - mass0[b]) / (double)Mb);
            CK(cudaMemcpyAsync(d_delta, delta.data(), sizeof(float) * batch, cudaMemcpyHostToDevice, m->stream));
            CK(evsur::shift_rho(m->next, batch, Mb, d_delta, m->stream));
            if ((rc = measure(m->next, nxt, &bad))) return rc;
        }
        // Interface position: nodes whose phase differs between the proposal and the
        // current fields.
        if (use_shift && !bad) {
            CK(evsur::phase_flips(d_fields, m->next, batch, Mb, cfg->rho_mid, d_flips, m->stream));
            CK(cudaMemcpyAsync(flips.data(), d_flips, sizeof(double) * batch, cudaMemcpyDeviceToHost, m->stream));
            CK(cudaStreamSynchronize(m->stream));
        }
        // Acceptance: finite and positive fields, cumulative mass drift against the
        // start, liquid-count change against the previous window, interface shift.
        bool accept = !bad;
        for (int b = 0; b < batch && accept && use_shift; ++b)
            if (!(flips[b] <= (double)cfg->max_interface_shift * (double)Mb)) accept = false;
        for (int b = 0; b < batch && accept; ++b) {
            const double dm = fabs(nxt[2 * b] - mass0[b]) / fabs(mass0[b]);
            const double da = fabs(nxt[2 * b + 1] - cur[2 * b + 1]) / fmax(cur[2 * b + 1], 1.0);
            if (!(dm <= cfg->max_mass_drift) || !(da <= cfg->max_area_change)) accept = false;
        }
        if (accept) {
            CK(cudaMemcpyAsync(d_fields, m->next, sizeof(float) * 4 * N, cudaMemcpyDeviceToDevice, m->stream));
            cur.swap(nxt);
            lb_current = false;
        } else {
            // Lattice Boltzmann window; after a surrogate window it restarts from the
            // local equilibrium of the current fields.
            CK(cudaStreamSynchronize(m->stream));
            int lrc = lb_current ? LBM_OK : lbm_reset_device(lb, d_fields, d_fields + N, d_fields + 3 * N);
            if (lrc == LBM_OK) lrc = lbm_step(lb, cfg->steps);
            if (lrc == LBM_OK) lrc = lbm_moments_device(lb, d_fields, d_fields + N, d_fields + 3 * N);
            if (lrc == LBM_OK) lrc = lbm_sync(lb);
            if (lrc != LBM_OK) return fail(m, SUR_ECUDA, "fallback lattice Boltzmann window: %s", lbm_last_error(lb));
            if ((rc = measure(d_fields, cur, &bad))) return rc;
            if (bad) {
                if (h_used_lb) h_used_lb[w] = 1;
                if (n_fallback) *n_fallback = fallbacks + 1;
                return fail(m, SUR_EUNPHYSICAL, "lattice Boltzmann window %d ended non-finite or non-positive", w);
            }
            lb_current = true;
            ++fallbacks;
        }
        if (h_used_lb) h_used_lb[w] = accept ? 0 : 1;
    }
    CK(cudaStreamSynchronize(m->stream));
    if (n_fallback) *n_fallback = fallbacks;
    return SUR_OK;
}

const char *sur_last_error(const sur_model *m) { return m ? m->err : "no model"; }

}  // extern "C"

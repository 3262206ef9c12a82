// C ABI of the Enskog-Vlasov lattice Boltzmann library (declared in include/evlbm.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>
#include <vector>

#include "../../include/evlbm.h"
#include "dispatch.h"
#include "trace.h"

using evlbm::KParams;

struct lbm_ctx {
    lbm_params P;
    KParams K;
    cudaStream_t stream;
    int Q, D;
    long long N;
    size_t pop_bytes;      // bytes per stored population
    size_t real_bytes;     // bytes per scratch value (8 for FP64, 4 otherwise)
    void *f[2], *g[2];
    void *R[2];            // per-node reference records of 16-bit storage ([N] of 16 bytes)
    int cur;
    void *RT_iso;          // frozen R*T field (thermal = 0), in the scratch precision
    void *scratch;         // stage-kernel fields, allocated on first use
    void *red;             // reduction work space
    long long steps;
    char err[512];
};

namespace {

thread_local char g_init_err[512] = "";

int fail(lbm_ctx *c, int code, const char *fmt, ...)
{
    char *dst = c ? c->err : g_init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(lbm_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(ctx, call)                                               \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);  \
    } while (0)

bool fp64(const lbm_ctx *c) { return c->P.precision == LBM_FP64; }

int ensure_scratch(lbm_ctx *c)
{
    if (c->scratch) return LBM_OK;
    CK(c, cudaMalloc(&c->scratch, c->real_bytes * evlbm::kRefFieldCount * (size_t)c->N));
    return LBM_OK;
}

int validate(const lbm_params *p)
{
    if (!p) return fail(nullptr, LBM_EINVAL, "params is NULL");
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q27) return fail(nullptr, LBM_EINVAL, "lattice must be 0 or 1");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(nullptr, LBM_EINVAL, "lattice sizes must be >= 1");
    if ((long long)p->nx * p->ny * p->nz > (1LL << 31) - 1)
        return fail(nullptr, LBM_EINVAL, "more than 2^31-1 nodes");
    if (p->eos != LBM_EOS_VDW && p->eos != LBM_EOS_CS) return fail(nullptr, LBM_EINVAL, "eos must be 0 or 1");
    if (!(p->a >= 0.0) || !(p->b >= 0.0) || !(p->kappa >= 0.0) || !(p->R > 0.0))
        return fail(nullptr, LBM_EINVAL, "a, b, kappa must be >= 0 and R > 0");
    if (!(p->tau > 0.0) || !(p->lambda > 0.0)) return fail(nullptr, LBM_EINVAL, "tau and lambda must be > 0");
    if (p->thermal != 0 && p->thermal != 1) return fail(nullptr, LBM_EINVAL, "thermal must be 0 or 1");
    if (p->precision < LBM_FP64 || p->precision > LBM_BF16_DEV)
        return fail(nullptr, LBM_EINVAL, "precision must be 0..3");
    if (p->force_form != 0 && p->force_form != 1) return fail(nullptr, LBM_EINVAL, "force_form must be 0 or 1");
    return LBM_OK;
}

// Fills the kernel parameter block.
void fill_kparams(lbm_ctx *c)
{
    const lbm_params &p = c->P;
    KParams &k = c->K;
    memset(&k, 0, sizeof(k));
    k.nx = p.nx;
    k.ny = p.ny;
    k.nz = p.nz;
    k.N = c->N;
    k.eos = p.eos;
    k.thermal = p.thermal;
    k.force_form = p.force_form;
    k.a = p.a;
    k.b = p.b;
    k.kappa = p.kappa;
    k.lambda = p.lambda;
    const double beta = 1.0 / (2.0 * p.tau + 1.0);   // Eq. (beta), dt = 1
    k.c_eq = 2.0 * beta;
    k.c_star = (1.0 / p.lambda) * (1.0 - beta);      // (dt/lambda)(1 - beta)
}

bool dev16(const lbm_ctx *c) { return c->P.precision == LBM_FP16_DEV || c->P.precision == LBM_BF16_DEV; }

int run_macro(lbm_ctx *c)
{
    int rc = ensure_scratch(c);
    if (rc) return rc;
    cudaError_t e = fp64(c) ? evlbm::ref_macro_f64(c->Q, c->K, c->scratch, c->RT_iso, c->f[c->cur], c->g[c->cur],
                                                  c->stream)
                            : evlbm::ref_macro_f32(c->P.precision, c->Q, c->K, c->scratch, c->RT_iso,
                                                   c->f[c->cur], c->g[c->cur], c->R[c->cur], c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "moment stages");
    return LBM_OK;
}

// Copies `count` scratch values starting at field offset `off` (in units of N) to host doubles.
int copy_field(lbm_ctx *c, long long off, long long count, double *dst, double scale_div)
{
    const size_t bytes = c->real_bytes * (size_t)count;
    const char *src = static_cast<const char *>(c->scratch) + c->real_bytes * (size_t)(off * c->N);
    if (fp64(c)) {
        CK(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        if (scale_div != 1.0)
            for (long long k = 0; k < count; ++k) dst[k] = dst[k] / scale_div;
    } else {
        std::vector<float> tmp((size_t)count);
        CK(c, cudaMemcpyAsync(tmp.data(), src, bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        for (long long k = 0; k < count; ++k) dst[k] = double(tmp[k]) / scale_div;
    }
    return LBM_OK;
}

void free_all(lbm_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->f[k]) cudaFree(c->f[k]);
        if (c->g[k]) cudaFree(c->g[k]);
        if (c->R[k]) cudaFree(c->R[k]);
    }
    if (c->RT_iso) cudaFree(c->RT_iso);
    if (c->scratch) cudaFree(c->scratch);
    if (c->red) cudaFree(c->red);
}

}  // namespace

namespace {
// RT = R * T on the device (FP32 contexts keep their scratch fields in FP32).
__global__ void k_scale_field(const float *T, float R, long long N, float *RT)
{
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x)
        RT[n] = R * T[n];
}
// Initial fields, FP64 as the caller passed them (rho [N], u [D][N], T [N]), checked and
// converted on the device: out = (rho, u, R T) in the scratch precision; *bad = the lowest
// node with rho or T not finite and > 0 or u not finite (left at N when all are valid).
template <typename real>
__global__ void k_prepare_fields(const double *in, int D, long long N, double R, real *out, long long *bad)
{
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const double rho = in[n], T = in[(D + 1) * N + n];
        bool ok = rho > 0.0 && isfinite(rho) && T > 0.0 && isfinite(T);
        for (int a = 0; a < D; ++a) {
            const double v = in[(1 + a) * N + n];
            ok = ok && isfinite(v);
            out[(1 + a) * N + n] = real(v);
        }
        out[n] = real(rho);
        out[(D + 1) * N + n] = real(R * T);
        if (!ok) atomicMin(reinterpret_cast<unsigned long long *>(bad), (unsigned long long)n);
    }
}
}  // namespace

extern "C" {

int lbm_init(const lbm_params *params, const double *rho, const double *u, const double *T, void *stream,
             lbm_ctx **out)
{
    g_init_err[0] = 0;
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(params);
    if (rc) return rc;
    if (!rho || !u || !T) return fail(nullptr, LBM_EINVAL, "rho, u and T must be host arrays");

    lbm_ctx *c = static_cast<lbm_ctx *>(calloc(1, sizeof(lbm_ctx)));
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    c->P = *params;
    c->stream = static_cast<cudaStream_t>(stream);
    c->Q = params->lattice == LBM_D2Q9 ? 9 : 27;
    c->D = params->lattice == LBM_D2Q9 ? 2 : 3;
    c->N = (long long)params->nx * params->ny * params->nz;
    c->pop_bytes = params->precision == LBM_FP64 ? 8 : (params->precision == LBM_FP32 ? 4 : 2);
    c->real_bytes = params->precision == LBM_FP64 ? 8 : 4;
    const long long N = c->N;
    const int D = c->D;

    fill_kparams(c);

    // Device state.
    const size_t pop = c->pop_bytes * (size_t)c->Q * (size_t)N;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&c->f[k], pop);
        if (e == cudaSuccess && params->thermal) e = cudaMalloc(&c->g[k], pop);
        if (e == cudaSuccess && dev16(c)) e = cudaMalloc(&c->R[k], evlbm::kRecBytes * (size_t)N);
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->red, evlbm::totals_work_bytes(N));
    if (e == cudaSuccess) e = cudaMalloc(&c->RT_iso, c->real_bytes * (size_t)N);
    // The caller's FP64 fields go to the device as they are (one copy each, DMA when the
    // host arrays are pinned), followed by the index word; the check and the conversion to
    // the scratch precision -- rho [N], u [D][N], RT [N] = R T -- run in one kernel.
    const size_t nf = (size_t)(D + 2) * (size_t)N;
    void *d_fields = nullptr, *d_in = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_fields, c->real_bytes * nf);
    if (e == cudaSuccess) e = cudaMalloc(&d_in, sizeof(double) * nf + sizeof(long long));
    if (e != cudaSuccess) {
        const int code = cuda_fail(nullptr, e, "lbm_init allocation");
        if (d_fields) cudaFree(d_fields);
        if (d_in) cudaFree(d_in);
        free_all(c);
        free(c);
        return code;
    }
    double *din = static_cast<double *>(d_in);
    long long *d_bad = reinterpret_cast<long long *>(din + nf);
    long long bad = N;
    e = cudaMemcpyAsync(din, rho, sizeof(double) * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(din + N, u, sizeof(double) * D * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(din + (D + 1) * N, T, sizeof(double) * N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_bad, &bad, sizeof(bad), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        long long blocks = (N + 255) / 256;
        if (blocks > 8192) blocks = 8192;
        if (c->real_bytes == 8)
            k_prepare_fields<double><<<(int)blocks, 256, 0, c->stream>>>(din, D, N, params->R,
                                                                         static_cast<double *>(d_fields), d_bad);
        else
            k_prepare_fields<float><<<(int)blocks, 256, 0, c->stream>>>(din, D, N, params->R,
                                                                        static_cast<float *>(d_fields), d_bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_in);
    if (e == cudaSuccess && bad < N) {
        cudaFree(d_fields);
        free_all(c);
        free(c);
        return fail(nullptr, LBM_ENONFINITE, "rho and T must be finite and > 0 and u finite (node %lld)", bad);
    }
    const char *dF = static_cast<const char *>(d_fields);
    const void *d_rho = dF, *d_u = dF + c->real_bytes * N, *d_RT = dF + c->real_bytes * (D + 1) * N;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->RT_iso, d_RT, c->real_bytes * N, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = fp64(c) ? evlbm::ref_init_f64(c->Q, c->K, d_rho, d_u, d_RT, c->f[0], c->g[0], c->stream)
                    : evlbm::ref_init_f32(params->precision, c->Q, c->K, d_rho, d_u, d_RT, c->f[0], c->g[0],
                                          c->R[0], c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_fields);
    if (e != cudaSuccess) {
        const int code = cuda_fail(nullptr, e, "lbm_init");
        free_all(c);
        free(c);
        return code;
    }
    c->cur = 0;
    *out = c;
    return LBM_OK;
}

int lbm_step(lbm_ctx *c, int n_steps)
{
    evtrace::Range trace_("lbm_step");
    if (!c) return LBM_EINVAL;
    if (n_steps < 0) return fail(c, LBM_EINVAL, "n_steps must be >= 0");
    const bool fused = !fp64(c) && evlbm::fused2d_supported(c->P.precision, c->Q, c->K);
    const bool fused3 = !fp64(c) && evlbm::fused3d_supported(c->P.precision, c->Q, c->K);
    if (!fused && !fused3) {
        int rc = ensure_scratch(c);
        if (rc) return rc;
    }
    for (int s = 0; s < n_steps; ++s) {
        const int nx = c->cur ^ 1;
        cudaError_t e;
        if (fused)
            e = evlbm::fused2d_step(c->P.precision, c->K, c->f[c->cur], c->g[c->cur], c->f[nx], c->g[nx], c->RT_iso,
                                    c->R[c->cur], c->R[nx], c->stream);
        else if (fused3)
            e = evlbm::fused3d_step(c->P.precision, c->K, c->f[c->cur], c->g[c->cur], c->f[nx], c->g[nx], c->RT_iso,
                                    c->R[c->cur], c->R[nx], c->stream);
        else if (fp64(c))
            e = evlbm::ref_step_f64(c->Q, c->K, c->scratch, c->RT_iso, c->f[c->cur], c->g[c->cur], c->f[nx],
                                    c->g[nx], c->stream);
        else
            e = evlbm::ref_step_f32(c->P.precision, c->Q, c->K, c->scratch, c->RT_iso, c->f[c->cur], c->g[c->cur],
                                    c->f[nx], c->g[nx], c->R[c->cur], c->R[nx], c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step");
        c->cur = nx;
        c->steps++;
    }
    return LBM_OK;
}

int lbm_moments(lbm_ctx *c, double *rho, double *u, double *T, double *F)
{
    if (!c) return LBM_EINVAL;
    int rc = run_macro(c);
    if (rc) return rc;
    using O = evlbm::FieldOffsets;
    const long long N = c->N;
    if (rho && (rc = copy_field(c, O::rho, N, rho, 1.0))) return rc;
    if (u && (rc = copy_field(c, O::u, c->D * N, u, 1.0))) return rc;
    if (T && (rc = copy_field(c, O::RT, N, T, c->P.R))) return rc;
    if (F && (rc = copy_field(c, O::F, c->D * N, F, 1.0))) return rc;
    return LBM_OK;
}

int lbm_reset_device(lbm_ctx *c, const float *d_rho, const float *d_u, const float *d_T)
{
    if (!c) return LBM_EINVAL;
    if (fp64(c)) return fail(c, LBM_EINVAL, "lbm_reset_device needs an FP32, FP16_DEV or BF16_DEV context");
    if (!d_rho || !d_u || !d_T) return fail(c, LBM_EINVAL, "d_rho, d_u and d_T must be device arrays");
    const long long N = c->N;
    long long blocks = (N + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_scale_field<<<(int)blocks, 256, 0, c->stream>>>(d_T, float(c->P.R), N, static_cast<float *>(c->RT_iso));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = evlbm::ref_init_f32(c->P.precision, c->Q, c->K, d_rho, d_u, c->RT_iso, c->f[c->cur], c->g[c->cur],
                                c->R[c->cur], c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_reset_device");
    return LBM_OK;
}

int lbm_moments_device(lbm_ctx *c, float *d_rho, float *d_u, float *d_T)
{
    if (!c) return LBM_EINVAL;
    int rc = run_macro(c);
    if (rc) return rc;
    cudaError_t e = fp64(c) ? evlbm::ref_export_f64(c->Q, c->K, c->scratch, c->P.R, d_rho, d_u, d_T, c->stream)
                            : evlbm::ref_export_f32(c->Q, c->K, c->scratch, c->P.R, d_rho, d_u, d_T, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_moments_device");
    return LBM_OK;
}

int lbm_populations(lbm_ctx *c, double *f, double *g)
{
    if (!c || !f) return c ? fail(c, LBM_EINVAL, "f is NULL") : LBM_EINVAL;
    const size_t cnt = (size_t)c->Q * (size_t)c->N;
    if (fp64(c)) {
        CK(c, cudaMemcpyAsync(f, c->f[c->cur], sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
        if (g && c->P.thermal)
            CK(c, cudaMemcpyAsync(g, c->g[c->cur], sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }
    double *tmp = nullptr;
    CK(c, cudaMalloc(&tmp, sizeof(double) * cnt));
    for (int which = 0; which < (c->P.thermal && g ? 2 : 1); ++which) {
        cudaError_t e = evlbm::expand_f32(c->P.precision, c->Q, c->K, which ? c->g[c->cur] : c->f[c->cur],
                                          c->R[c->cur], tmp, which, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(which ? g : f, tmp, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(c, e, "lbm_populations");
        }
    }
    cudaFree(tmp);
    return LBM_OK;
}

int lbm_conserved(lbm_ctx *c, double out[5])
{
    if (!c || !out) return c ? fail(c, LBM_EINVAL, "out is NULL") : LBM_EINVAL;
    int bad = 0;
    cudaError_t e = evlbm::totals(c->P.precision, c->Q, c->K, c->f[c->cur], c->g[c->cur], c->R[c->cur], c->red, out,
                                  &bad, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_conserved");
    if (bad) return fail(c, LBM_ENONFINITE, "non-finite population after %lld steps", c->steps);
    return LBM_OK;
}

long long lbm_step_count(const lbm_ctx *c) { return c ? c->steps : -1; }

long long lbm_bounds_violations(void)
{
    const long long v[4] = {evlbm::fused2d_oob(), evlbm::fused2d16_oob(), evlbm::fused3d_oob(), evlbm::batch_oob()};
    long long total = 0;
    for (long long x : v) {
        if (x < 0) return x;
        total += x;
    }
    return total;
}

int lbm_launches_per_step(const lbm_ctx *c)
{
    if (!c) return -1;
    return (!fp64(c) && (evlbm::fused2d_supported(c->P.precision, c->Q, c->K) ||
                         evlbm::fused3d_supported(c->P.precision, c->Q, c->K)))
               ? 1
               : (c->K.walls ? 5 : 4);
}

int lbm_set_walls(lbm_ctx *c, int enable, const double u_lo[3], const double u_hi[3], double T_w)
{
    if (!c) return LBM_EINVAL;
    if (enable != 0 && enable != 1) return fail(c, LBM_EINVAL, "enable must be 0 or 1");
    if (!enable) {
        c->K.walls = 0;
        return LBM_OK;
    }
    if (!u_lo || !u_hi) return fail(c, LBM_EINVAL, "u_lo and u_hi must be 3-vectors");
    if (dev16(c)) return fail(c, LBM_EINVAL, "walls need FP64 or FP32 storage");
    if (c->P.nx < 3) return fail(c, LBM_EINVAL, "walls need nx >= 3");
    if (c->P.kappa != 0.0) return fail(c, LBM_EINVAL, "walls need kappa = 0 (a single-phase fluid)");
    if (!(T_w > 0.0) || !isfinite(T_w)) return fail(c, LBM_EINVAL, "T_w must be finite and > 0");
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(u_lo[a]) || !isfinite(u_hi[a])) return fail(c, LBM_EINVAL, "wall velocities must be finite");
        if (a == 0 && (u_lo[a] != 0.0 || u_hi[a] != 0.0))
            return fail(c, LBM_EINVAL, "the walls move parallel to themselves (u_x = 0)");
        if (a == 2 && c->D == 2 && (u_lo[a] != 0.0 || u_hi[a] != 0.0))
            return fail(c, LBM_EINVAL, "D2Q9: u_z of the walls must be 0");
        c->K.wall_u[0][a] = u_lo[a];
        c->K.wall_u[1][a] = u_hi[a];
    }
    c->K.wall_RT = c->P.R * T_w;
    c->K.walls = 1;
    return LBM_OK;
}

int lbm_set_tile(lbm_ctx *c, int tile_w, int tile_h)
{
    if (!c) return LBM_EINVAL;
    bool ok = tile_w == 0 && tile_h == 0;
    if (c->Q == 27) {
        ok = ok || ((tile_w == 0 || tile_w == evlbm::fused3d_tile_w(c->P.precision)) && tile_h >= 1);
        if (!ok)
            return fail(c, LBM_EINVAL, "D3Q27: tile_w must be 0 or the kernel's tile width (%d) and tile_h (z-chunk) >= 1",
                        evlbm::fused3d_tile_w(c->P.precision));
    } else {
        for (int k = 0; k < evlbm::kFusedWidthCount; ++k)
            ok = ok || (tile_w == evlbm::kFusedWidths[k] && (tile_h >= 1 || tile_h == LBM_TILE_BALANCED));
        if (!ok)
            return fail(c, LBM_EINVAL,
                        "tile_w must be one of 64,96,128,192 and tile_h >= 1 or LBM_TILE_BALANCED (or both 0)");
    }
    c->K.tile_w = (c->Q == 27 && tile_h >= 1) ? evlbm::fused3d_tile_w(c->P.precision) : tile_w;
    c->K.tile_h = tile_h;
    return LBM_OK;
}

int lbm_get_tile(const lbm_ctx *c, int *tile_w, int *tile_h)
{
    if (!c) return LBM_EINVAL;
    if (tile_w) *tile_w = c->K.tile_w;
    if (tile_h) *tile_h = c->K.tile_h;
    return LBM_OK;
}

// z-chunk height of the fused D3Q27 kernel by timed probes on the live state
// (its output buffer is the spare one, so the state is unchanged).
// Rounds of the autotuners' candidate sweep (each candidate keeps its fastest round).
constexpr int kAutotuneRounds = 2;

static int autotune3d(lbm_ctx *c, int probe_steps, int *tile_w, int *tile_h)
{
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    const int heights[] = {8, 16, 32, 64, 128, 256};
    const int nx = c->cur ^ 1;
    float tmin[6] = {1e30f, 1e30f, 1e30f, 1e30f, 1e30f, 1e30f};
    KParams K = c->K;
    cudaError_t e = cudaSuccess;
    // Two rounds over the candidates, each keeping its faster time: a single probe of a
    // few launches is not repeatable to the few per cent that separate neighbouring chunks.
    for (int round = 0; round < kAutotuneRounds; ++round)
    for (int hi = 0; hi < 6 && e == cudaSuccess; ++hi) {
        const int H = heights[hi] < c->P.nz ? heights[hi] : c->P.nz;
        if (hi > 0 && H == (heights[hi - 1] < c->P.nz ? heights[hi - 1] : c->P.nz)) continue;
        K.tile_w = evlbm::fused3d_tile_w(c->P.precision);
        K.tile_h = H;
        for (int s = 0; s <= probe_steps && e == cudaSuccess; ++s) {
            if (s == 1) e = cudaEventRecord(e0, c->stream);
            if (e == cudaSuccess)
                e = evlbm::fused3d_step(c->P.precision, K, c->f[c->cur], c->g[c->cur], c->f[nx], c->g[nx],
                                        c->RT_iso, c->R[c->cur], c->R[nx], c->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < tmin[hi]) tmin[hi] = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_autotune");
    int bh = 0;
    float best = 1e30f;
    for (int hi = 0; hi < 6; ++hi)
        if (tmin[hi] < best) {
            best = tmin[hi];
            bh = heights[hi] < c->P.nz ? heights[hi] : c->P.nz;
        }
    c->K.tile_w = evlbm::fused3d_tile_w(c->P.precision);
    c->K.tile_h = bh;
    if (tile_w) *tile_w = evlbm::fused3d_tile_w(c->P.precision);
    if (tile_h) *tile_h = bh;
    return LBM_OK;
}

int lbm_autotune(lbm_ctx *c, int probe_steps, int *tile_w, int *tile_h)
{
    if (!c || probe_steps < 1) return c ? fail(c, LBM_EINVAL, "probe_steps must be >= 1") : LBM_EINVAL;
    if (tile_w) *tile_w = 0;
    if (tile_h) *tile_h = 0;
    if (!fp64(c) && evlbm::fused3d_supported(c->P.precision, c->Q, c->K)) return autotune3d(c, probe_steps, tile_w, tile_h);
    if (fp64(c) || !evlbm::fused2d_supported(c->P.precision, c->Q, c->K)) return LBM_OK;
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    const int heights[] = {16, 32, 64, 128, 256, LBM_TILE_BALANCED};
    const int nx = c->cur ^ 1;
    std::vector<float> tmin(evlbm::kFusedWidthCount * 6, 1e30f);
    KParams K = c->K;
    cudaError_t e = cudaSuccess;
    for (int round = 0; round < kAutotuneRounds; ++round)
    for (int wi = 0; wi < evlbm::kFusedWidthCount && e == cudaSuccess; ++wi) {
        const int W = evlbm::kFusedWidths[wi];
        if (W > 2 * c->P.nx && W != evlbm::kFusedWidths[0]) continue;
        for (int hi = 0; hi < 6 && e == cudaSuccess; ++hi) {
            const int H = heights[hi] < c->P.ny ? heights[hi] : c->P.ny;    // the balanced grid stays -1
            if (hi > 0 && hi < 5 && H == (heights[hi - 1] < c->P.ny ? heights[hi - 1] : c->P.ny)) continue;
            K.tile_w = W;
            K.tile_h = H;
            // One untimed launch, then probe_steps timed ones; input stays c->f[c->cur].
            for (int s = 0; s <= probe_steps && e == cudaSuccess; ++s) {
                if (s == 1) e = cudaEventRecord(e0, c->stream);
                if (e == cudaSuccess)
                    e = evlbm::fused2d_step(c->P.precision, K, c->f[c->cur], c->g[c->cur], c->f[nx], c->g[nx],
                                            c->RT_iso, c->R[c->cur], c->R[nx], c->stream);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < tmin[wi * 6 + hi]) tmin[wi * 6 + hi] = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_autotune");
    int bw = 0, bh = 0;
    float best = 1e30f;
    for (int wi = 0; wi < evlbm::kFusedWidthCount; ++wi)
        for (int hi = 0; hi < 6; ++hi)
            if (tmin[wi * 6 + hi] < best) {
                best = tmin[wi * 6 + hi];
                bw = evlbm::kFusedWidths[wi];
                bh = heights[hi] < c->P.ny ? heights[hi] : c->P.ny;
            }
    c->K.tile_w = bw;
    c->K.tile_h = bh;
    if (tile_w) *tile_w = bw;
    if (tile_h) *tile_h = bh;
    return LBM_OK;
}

int lbm_sync(lbm_ctx *c)
{
    if (!c) return LBM_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_free(lbm_ctx *c)
{
    if (!c) return LBM_OK;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    free(c);
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err : g_init_err; }

int lbm_critical_point(int eos, double a, double b, double out[2])
{
    if (!out || (eos != LBM_EOS_VDW && eos != LBM_EOS_CS) || !(a > 0.0) || !(b > 0.0)) return LBM_EINVAL;
    if (eos == LBM_EOS_VDW) {
        out[0] = 1.0 / (3.0 * b);
        out[1] = 8.0 * a / (27.0 * b);
        return LBM_OK;
    }
    auto y1 = [](double e) { return (1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e) / pow(1 - e, 4); };
    auto y2 = [](double e) {
        return (4 + 8 * e - 12 * e * e + 4 * e * e * e) / pow(1 - e, 4) +
               4 * (1 + 4 * e + 4 * e * e - 4 * e * e * e + e * e * e * e) / pow(1 - e, 5);
    };
    double lo = 0.01, hi = 0.4;
    for (int k = 0; k < 200; ++k) {
        const double mid = 0.5 * (lo + hi);
        if ((y1(lo) - lo * y2(lo)) * (y1(mid) - mid * y2(mid)) <= 0) hi = mid;
        else lo = mid;
    }
    const double eta = 0.5 * (lo + hi);
    out[0] = 4.0 * eta / b;
    out[1] = 8.0 * a / (b * y2(eta));
    return LBM_OK;
}

int lbm_coexistence(int eos, double a, double b, double RT, double out[2])
{
    double crit[2];
    if (!out || lbm_critical_point(eos, a, b, crit) != LBM_OK) return LBM_EINVAL;
    if (!(RT > 0.0) || !(RT < crit[1])) return LBM_EINVAL;
    int status = 0;
    cudaError_t e = evlbm::coexistence(eos, a, b, RT, crit[0], out, &status);
    if (e != cudaSuccess) return LBM_ECUDA;
    if (status == 1) return LBM_EINVAL;
    if (status != 0) return LBM_ETIMEOUT;
    return LBM_OK;
}

int lbm_spinodal(int eos, double a, double b, double RT, double out[2])
{
    double crit[2];
    if (!out || lbm_critical_point(eos, a, b, crit) != LBM_OK) return LBM_EINVAL;
    if (!(RT > 0.0) || !(RT < crit[1])) return LBM_EINVAL;
    return evlbm::spinodal(eos, a, b, RT, crit[0], out) ? LBM_EINVAL : LBM_OK;
}

int lbm_interface(int eos, double a, double b, double RT, double kappa, double out[2])
{
    if (!out || !(kappa > 0.0)) return LBM_EINVAL;
    double co[2];
    const int rc = lbm_coexistence(eos, a, b, RT, co);
    if (rc != LBM_OK) return rc;
    evlbm::interface(eos, a, b, RT, kappa, co[0], co[1], &out[0], &out[1]);
    return LBM_OK;
}


// ---------------------------------------------------------------------------
// Checkpoint and resume.  File layout (little-endian, fixed-width fields):
//   "EVLBMCKP" | u32 version | u32 0 | i32 lattice nx ny nz eos thermal precision
//   force_form | f64 a b R kappa tau lambda | i64 steps | u64 bytes of the f, g,
//   reference-state and frozen-RT sections | the sections, in that order, exactly
//   as the context stores them on the device.
// ---------------------------------------------------------------------------
namespace {

constexpr char kCkMagic[8] = {'E', 'V', 'L', 'B', 'M', 'C', 'K', 'P'};
constexpr uint32_t kCkVersion = 2;            // 2: 16-bit storage records are FP32, 24 bytes per node
constexpr size_t kCkHeader = 8 + 4 + 4 + 8 * 4 + 6 * 8 + 8 + 4 * 8;
constexpr size_t kCkChunk = 64u << 20;          // host staging per transfer

struct CkLayout {
    void *dev[4];
    size_t bytes[4];
};

CkLayout ck_layout(const lbm_ctx *c)
{
    const size_t pop = c->pop_bytes * (size_t)c->Q * (size_t)c->N;
    CkLayout L;
    L.dev[0] = c->f[c->cur];
    L.bytes[0] = pop;
    L.dev[1] = c->g[c->cur];
    L.bytes[1] = c->P.thermal ? pop : 0;
    L.dev[2] = c->R[c->cur];
    L.bytes[2] = dev16(c) ? evlbm::kRecBytes * (size_t)c->N : 0;
    L.dev[3] = c->RT_iso;
    L.bytes[3] = c->P.thermal ? 0 : c->real_bytes * (size_t)c->N;
    return L;
}

void ck_header(const lbm_ctx *c, const CkLayout &L, unsigned char *h)
{
    size_t o = 0;
    auto put = [&](const void *v, size_t n) { memcpy(h + o, v, n); o += n; };
    const uint32_t ver = kCkVersion, zero = 0;
    put(kCkMagic, 8);
    put(&ver, 4);
    put(&zero, 4);
    const int32_t iv[8] = {c->P.lattice, c->P.nx, c->P.ny, c->P.nz, c->P.eos, c->P.thermal, c->P.precision,
                           c->P.force_form};
    put(iv, sizeof(iv));
    const double dv[6] = {c->P.a, c->P.b, c->P.R, c->P.kappa, c->P.tau, c->P.lambda};
    put(dv, sizeof(dv));
    const int64_t st = c->steps;
    put(&st, 8);
    for (int k = 0; k < 4; ++k) {
        const uint64_t b = L.bytes[k];
        put(&b, 8);
    }
}

}  // namespace

int lbm_save(lbm_ctx *c, const char *path)
{
    if (!c || !path) return c ? fail(c, LBM_EINVAL, "path is NULL") : LBM_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    const CkLayout L = ck_layout(c);
    unsigned char h[kCkHeader];
    ck_header(c, L, h);
    char tmp[4096];
    if (snprintf(tmp, sizeof(tmp), "%s.tmp", path) >= (int)sizeof(tmp)) return fail(c, LBM_EINVAL, "path too long");
    FILE *fp = fopen(tmp, "wb");
    if (!fp) return fail(c, LBM_EIO, "lbm_save: cannot open %s for writing", tmp);
    size_t largest = 0;
    for (int k = 0; k < 4; ++k) largest = L.bytes[k] > largest ? L.bytes[k] : largest;
    const size_t chunk = largest < kCkChunk ? largest : kCkChunk;
    unsigned char *buf = chunk ? static_cast<unsigned char *>(malloc(chunk)) : nullptr;
    int rc = LBM_OK;
    if (chunk && !buf) rc = fail(c, LBM_ENOMEM, "lbm_save: host staging buffer");
    if (rc == LBM_OK && fwrite(h, 1, kCkHeader, fp) != kCkHeader) rc = fail(c, LBM_EIO, "lbm_save: write failed");
    for (int k = 0; k < 4 && rc == LBM_OK; ++k)
        for (size_t o = 0; o < L.bytes[k] && rc == LBM_OK; o += chunk) {
            const size_t n = L.bytes[k] - o < chunk ? L.bytes[k] - o : chunk;
            cudaError_t e = cudaMemcpyAsync(buf, static_cast<const char *>(L.dev[k]) + o, n, cudaMemcpyDeviceToHost,
                                            c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) rc = cuda_fail(c, e, "lbm_save");
            else if (fwrite(buf, 1, n, fp) != n) rc = fail(c, LBM_EIO, "lbm_save: write failed");
        }
    free(buf);
    if (fclose(fp) != 0 && rc == LBM_OK) rc = fail(c, LBM_EIO, "lbm_save: close failed");
    if (rc == LBM_OK && rename(tmp, path) != 0) rc = fail(c, LBM_EIO, "lbm_save: cannot rename %s to %s", tmp, path);
    if (rc != LBM_OK) remove(tmp);
    return rc;
}

int lbm_load(lbm_ctx *c, const char *path)
{
    if (!c || !path) return c ? fail(c, LBM_EINVAL, "path is NULL") : LBM_EINVAL;
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(c, LBM_EIO, "lbm_load: cannot open %s", path);
    unsigned char h[kCkHeader];
    if (fread(h, 1, kCkHeader, fp) != kCkHeader) {
        fclose(fp);
        return fail(c, LBM_EIO, "lbm_load: %s is shorter than a checkpoint header", path);
    }
    if (memcmp(h, kCkMagic, 8) != 0) {
        fclose(fp);
        return fail(c, LBM_EINVAL, "lbm_load: %s is not a checkpoint of this library", path);
    }
    uint32_t ver;
    memcpy(&ver, h + 8, 4);
    if (ver != kCkVersion) {
        fclose(fp);
        return fail(c, LBM_EINVAL, "lbm_load: checkpoint version %u, expected %u", ver, kCkVersion);
    }
    // The context must describe the same lattice and model: compare every field.
    const CkLayout L = ck_layout(c);
    unsigned char mine[kCkHeader];
    ck_header(c, L, mine);
    static const char *const names[] = {"lattice", "nx", "ny", "nz", "eos", "thermal", "precision", "force_form",
                                        "a", "b", "R", "kappa", "tau", "lambda"};
    for (int k = 0; k < 14; ++k) {
        const size_t o = 16 + (k < 8 ? 4 * k : 32 + 8 * (k - 8)), n = k < 8 ? 4 : 8;
        if (memcmp(h + o, mine + o, n) != 0) {
            fclose(fp);
            return fail(c, LBM_EINVAL, "lbm_load: %s of the checkpoint differs from the context's", names[k]);
        }
    }
    int64_t steps;
    memcpy(&steps, h + 16 + 32 + 48, 8);
    size_t total = kCkHeader;
    for (int k = 0; k < 4; ++k) {
        uint64_t b;
        memcpy(&b, h + 16 + 32 + 48 + 8 + 8 * k, 8);
        if (b != L.bytes[k]) {
            fclose(fp);
            return fail(c, LBM_EINVAL, "lbm_load: section %d holds %llu bytes, the context needs %llu", k,
                        (unsigned long long)b, (unsigned long long)L.bytes[k]);
        }
        total += b;
    }
    if (fseek(fp, 0, SEEK_END) != 0 || ftell(fp) != (long)total || fseek(fp, (long)kCkHeader, SEEK_SET) != 0) {
        fclose(fp);
        return fail(c, LBM_EIO, "lbm_load: %s is truncated or has trailing bytes (%zu expected)", path, total);
    }
    // The populations and reference states go to the spare buffers and the frozen R T
    // field to host memory; only when every section has been read does the context
    // switch to them, so a failed load leaves the state as it was.
    void *dst[3] = {c->f[c->cur ^ 1], c->g[c->cur ^ 1], c->R[c->cur ^ 1]};
    size_t largest = 0;
    for (int k = 0; k < 3; ++k) largest = L.bytes[k] > largest ? L.bytes[k] : largest;
    const size_t chunk = largest < kCkChunk ? largest : kCkChunk;
    unsigned char *buf = chunk ? static_cast<unsigned char *>(malloc(chunk)) : nullptr;
    unsigned char *rt = L.bytes[3] ? static_cast<unsigned char *>(malloc(L.bytes[3])) : nullptr;
    int rc = LBM_OK;
    if ((chunk && !buf) || (L.bytes[3] && !rt)) rc = fail(c, LBM_ENOMEM, "lbm_load: host staging buffer");
    if (rc == LBM_OK) {
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "lbm_load");
    }
    for (int k = 0; k < 3 && rc == LBM_OK; ++k)
        for (size_t o = 0; o < L.bytes[k] && rc == LBM_OK; o += chunk) {
            const size_t n = L.bytes[k] - o < chunk ? L.bytes[k] - o : chunk;
            if (fread(buf, 1, n, fp) != n) {
                rc = fail(c, LBM_EIO, "lbm_load: read failed");
                break;
            }
            cudaError_t e = cudaMemcpyAsync(static_cast<char *>(dst[k]) + o, buf, n, cudaMemcpyHostToDevice,
                                            c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) rc = cuda_fail(c, e, "lbm_load");
        }
    if (rc == LBM_OK && L.bytes[3] && fread(rt, 1, L.bytes[3], fp) != L.bytes[3])
        rc = fail(c, LBM_EIO, "lbm_load: read failed");
    if (rc == LBM_OK && L.bytes[3]) {
        cudaError_t e = cudaMemcpyAsync(L.dev[3], rt, L.bytes[3], cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = cuda_fail(c, e, "lbm_load");
    }
    free(buf);
    free(rt);
    fclose(fp);
    if (rc == LBM_OK) c->cur ^= 1;
    if (rc == LBM_OK) c->steps = steps;
    return rc;
}

}  // extern "C"

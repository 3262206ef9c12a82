// FP64 device reductions of the conserved totals and the FP64 Maxwell
// construction of the coexisting densities.
#include <math.h>
#include "dispatch.h"
#include "ref_kernels.cuh"

namespace evlbm {

namespace {

constexpr int kRedBlocks = 608;   // 4 x 152 SMs
constexpr int kRedThreads = 256;

// Each thread sums its nodes in ascending order, the block combines the threads
// in a fixed tree; the result does not depend on scheduling.  16-bit storage is
// expanded with the node's reference equilibrium first.
template <typename S, int Q>
__global__ void __launch_bounds__(kRedThreads) k_totals_partial(KParams p, const S *f, const S *g, const float *R,
                                                                 double *partial, int *nonfinite)
{
    __shared__ double sh[5][kRedThreads];
    double acc[5] = {0, 0, 0, 0, 0};
    int bad = 0;
    const long long N = p.N;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        Ref16 r{};
        if constexpr (Store<S>::dev) r = load_rec(R, N, n);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            double fi = double(Store<S>::load(f + i * N + n));
            if constexpr (Store<S>::dev) fi = double(decode_f<Q>(cx_of(i), cy_of(i), cz_of(i, Q), r, float(fi)));
            bad |= !isfinite(fi);
            acc[0] += fi;
            const int c[3] = {cx_of(i), cy_of(i), cz_of(i, Q)};
#pragma unroll
            for (int a = 0; a < 3; ++a)
                acc[1 + a] += c[a] == 1 ? fi : (c[a] == -1 ? -fi : 0.0);
            if (p.thermal) {
                double gi = double(Store<S>::load(g + i * N + n));
                if constexpr (Store<S>::dev) gi = double(decode_g<Q>(cx_of(i), cy_of(i), cz_of(i, Q), r, float(gi)));
                bad |= !isfinite(gi);
                acc[4] += gi;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) partial[k * kRedBlocks + blockIdx.x] = sh[k][0];
    if (bad) atomicOr(nonfinite, 1);
}

__global__ void k_totals_final(const double *partial, double *out)
{
    __shared__ double sh[5][1024];
    for (int k = 0; k < 5; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) v += partial[k * kRedBlocks + b];
        sh[k][threadIdx.x] = v;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) out[k] = sh[k][0];
}

template <typename S>
cudaError_t totals_s(int Q, const KParams &p, const void *f, const void *g, const void *R, void *work,
                     cudaStream_t st)
{
    double *partial = static_cast<double *>(work);
    double *out = partial + 5 * kRedBlocks;
    int *flag = reinterpret_cast<int *>(out + 8);
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (Q == 9)
        k_totals_partial<S, 9><<<kRedBlocks, kRedThreads, 0, st>>>(
            p, static_cast<const S *>(f), static_cast<const S *>(g), static_cast<const float *>(R), partial, flag);
    else
        k_totals_partial<S, 27><<<kRedBlocks, kRedThreads, 0, st>>>(
            p, static_cast<const S *>(f), static_cast<const S *>(g), static_cast<const float *>(R), partial, flag);
    k_totals_final<<<1, 1024, 0, st>>>(partial, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Maxwell construction: p(rho_v) = p(rho_l), mu(rho_v) = mu(rho_l) for
// p = P_E - a rho^2 (Enskog pressure in the vdW or Carnahan-Starling form plus
// the Vlasov pressure), by bisection on the pressure level and Newton polish.
// ---------------------------------------------------------------------------
struct Eos {
    int kind;
    double a, b, RT;
    __host__ __device__ double rho_max() const { return kind == 0 ? 1.0 / b : 4.0 / b; }
    __host__ __device__ double p(double r) const
    {
        if (kind == 0) return r * RT / (1.0 - b * r) - a * r * r;
        const double e = 0.25 * b * r;
        return r * RT * (1.0 + e + e * e - e * e * e) / ((1.0 - e) * (1.0 - e) * (1.0 - e)) - a * r * r;
    }
    __host__ __device__ double dp(double r) const
    {
        if (kind == 0) return RT / ((1.0 - b * r) * (1.0 - b * r)) - 2.0 * a * r;
        const double e = 0.25 * b * r, om = 1.0 - e;
        return RT * (1.0 + 4.0 * e + 4.0 * e * e - 4.0 * e * e * e + e * e * e * e) / (om * om * om * om) -
               2.0 * a * r;
    }
    __host__ __device__ double mu(double r) const
    {
        if (kind == 0) return RT * (log(r / (1.0 - b * r)) + b * r / (1.0 - b * r)) - 2.0 * a * r;
        const double e = 0.25 * b * r, om = 1.0 - e;
        return RT * (log(r) + (8.0 * e - 9.0 * e * e + 3.0 * e * e * e) / (om * om * om)) - 2.0 * a * r;
    }
};

// Root of a monotone function on [lo, hi] by bisection (fixed number of halvings).
template <typename Fn>
__host__ __device__ double bisect(Fn fn, double lo, double hi, int halvings)
{
    double flo = fn(lo);
    for (int k = 0; k < halvings; ++k) {
        const double mid = 0.5 * (lo + hi), fm = fn(mid);
        if ((flo <= 0.0) == (fm <= 0.0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
    }
    return 0.5 * (lo + hi);
}

__global__ void k_coexistence(Eos E, double rho_c, double *out, int *status)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double rmax = E.rho_max() * (1.0 - 1e-12);
    // Spinodal densities: dp/drho = 0 on either side of the critical density.
    const double s1 = bisect([&](double r) { return E.dp(r); }, 1e-12 * rho_c, rho_c, 80);
    const double s2 = bisect([&](double r) { return E.dp(r); }, rho_c, rmax, 80);
    if (!(E.dp(0.5 * (s1 + s2)) < 0.0)) {
        *status = 1;   // no van der Waals loop: above the critical temperature
        return;
    }
    // Pressure level with equal chemical potentials, by bisection to 1e-9 relative,
    // then Newton on (p(rho_l) - p(rho_v), mu(rho_l) - mu(rho_v)).
    double Plo = fmax(E.p(s2), 0.0), Phi = E.p(s1), rv = 0.0, rl = 0.0;
    for (int k = 0; k < 100 && Phi - Plo > 1e-9 * Phi; ++k) {
        const double P = 0.5 * (Plo + Phi);
        rv = bisect([&](double r) { return E.p(r) - P; }, 1e-300, s1, 64);
        rl = bisect([&](double r) { return E.p(r) - P; }, s2, rmax, 64);
        if (E.mu(rl) < E.mu(rv)) Phi = P;   // liquid favoured: above saturation
        else Plo = P;
    }
    const double P = 0.5 * (Plo + Phi);
    rv = bisect([&](double r) { return E.p(r) - P; }, 1e-300, s1, 64);
    rl = bisect([&](double r) { return E.p(r) - P; }, s2, rmax, 64);
    int it = 0;
    for (; it < 100; ++it) {
        const double F1 = E.p(rl) - E.p(rv), F2 = E.mu(rl) - E.mu(rv);
        const double pl = E.dp(rl), pv = E.dp(rv);
        // Jacobian of (F1, F2) in (rv, rl): dmu/drho = (dp/drho)/rho.
        const double J11 = -pv, J12 = pl, J21 = -pv / rv, J22 = pl / rl;
        const double det = J11 * J22 - J12 * J21;
        const double dv = (-F1 * J22 + F2 * J12) / det;
        const double dl = (-F2 * J11 + F1 * J21) / det;
        rv += dv;
        rl += dl;
        if (fabs(dv) <= 1e-14 * rv && fabs(dl) <= 1e-14 * rl) break;
    }
    out[0] = rv;
    out[1] = rl;
    *status = (it < 100 && rv > 0.0 && rl > rv) ? 0 : 2;
}

}  // namespace

int spinodal(int eos, double a, double b, double RT, double rho_c, double out[2])
{
    const Eos E{eos, a, b, RT};
    const double rmax = E.rho_max() * (1.0 - 1e-12);
    out[0] = bisect([&](double r) { return E.dp(r); }, 1e-12 * rho_c, rho_c, 200);
    out[1] = bisect([&](double r) { return E.dp(r); }, rho_c, rmax, 200);
    return E.dp(0.5 * (out[0] + out[1])) < 0.0 ? 0 : 1;
}

// Planar interface of square-gradient theory between the coexisting densities:
// kappa/2 (d rho/dx)^2 = omega(rho), omega(rho) = int_{rho_v}^{rho} (mu(s) - mu_sat) ds
// (the excess grand-potential density; it vanishes at both coexisting densities because
// their pressures and chemical potentials are equal).  omega is accumulated on a uniform
// grid of 10 M cells by Simpson's rule in each cell; the 10-90 % width integrates
// |d rho/dx|^-1 over the cells M .. 9M (rho_v + 0.1 .. 0.9 (rho_l - rho_v)) and the
// tension sigma = int kappa |d rho/dx| d rho over all cells, both by the trapezoid rule.
void interface(int eos, double a, double b, double RT, double kappa, double rv, double rl, double *width,
               double *sigma)
{
    const Eos E{eos, a, b, RT};
    const int M = 8192, cells = 10 * M;
    const double h = (rl - rv) / cells, mu_sat = E.mu(rv);
    double omega = 0.0, w = 0.0, sg = 0.0, grad0 = 0.0;
    for (int k = 0; k < cells; ++k) {
        const double r0 = rv + k * h, r1 = rv + (k + 1) * h;
        omega += h / 6.0 * ((E.mu(r0) - mu_sat) + 4.0 * (E.mu(0.5 * (r0 + r1)) - mu_sat) + (E.mu(r1) - mu_sat));
        const double grad1 = sqrt(fmax(2.0 * omega / kappa, 0.0));     // |d rho/dx| at r1
        sg += 0.5 * h * kappa * (grad0 + grad1);
        if (k >= M && k < 9 * M) w += 0.5 * h * (1.0 / grad0 + 1.0 / grad1);
        grad0 = grad1;
    }
    *width = w;
    *sigma = sg;
}

size_t totals_work_bytes(long long) { return sizeof(double) * (5 * kRedBlocks + 8) + 64; }

cudaError_t totals(int prec, int Q, const KParams &p, const void *f, const void *g, const void *R, void *work,
                   double *h_out, int *h_nonfinite, cudaStream_t st)
{
    cudaError_t e;
    switch (prec) {
    case 0: e = totals_s<double>(Q, p, f, g, R, work, st); break;
    case 1: e = totals_s<float>(Q, p, f, g, R, work, st); break;
    case 2: e = totals_s<__half>(Q, p, f, g, R, work, st); break;
    default: e = totals_s<__nv_bfloat16>(Q, p, f, g, R, work, st); break;
    }
    if (e != cudaSuccess) return e;
    double *out = static_cast<double *>(work) + 5 * kRedBlocks;
    if ((e = cudaMemcpyAsync(h_out, out, 5 * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(h_nonfinite, out + 8, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t coexistence(int eos, double a, double b, double RT, double rho_c, double *h_out, int *h_status)
{
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 4 * sizeof(double));
    if (e != cudaSuccess) return e;
    double *d_out = static_cast<double *>(buf);
    int *d_status = reinterpret_cast<int *>(d_out + 2);
    Eos E{eos, a, b, RT};
    k_coexistence<<<1, 32>>>(E, rho_c, d_out, d_status);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(h_out, d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    return e;
}

}  // namespace evlbm

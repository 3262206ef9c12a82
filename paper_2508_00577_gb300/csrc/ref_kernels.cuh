// Stage-by-stage kernels of the Enskog-Vlasov lattice Boltzmann step
// (Karlin & Hosseini, arXiv 2508.00577), one thread per node, one kernel per
// stage, every intermediate field stored in global memory.
//
// The arithmetic follows a fixed reference order: every expression below is
// evaluated in the same sequence of IEEE operations as the plain definition of
// the step (sums in ascending population index, products in axis order,
// expressions left to right).  Compiled in FP64 with multiply-add contraction
// disabled, the populations are therefore bit-identical to any other FP64
// evaluation in that order.  Instantiated in FP32 it serves lattices and
// storage formats that have no fused kernel.
#pragma once

#include "common.cuh"
#include "dev16.cuh"

namespace evlbm {

template <int Q> struct Lat {
    static constexpr int D = (Q == 9) ? 2 : 3;
};

__host__ __device__ constexpr int c_of(int i, int a, int Q)
{
    return a == 0 ? cx_of(i) : (a == 1 ? cy_of(i) : cz_of(i, Q));
}

// 16-bit storage (dev16.cuh): a node stores its populations as deviations from its
// own local equilibrium next to its 16-byte reference record; a puller rebuilds
// h_i(y) = h^eq_i(R(y - c_i)) + w_i rho_R delta_i(y - c_i) (times e_R for g).
// FP32/FP64 storage holds the populations themselves.

struct Node {
    int x, y, z;
    long long n;
};

__device__ __forceinline__ bool node_of(const KParams &p, Node &nd)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return false;
    nd.n = n;
    nd.x = (int)(n % p.nx);
    long long r = n / p.nx;
    nd.y = (int)(r % p.ny);
    nd.z = (int)(r / p.ny);
    return true;
}

__device__ __forceinline__ long long shifted(const KParams &p, const Node &nd, int dx, int dy, int dz)
{
    int x = wrap1(nd.x + dx, p.nx), y = wrap1(nd.y + dy, p.ny), z = wrap1(nd.z + dz, p.nz);
    return (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
}

// Isotropic gradient d_a phi = (1/cs^2) sum_i w_i c_ia phi(x + c_i), cs^2 = 1/3.
template <typename real, int Q>
__device__ __forceinline__ real grad_iso(const KParams &p, const Node &nd, const real *phi, int a)
{
    real acc = real(0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int c = c_of(i, a, Q);
        if (c == 0) continue;
        const real w = real(w_of(i, Q));
        const real v = phi[shifted(p, nd, cx_of(i), cy_of(i), cz_of(i, Q))];
        acc = (c == 1) ? acc + w * v : acc - w * v;
    }
    return real(3.0) * acc;
}

// Isotropic Laplacian lap phi = (2/cs^2) sum_i w_i (phi(x + c_i) - phi(x)).
template <typename real, int Q>
__device__ __forceinline__ real lap_iso(const KParams &p, const Node &nd, const real *phi)
{
    real acc = real(0.0);
    const real c0 = phi[nd.n];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (cx_of(i) == 0 && cy_of(i) == 0 && cz_of(i, Q) == 0) continue;
        acc = acc + real(w_of(i, Q)) * (phi[shifted(p, nd, cx_of(i), cy_of(i), cz_of(i, Q))] - c0);
    }
    return real(6.0) * acc;
}

// Central difference (phi(x + e_a) - phi(x - e_a)) / 2.
template <typename real>
__device__ __forceinline__ real diff_c(const KParams &p, const Node &nd, const real *phi, int a)
{
    const int dx = a == 0, dy = a == 1, dz = a == 2;
    return real(0.5) * (phi[shifted(p, nd, dx, dy, dz)] - phi[shifted(p, nd, -dx, -dy, -dz)]);
}

// Compressibility Z = P_E/(rho RT) and the pseudo-adiabatic exponent of Eq. (gamma)
// for P0 = P_E = rho RT Z(rho): gamma0 = 1 + rho Z'/Z + 2/3 Z; with the temperature
// frozen the temperature term drops out (gamma0 = (dlnP0/dlnrho)_T).
template <typename real>
__device__ __forceinline__ void eos_Zg(int eos, int thermal, real b, real rho, real &Z, real &g0)
{
    real dlnZ;
    if (eos == 0) {
        Z = real(1.0) / (real(1.0) - b * rho);
        dlnZ = b * rho * Z;
    } else {
        const real eta = b * rho / real(4.0);
        const real num = real(1.0) + eta + eta * eta - eta * eta * eta;
        const real om = real(1.0) - eta;
        Z = num / (om * om * om);
        dlnZ = eta * (real(4.0) + real(4.0) * eta - real(2.0) * eta * eta) / (om * num);
    }
    g0 = thermal ? real(1.0) + dlnZ + real(2.0 / 3.0) * Z : real(1.0) + dlnZ;
}

// Psi_ia(xi, zeta) of Eq. (phi) for c in {-1, 0, 1}: 1 - zeta, (zeta +- xi)/2.
template <typename real>
__device__ __forceinline__ real psi(int c, real xi, real zeta)
{
    return c == 0 ? real(1.0) - zeta : (c == 1 ? real(0.5) * (zeta + xi) : real(0.5) * (zeta - xi));
}

// Psi's linear combination applied to the sequence (A0, A1, A2).
template <typename real>
__device__ __forceinline__ real psi_poly(int c, real A0, real A1, real A2)
{
    return c == 0 ? A0 - A2 : (c == 1 ? real(0.5) * (A2 + A1) : real(0.5) * (A2 - A1));
}

// f_i = rho prod_a Psi_ia(xi_a, zeta_a)  (Eqs. feq, f_star).
template <typename real, int Q>
__device__ __forceinline__ real prod_eq(int i, real rho, const real *xi, const real *zeta)
{
    real pr = real(1.0);
#pragma unroll
    for (int a = 0; a < Lat<Q>::D; ++a)
        pr = pr * psi<real>(c_of(i, a, Q), xi[a], zeta[a]);
    return rho * pr;
}

// g^eq_i = rho [ e prod_a PsiP_ia + sum_b PsiS_ib prod_{a!=b} PsiP_ia ], e = 3/2 RT,
// the operator form rho prod_a Psi_ia(O_a, O_a^2) E of Eq. (geq) evaluated with
// O^k_a 1 = (1, u, theta0 + u^2) and O^k_a (u^2/2) = (u^2/2, theta0 u + u^3/2,
// theta0^2 + 5/2 theta0 u^2 + u^4/2).
template <typename real, int Q>
__device__ __forceinline__ real geq_i(int i, real rho, const real *u, real theta0, real RT)
{
    constexpr int D = Lat<Q>::D;
    const real e = real(1.5) * RT;
    real PP[3], PS[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const real v = u[a];
        const real S0 = real(0.5) * v * v;
        const real S1 = theta0 * v + real(0.5) * v * v * v;
        const real S2 = theta0 * theta0 + real(2.5) * theta0 * v * v + real(0.5) * v * v * v * v;
        const int c = c_of(i, a, Q);
        PP[a] = psi_poly<real>(c, real(1.0), v, theta0 + v * v);
        PS[a] = psi_poly<real>(c, S0, S1, S2);
    }
    real pP = real(1.0);
#pragma unroll
    for (int a = 0; a < D; ++a) pP = pP * PP[a];
    real sS = real(0.0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
        real t = PS[b];
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (a != b) t = t * PP[a];
        sS = sS + t;
    }
    return rho * (e * pP + sS);
}

// ---------------------------------------------------------------------------
// Scratch fields of the stage kernels (each [N] unless noted).
// ---------------------------------------------------------------------------
template <typename real> struct RefFields {
    real *rho, *j /*[3][N]*/, *Gam;
    real *Pi /*[9][N]*/, *lap, *A;
    real *F /*[3][N]*/, *u /*[3][N]*/, *RT, *theta0, *P0, *gamma0, *flux /*[3][N]*/, *wq;
    real *m_in;           // mass streaming into each wall node this step (walls on)
    const real *RT_iso;   // frozen R*T field (thermal = 0)
};

// Initial populations f = f^eq(rho, u, theta0(rho, RT)), g = g^eq(rho, u, RT).
template <typename real, typename S, int Q>
__global__ void k_init(KParams p, const real *rho_in, const real *u_in, const real *RT_in, S *f, S *g, float *Rout)
{
    Node nd;
    if (!node_of(p, nd)) return;
    constexpr int D = Lat<Q>::D;
    const long long N = p.N, n = nd.n;
    const real rho = rho_in[n], RT = RT_in[n];
    real Z, g0;
    eos_Zg<real>(p.eos, p.thermal, real(p.b), rho, Z, g0);
    const real theta0 = RT * Z;
    real u[3] = {0, 0, 0}, zeta[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = u_in[a * N + n];
        zeta[a] = theta0 + u[a] * u[a];
    }
    EncTab tab{};
    if constexpr (Store<S>::dev) {
        const Ref16 r = make_rec(float(rho), float(u[0]), float(u[1]), float(u[2]), float(theta0), float(RT));
        store_rec(Rout, N, n, r);
        enc_tab<Q>(r, p.thermal != 0, tab);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const real v = prod_eq<real, Q>(i, rho, u, zeta);
        if constexpr (Store<S>::dev)
            Store<S>::store(f + i * N + n, encode_f<Q>(cx_of(i), cy_of(i), cz_of(i, Q), tab, float(v)));
        else Store<S>::store(f + i * N + n, v);
    }
    if (p.thermal) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const real v = geq_i<real, Q>(i, rho, u, theta0, RT);
            if constexpr (Store<S>::dev)
                Store<S>::store(g + i * N + n, encode_g<Q>(cx_of(i), cy_of(i), cz_of(i, Q), tab, float(v)));
            else Store<S>::store(g + i * N + n, v);
        }
    }
}

// Pulled populations h_i(x) = h~_i(x - c_i) of one node, f and (thermal) g.
template <typename real, typename S, int Q>
__device__ __forceinline__ void pull_node(const KParams &p, const Node &nd, const S *f, const S *g, const float *Rin,
                                          real *fo, real *go)
{
    const long long N = p.N;
    const bool wall = wall_col(p, nd.x);                 // a wall node keeps its own populations
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const long long src = wall ? nd.n : shifted(p, nd, -cx_of(i), -cy_of(i), -cz_of(i, Q));
        if constexpr (Store<S>::dev) {
            const Ref16 r = load_rec(Rin, N, src);
            fo[i] = decode_f<Q>(cx_of(i), cy_of(i), cz_of(i, Q), r, Store<S>::load(f + i * N + src));
            if (p.thermal)
                go[i] = decode_g<Q>(cx_of(i), cy_of(i), cz_of(i, Q), r, Store<S>::load(g + i * N + src));
        } else {
            fo[i] = real(Store<S>::load(f + i * N + src));
            if (p.thermal) go[i] = real(Store<S>::load(g + i * N + src));
        }
    }
}

// Stages 1-2: pull streaming f_i(x) = f~_i(x - c_i) and the raw moments
// rho = sum f_i, j_a = sum c_ia f_i, Gamma = sum g_i (ascending i).
template <typename real, typename S, int Q>
__global__ void k_moments(KParams p, const S *f, const S *g, const float *Rin, RefFields<real> w)
{
    Node nd;
    if (!node_of(p, nd)) return;
    constexpr int D = Lat<Q>::D;
    const long long N = p.N, n = nd.n;
    real fs[Q], gs[Q];
    pull_node<real, S, Q>(p, nd, f, g, Rin, fs, gs);
    real rho = real(0.0), j[3] = {real(0.0), real(0.0), real(0.0)}, Gam = real(0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const real fi = fs[i];
        rho = rho + fi;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int c = c_of(i, a, Q);
            if (c == 1) j[a] = j[a] + fi;
            else if (c == -1) j[a] = j[a] - fi;
        }
        if (p.thermal) Gam = Gam + gs[i];
    }
    w.rho[n] = rho;
#pragma unroll
    for (int a = 0; a < D; ++a) w.j[a * N + n] = j[a];
    w.Gam[n] = Gam;
    if (wall_col(p, nd.x)) {
        // Mass streaming into this wall node: the populations moving toward it (c_x = -1 at
        // x = 0, +1 at x = nx-1) pulled from the fluid, in ascending i.
        const int s = nd.x == 0 ? -1 : 1;
        real m = real(0.0);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (cx_of(i) == s) m = m + real(Store<S>::load(f + i * N + shifted(p, nd, -cx_of(i), -cy_of(i), -cz_of(i, Q))));
        w.m_in[n] = m;
    }
}

// Stage 3a: the Korteweg stress (divergence form) or the literal-form inputs.
//   Pi_ab = (-a rho^2 - kappa rho lap rho - 1/2 kappa |grad rho|^2) delta_ab + kappa d_a rho d_b rho
template <typename real, int Q>
__global__ void k_stress(KParams p, RefFields<real> w)
{
    Node nd;
    if (!node_of(p, nd)) return;
    constexpr int D = Lat<Q>::D;
    const long long N = p.N, n = nd.n;
    const real rho = w.rho[n];
    const real a = real(p.a), kappa = real(p.kappa);
    if (p.force_form == 0) {
        real gr[3];
#pragma unroll
        for (int d = 0; d < D; ++d) gr[d] = grad_iso<real, Q>(p, nd, w.rho, d);
        const real lr = lap_iso<real, Q>(p, nd, w.rho);
        real g2 = real(0.0);
#pragma unroll
        for (int d = 0; d < D; ++d) g2 = g2 + gr[d] * gr[d];
        const real s = -a * rho * rho - kappa * rho * lr - real(0.5) * kappa * g2;
#pragma unroll
        for (int d = 0; d < D; ++d)
#pragma unroll
            for (int e = 0; e < D; ++e) {
                const real t = kappa * gr[d] * gr[e];
                w.Pi[(d * 3 + e) * N + n] = (d == e) ? s + t : t;
            }
    } else {
        w.lap[n] = lap_iso<real, Q>(p, nd, w.rho);
        w.A[n] = a * rho * rho;
    }
}

// Stages 3b-5: force F (Enskog gauge: F = grad(a rho^2) + kappa rho grad(lap rho),
// Q~ = 0), shifted velocity (Eq. u_shift), energy, temperature, EOS, and the
// fields the gradient corrections differentiate.
template <typename real, int Q>
__global__ void k_macro(KParams p, RefFields<real> w)
{
    Node nd;
    if (!node_of(p, nd)) return;
    constexpr int D = Lat<Q>::D;
    const long long N = p.N, n = nd.n;
    const real rho = w.rho[n];
    real F[3] = {0, 0, 0}, u[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
        if (p.force_form == 0) {
            real div = real(0.0);
#pragma unroll
            for (int e = 0; e < D; ++e) div = div + grad_iso<real, Q>(p, nd, w.Pi + (d * 3 + e) * N, e);
            F[d] = -div;
        } else {
            F[d] = grad_iso<real, Q>(p, nd, w.A, d) + real(p.kappa) * rho * grad_iso<real, Q>(p, nd, w.lap, d);
        }
        if (wall_col(p, nd.x)) F[d] = real(0.0);           // no force on wall nodes
        u[d] = (w.j[d * N + n] + real(0.5) * F[d]) / rho;
    }
    real RT;
    if (p.thermal) {
        real uF = real(0.0), u2 = real(0.0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            uF = uF + u[d] * F[d];
            u2 = u2 + u[d] * u[d];
        }
        const real E = (w.Gam[n] + real(0.5) * uF) / rho;
        RT = real(2.0 / 3.0) * (E - real(0.5) * u2);
    } else {
        RT = w.RT_iso[n];
    }
    real Z, g0;
    eos_Zg<real>(p.eos, p.thermal, real(p.b), rho, Z, g0);
    const real theta0 = RT * Z;
    const real P0 = rho * theta0;
    w.RT[n] = RT;
    w.theta0[n] = theta0;
    w.P0[n] = P0;
    w.gamma0[n] = g0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        w.F[d * N + n] = F[d];
        w.u[d * N + n] = u[d];
        w.flux[d * N + n] = rho * u[d] * (u[d] * u[d] + real(3.0) * theta0 - real(1.0));
    }
    w.wq[n] = theta0 - RT;
}

// Stages 6-8: gradient corrections (Eqs. correction_u, correction_gamma,
// correction_q), equilibria (Eqs. feq, f_star, geq, gstar, g_corr) and the
// collision h~ = h + 2 beta (h^eq - h) + (dt/lambda)(1 - beta)(h* - h^eq).
template <typename real, typename S, int Q>
__global__ void k_collide(KParams p, RefFields<real> w, const S *f_src, const S *g_src, S *f_dst, S *g_dst,
                          const float *Rin, float *Rout)
{
    Node nd;
    if (!node_of(p, nd)) return;
    if (wall_col(p, nd.x)) return;                       // wall nodes: k_walls
    constexpr int D = Lat<Q>::D;
    const long long N = p.N, n = nd.n;
    const real lambda = real(p.lambda), c_eq = real(p.c_eq), c_star = real(p.c_star);
    const real rho = w.rho[n], RT = w.RT[n], theta0 = w.theta0[n], P0 = w.P0[n];
    real u[3] = {0, 0, 0}, F[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
        u[d] = w.u[d * N + n];
        F[d] = w.F[d * N + n];
    }
    real divu = real(0.0);
#pragma unroll
    for (int d = 0; d < D; ++d) divu = divu + diff_c<real>(p, nd, w.u + d * N, d);
    const real Phi1 = P0 * (real(5.0 / 3.0) - w.gamma0[n]) * divu;
    real Phi[3] = {0, 0, 0}, q[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
        // Phi_aa = Phi' - d_a[rho u_a (u_a^2 + 3 P0/rho - 1)]: the sign that cancels the
        // lattice bias c^3 = c of the third moment (Eq. correction_u).
        Phi[d] = Phi1 - diff_c<real>(p, nd, w.flux + d * N, d);
        q[d] = lambda * P0 * diff_c<real>(p, nd, w.wq, d) + lambda * u[d] * Phi1;
    }
    real us[3] = {0, 0, 0}, zeq[3] = {0, 0, 0}, zs[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
        us[d] = u[d] + lambda * F[d] / rho;
        zeq[d] = theta0 + u[d] * u[d];
        zs[d] = theta0 + us[d] * us[d] + lambda * Phi[d] / rho;
    }
    real fs[Q], gs[Q];
    pull_node<real, S, Q>(p, nd, f_src, g_src, Rin, fs, gs);
    EncTab tab{};
    if constexpr (Store<S>::dev) {
        const Ref16 r = make_rec(float(rho), float(u[0]), float(u[1]), float(u[2]), float(theta0), float(RT));
        store_rec(Rout, N, n, r);
        enc_tab<Q>(r, p.thermal != 0, tab);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const real h = fs[i];
        const real feq = prod_eq<real, Q>(i, rho, u, zeq);
        const real fst = prod_eq<real, Q>(i, rho, us, zs);
        const real v = h + c_eq * (feq - h) + c_star * (fst - feq);
        if constexpr (Store<S>::dev)
            Store<S>::store(f_dst + i * N + n, encode_f<Q>(cx_of(i), cy_of(i), cz_of(i, Q), tab, float(v)));
        else Store<S>::store(f_dst + i * N + n, v);
    }
    if (p.thermal) {
        real FF = real(0.0);
#pragma unroll
        for (int d = 0; d < D; ++d) FF = FF + F[d] * F[d];
        const real RTs = RT - lambda * lambda / (real(3.0) * rho * rho) * FF;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const real h = gs[i];
            const real geq = geq_i<real, Q>(i, rho, u, theta0, RT);
            real gst = geq_i<real, Q>(i, rho, us, theta0, RTs);
            const int c2 = cx_of(i) * cx_of(i) + cy_of(i) * cy_of(i) + cz_of(i, Q) * cz_of(i, Q);
            if (c2 == 1) {
                real cq = real(0.0);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const int c = c_of(i, d, Q);
                    if (c == 1) cq = cq + q[d];
                    else if (c == -1) cq = cq - q[d];
                }
                gst = gst + real(0.5) * cq;
            }
            const real v = h + c_eq * (geq - h) + c_star * (gst - geq);
            if constexpr (Store<S>::dev)
                Store<S>::store(g_dst + i * N + n, encode_g<Q>(cx_of(i), cy_of(i), cz_of(i, Q), tab, float(v)));
            else Store<S>::store(g_dst + i * N + n, v);
        }
    }
}

// Density rho_w of a wall node at temperature RT with P_E(rho_w, RT) = P: van der Waals
// form in closed form, rho = P / (RT + b P); Carnahan-Starling by sixteen Newton steps from
// the ideal-gas value P / RT, dP_E/drho = RT (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4)/(1 - eta)^4.
template <typename real>
__device__ __forceinline__ real wall_density(const KParams &p, real P, real RT)
{
    const real b = real(p.b);
    if (p.eos == 0) return P / (RT + b * P);
    real rho = P / RT;
    for (int k = 0; k < 16; ++k) {
        const real eta = b * rho / real(4.0);
        const real num = real(1.0) + eta + eta * eta - eta * eta * eta;
        const real om = real(1.0) - eta;
        const real Z = num / (om * om * om);
        const real dn = real(1.0) + real(4.0) * eta + real(4.0) * eta * eta - real(4.0) * eta * eta * eta +
                        eta * eta * eta * eta;
        rho = rho - (rho * RT * Z - P) / (RT * (dn / (om * om * om * om)));
    }
    return rho;
}

// Wall nodes after the collision (diffuse reflection): the equilibria at the wall velocity
// and temperature with the density rho_w that returns the absorbed mass m_in, P_E(rho_w) =
// 2 m_in (the populations leaving a wall with u_x = 0 carry rho_w theta0 / 2).  One thread
// per wall node: index k < 2 ny nz, side k % 2 (0: x = 0, 1: x = nx-1).  FP32/FP64 storage.
template <typename real, typename S, int Q>
__global__ void k_walls(KParams p, RefFields<real> w, S *f, S *g)
{
    constexpr int D = Lat<Q>::D;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2LL * p.ny * p.nz) return;
    const int side = (int)(k % 2);
    const long long row = k / 2;                          // y + ny z
    const long long N = p.N, n = row * p.nx + (side ? p.nx - 1 : 0);
    const real RT = real(p.wall_RT);
    const real rho = wall_density<real>(p, real(2.0) * w.m_in[n], RT);
    real Z, g0;
    eos_Zg<real>(p.eos, p.thermal, real(p.b), rho, Z, g0);
    const real theta0 = RT * Z;
    real u[3] = {0, 0, 0}, zeta[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = real(p.wall_u[side][a]);
        zeta[a] = theta0 + u[a] * u[a];
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) Store<S>::store(f + i * N + n, prod_eq<real, Q>(i, rho, u, zeta));
    if (p.thermal)
#pragma unroll
        for (int i = 0; i < Q; ++i) Store<S>::store(g + i * N + n, geq_i<real, Q>(i, rho, u, theta0, RT));
}

// Output of the macroscopic fields as FP32 (device) for callers that keep them on the GPU.
template <typename real, int Q>
__global__ void k_export_f32(KParams p, RefFields<real> w, double R, float *rho, float *u, float *T)
{
    Node nd;
    if (!node_of(p, nd)) return;
    constexpr int D = Lat<Q>::D;
    const long long N = p.N, n = nd.n;
    if (rho) rho[n] = float(w.rho[n]);
    if (T) T[n] = float(double(w.RT[n]) / R);
    if (u)
#pragma unroll
        for (int d = 0; d < D; ++d) u[d * N + n] = float(w.u[d * N + n]);
}

// Post-collision populations expanded to FP64 (16-bit storage adds the node's
// reference equilibrium back).
template <typename S, int Q>
__global__ void k_expand(KParams p, const S *src, const float *R, double *dst, int which)
{
    Node nd;
    if (!node_of(p, nd)) return;
    const long long N = p.N, n = nd.n;
    Ref16 r{};
    if constexpr (Store<S>::dev) r = load_rec(R, N, n);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        double v = double(Store<S>::load(src + i * N + n));
        if constexpr (Store<S>::dev)
            v = which == 0 ? double(decode_f<Q>(cx_of(i), cy_of(i), cz_of(i, Q), r, float(v)))
                           : double(decode_g<Q>(cx_of(i), cy_of(i), cz_of(i, Q), r, float(v)));
        dst[i * N + n] = v;
    }
}

}  // namespace evlbm

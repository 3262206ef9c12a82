// 16-bit population storage of the Enskog-Vlasov lattice Boltzmann step: each
// post-collision population h~_i(x) is stored in FP16 or BF16 as its deviation from
// the local equilibrium of the node x that wrote it, scaled by its lattice weight,
//   delta_i = (h~_i - f^eq_i(R)) / (w_i rho_R)              (f)
//   delta_i = (h~_i - g^eq_i(R)) / (w_i rho_R e_R)           (g, e = 3/2 RT)
// next to that node's reference record R = (rho, u_x, u_y, u_z, theta0, e) in FP32.
// The equilibria are those of Eqs. (feq) and (geq) evaluated at R; arithmetic is FP32.
//
// Records: a node's (rho, u_x, u_y, u_z) is one 16-byte word and its (theta0, e) one
// 8-byte word, in two arrays [N] (24 bytes per node), so that a puller fetches the
// reference of a source node with two vector loads.  Populations are [Q][N] of 2 bytes.
// Because the record holds the writer's own FP32 state, a writer that evaluates its
// equilibria with the functions below already has the references it must subtract.
//
// A puller must rebuild exactly the reference value the writer subtracted.  Every
// function below that enters a reference is written with explicit round-to-nearest
// intrinsics (no multiply-add contraction, no reassociation), so that all kernels
// that include this header -- whatever the compiler does around them -- produce the
// same bits from the same record.
#pragma once

#include "common.cuh"

namespace evlbm {

// Raw 16-bit values of the storage types (FP16, BF16) to and from FP32.
template <typename S> struct Bits16;
template <> struct Bits16<__half> {
    __device__ static __forceinline__ float to_f(unsigned short b) { return __half2float(__ushort_as_half(b)); }
    __device__ static __forceinline__ unsigned short from_f(float v) { return __half_as_ushort(__float2half_rn(v)); }
};
template <> struct Bits16<__nv_bfloat16> {
    __device__ static __forceinline__ float to_f(unsigned short b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
    __device__ static __forceinline__ unsigned short from_f(float v)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
};

// Reference state of a node.
struct Ref16 {
    float rho, u[3], th, e;
};

// Bytes of one node's record: (rho, u_x, u_y, u_z) in the first array, (theta0, e) in
// the second; a record buffer of N nodes holds kRecBytes * N bytes.
constexpr size_t kRecBytes = 4 * sizeof(float) + 2 * sizeof(float);

// Record of node n of a lattice of N nodes (read-only path).
__device__ __forceinline__ Ref16 load_rec(const float *R, long long N, long long n)
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(R) + n);
    const float2 b = __ldg(reinterpret_cast<const float2 *>(R + 4 * N) + n);
    return Ref16{a.x, {a.y, a.z, a.w}, b.x, b.y};
}

// The record a node writes for its state (rho, u, theta0, RT).
__device__ __forceinline__ Ref16 make_rec(float rho, float ux, float uy, float uz, float th, float RT)
{
    return Ref16{rho, {ux, uy, uz}, th, __fmul_rn(1.5f, RT)};
}

__device__ __forceinline__ void store_rec(float *R, long long N, long long n, const Ref16 &r)
{
    reinterpret_cast<float4 *>(R)[n] = make_float4(r.rho, r.u[0], r.u[1], r.u[2]);
    reinterpret_cast<float2 *>(R + 4 * N)[n] = make_float2(r.th, r.e);
}

// Per-axis factors of the equilibria at velocity component u (Eq. phi with
// xi = u, zeta = theta0 + u^2): P(c) = 1 - zeta (c = 0), (zeta +- u)/2 (c = +-1).
__device__ __forceinline__ float refP(int c, float u, float th)
{
    const float z = __fmaf_rn(u, u, th);
    return c == 0 ? __fadd_rn(1.f, -z) : __fmul_rn(0.5f, c > 0 ? __fadd_rn(z, u) : __fadd_rn(z, -u));
}

// The same linear combination applied to the energy moments (u^2/2, theta0 u + u^3/2,
// theta0^2 + 5/2 theta0 u^2 + u^4/2) (the closed form of Eq. geq).
__device__ __forceinline__ float refS(int c, float u, float th)
{
    const float u2 = __fmul_rn(u, u);
    const float S0 = __fmul_rn(0.5f, u2);
    const float S2 = __fmaf_rn(th, th, __fmul_rn(u2, __fmaf_rn(2.5f, th, S0)));
    if (c == 0) return __fadd_rn(S0, -S2);
    const float S1 = __fmul_rn(u, __fmaf_rn(0.5f, u2, th));
    return __fmul_rn(0.5f, c > 0 ? __fadd_rn(S2, S1) : __fadd_rn(S2, -S1));
}

// Lattice weight w_i of population (cx, cy, cz) as an FP32 constant (cz ignored for Q = 9).
template <int Q>
__host__ __device__ constexpr float wgt16(int cx, int cy, int cz)
{
    return Q == 9 ? float((cx ? 1.0 / 6.0 : 2.0 / 3.0) * (cy ? 1.0 / 6.0 : 2.0 / 3.0))
                  : float((cx ? 1.0 / 6.0 : 2.0 / 3.0) * (cy ? 1.0 / 6.0 : 2.0 / 3.0) * (cz ? 1.0 / 6.0 : 2.0 / 3.0));
}

// f^eq_i(R) = (rho P_x) (P_y P_z): the first factor per c_x, the second per (c_y, c_z).
// Writers that tabulate the factors must combine them in this order.
__device__ __forceinline__ float ref_f_of(float rPx, float PyPz) { return __fmul_rn(rPx, PyPz); }
// g^eq_i(R) = rho (e P_x + S_x) (P_y P_z) + (rho P_x) (S_y P_z + P_y S_z).
__device__ __forceinline__ float ref_g_of(float Ax, float rPx, float PyPz, float Dyz)
{
    return __fmaf_rn(Ax, PyPz, __fmul_rn(rPx, Dyz));
}
__device__ __forceinline__ float ref_A(float rho, float e, float Px, float Sx) { return __fmul_rn(rho, __fmaf_rn(e, Px, Sx)); }
__device__ __forceinline__ float ref_D(float Py, float Sy, float Pz, float Sz) { return __fmaf_rn(Sy, Pz, __fmul_rn(Py, Sz)); }

// Population i = (cx, cy, cz) of f rebuilt from a record and a stored deviation.
template <int Q>
__device__ __forceinline__ float decode_f(int cx, int cy, int cz, const Ref16 &r, float d)
{
    const float rPx = __fmul_rn(r.rho, refP(cx, r.u[0], r.th));
    const float PyPz = Q == 9 ? refP(cy, r.u[1], r.th) : __fmul_rn(refP(cy, r.u[1], r.th), refP(cz, r.u[2], r.th));
    return __fmaf_rn(__fmul_rn(wgt16<Q>(cx, cy, cz), r.rho), d, ref_f_of(rPx, PyPz));
}

template <int Q>
__device__ __forceinline__ float decode_g(int cx, int cy, int cz, const Ref16 &r, float d)
{
    const float Px = refP(cx, r.u[0], r.th), Py = refP(cy, r.u[1], r.th);
    const float Sx = refS(cx, r.u[0], r.th), Sy = refS(cy, r.u[1], r.th);
    float PyPz, Dyz;
    if (Q == 9) {
        PyPz = Py;
        Dyz = Sy;
    } else {
        const float Pz = refP(cz, r.u[2], r.th), Sz = refS(cz, r.u[2], r.th);
        PyPz = __fmul_rn(Py, Pz);
        Dyz = ref_D(Py, Sy, Pz, Sz);
    }
    const float ref = ref_g_of(ref_A(r.rho, r.e, Px, Sx), __fmul_rn(r.rho, Px), PyPz, Dyz);
    return __fmaf_rn(__fmul_rn(__fmul_rn(wgt16<Q>(cx, cy, cz), r.rho), r.e), d, ref);
}

// Both populations of one source node (shares the per-axis factors).
template <int Q>
__device__ __forceinline__ void decode_fg(int cx, int cy, int cz, const Ref16 &r, float df, float dg, float &hf,
                                          float &hg)
{
    const float Px = refP(cx, r.u[0], r.th), Py = refP(cy, r.u[1], r.th);
    const float Sx = refS(cx, r.u[0], r.th), Sy = refS(cy, r.u[1], r.th);
    float PyPz, Dyz;
    if (Q == 9) {
        PyPz = Py;
        Dyz = Sy;
    } else {
        const float Pz = refP(cz, r.u[2], r.th), Sz = refS(cz, r.u[2], r.th);
        PyPz = __fmul_rn(Py, Pz);
        Dyz = ref_D(Py, Sy, Pz, Sz);
    }
    const float rPx = __fmul_rn(r.rho, Px);
    const float ws = __fmul_rn(wgt16<Q>(cx, cy, cz), r.rho);
    hf = __fmaf_rn(ws, df, ref_f_of(rPx, PyPz));
    hg = __fmaf_rn(__fmul_rn(ws, r.e), dg, ref_g_of(ref_A(r.rho, r.e, Px, Sx), rPx, PyPz, Dyz));
}

// Encoding against a node's own record: the per-axis tables a writer builds once per
// node and the deviation of population (cx, cy, cz).
struct EncTab {
    float rP[3], A[3];          // rho P_x(c), rho (e P_x + S_x)(c), c = -1, 0, 1
    float P[2][3], S[2][3];     // P and S of the y and z axes
    float inv_f, inv_g;         // 1 / rho and 1 / (rho e)
};

template <int Q>
__device__ __forceinline__ void enc_tab(const Ref16 &r, bool thermal, EncTab &t)
{
#pragma unroll
    for (int c = -1; c <= 1; ++c) {
        const float Px = refP(c, r.u[0], r.th);
        t.rP[c + 1] = __fmul_rn(r.rho, Px);
        t.P[0][c + 1] = refP(c, r.u[1], r.th);
        t.P[1][c + 1] = Q == 9 ? 1.f : refP(c, r.u[2], r.th);
        if (thermal) {
            t.A[c + 1] = ref_A(r.rho, r.e, Px, refS(c, r.u[0], r.th));
            t.S[0][c + 1] = refS(c, r.u[1], r.th);
            t.S[1][c + 1] = Q == 9 ? 0.f : refS(c, r.u[2], r.th);
        }
    }
    t.inv_f = 1.f / r.rho;
    t.inv_g = thermal ? 1.f / (r.rho * r.e) : 0.f;
}

// 1 / w_i as a product of the exact binary factors 3/2 (c = 0) and 6 (c = +-1).
template <int Q>
__host__ __device__ constexpr float inv_wq(int cx, int cy, int cz)
{
    return Q == 9 ? (cx ? 6.f : 1.5f) * (cy ? 6.f : 1.5f)
                  : (cx ? 6.f : 1.5f) * (cy ? 6.f : 1.5f) * (cz ? 6.f : 1.5f);
}

template <int Q>
__device__ __forceinline__ float encode_f(int cx, int cy, int cz, const EncTab &t, float v)
{
    const float PyPz = Q == 9 ? t.P[0][cy + 1] : __fmul_rn(t.P[0][cy + 1], t.P[1][cz + 1]);
    return (v - ref_f_of(t.rP[cx + 1], PyPz)) * (t.inv_f * inv_wq<Q>(cx, cy, cz));
}

template <int Q>
__device__ __forceinline__ float encode_g(int cx, int cy, int cz, const EncTab &t, float v)
{
    float PyPz, Dyz;
    if (Q == 9) {
        PyPz = t.P[0][cy + 1];
        Dyz = t.S[0][cy + 1];
    } else {
        PyPz = __fmul_rn(t.P[0][cy + 1], t.P[1][cz + 1]);
        Dyz = ref_D(t.P[0][cy + 1], t.S[0][cy + 1], t.P[1][cz + 1], t.S[1][cz + 1]);
    }
    return (v - ref_g_of(t.A[cx + 1], t.rP[cx + 1], PyPz, Dyz)) * (t.inv_g * inv_wq<Q>(cx, cy, cz));
}

}  // namespace evlbm

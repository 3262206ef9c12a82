// Shared device-side definitions of the Enskog-Vlasov lattice Boltzmann kernels
// (Karlin & Hosseini, arXiv 2508.00577).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace evlbm {

// Kernel-side copy of the model parameters (passed by value).
struct KParams {
    int nx, ny, nz;
    long long N;         // nx*ny*nz
    int eos;             // 0 vdW form of P_E, 1 Carnahan-Starling
    int thermal;         // 1: f and g; 0: frozen temperature
    int force_form;      // 0 divergence (Korteweg stress), 1 literal
    double a, b, kappa, lambda;
    double c_eq;         // 2 beta
    double c_star;       // (dt/lambda)(1 - beta)
    int tile_w, tile_h;  // launch shape of the fused kernel (0 = default)
    int walls;           // 1: the columns x = 0 and x = nx-1 are wall nodes (lbm_set_walls)
    double wall_u[2][3]; // velocity of the wall at x = 0 and at x = nx-1
    double wall_RT;      // R T_w of both walls
};

// Wall nodes (the thermal Couette set-up: u and T prescribed at x = 0 and x = L_x; the
// paper gives no wall scheme, the reading here is a diffusely reflecting wall): with walls
// on, the columns x = 0 and x = nx-1 do not stream (their moments are those of their own
// populations), carry no force and do not collide; they absorb the populations streaming
// into them (mass m) and their populations become the equilibria f^eq(rho_w, u_w,
// theta0(rho_w, R T_w)), g^eq(rho_w, u_w, R T_w) (Eqs. feq, geq) with P_E(rho_w, R T_w) = 2 m,
// which returns the absorbed mass to the fluid.
__host__ __device__ inline bool wall_col(const KParams &p, int x) { return p.walls && (x == 0 || x == p.nx - 1); }

// Velocity set: i = (cx+1) + 3(cy+1) + 9(cz+1).
__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i, int Q) { return Q == 27 ? i / 9 - 1 : 0; }

// 1-D weights of the product lattice: the rest equilibrium Psi(0, 1/3) per axis.
__host__ __device__ constexpr double w1_of(int c) { return c == 0 ? (2.0 / 3.0) : (1.0 / 6.0); }

// Lattice weight w_i as the product of the 1-D weights, multiplied in axis order.
__host__ __device__ constexpr double w_of(int i, int Q)
{
    return Q == 9 ? (1.0 * w1_of(cx_of(i))) * w1_of(cy_of(i))
                  : ((1.0 * w1_of(cx_of(i))) * w1_of(cy_of(i))) * w1_of(cz_of(i, Q));
}

// ---------------------------------------------------------------------------
// Population storage.  FP64/FP32 store the population itself; FP16/BF16 store
// the deviation f_i - w_i * ref from the rest equilibrium of a reference state.
// ---------------------------------------------------------------------------
template <typename S> struct Store;

template <> struct Store<double> {
    static constexpr bool dev = false;
    __device__ static __forceinline__ double load(const double *p) { return __ldg(p); }
    __device__ static __forceinline__ void store(double *p, double v) { *p = v; }
};
template <> struct Store<float> {
    static constexpr bool dev = false;
    __device__ static __forceinline__ float load(const float *p) { return __ldg(p); }
    __device__ static __forceinline__ void store(float *p, float v) { *p = v; }
};
template <> struct Store<__half> {
    static constexpr bool dev = true;
    // Value after a round trip through the storage format (registers only).
    __device__ static __forceinline__ float round(float v) { return __half2float(__float2half_rn(v)); }
    __device__ static __forceinline__ float load(const __half *p) { return __half2float(__ldg(p)); }
    __device__ static __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr bool dev = true;
    __device__ static __forceinline__ float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    __device__ static __forceinline__ float load(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    __device__ static __forceinline__ void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// Periodic neighbour index of node (x, y, z) shifted by (dx, dy, dz) with |d| <= 1.
__device__ __forceinline__ int wrap1(int v, int n)
{
    v = v < 0 ? v + n : v;
    return v >= n ? v - n : v;
}

}  // namespace evlbm

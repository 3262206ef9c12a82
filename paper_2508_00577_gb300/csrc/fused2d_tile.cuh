// Tile body of the fused single-pass D2Q9 step of the Enskog-Vlasov lattice
// Boltzmann model (Karlin & Hosseini, arXiv 2508.00577), FP32 arithmetic with FP32
// storage or FP16 / BF16 deviation storage (dev16.cuh); used by the per-step kernels
// (fused2d_launch.cuh, instantiated in fused2d.cu and fused2d16.cu) and, FP32 only, the
// persistent batched driver (batch.cu).
//
// One kernel does the whole step of Eq. (pre_LBM): pull streaming, raw moments,
// the Enskog-gauge force F = grad(a rho^2) + kappa rho grad(lap rho) in
// divergence (Korteweg-stress) form, the shifted velocity and energy
// (Eqs. u_shift, T_shift), the EOS and gamma0 (Eq. gamma), the gradient
// corrections Phi, Phi', q' (Eqs. correction_u/gamma/q), the equilibria
// (Eqs. feq, f_star, geq, gstar, g_corr) and the collision.
//
// Work decomposition.  A CTA owns a strip of W output columns of one 2-D layer
// and marches down a chunk of H rows, two rows per iteration: every value a
// thread handles is a float2 holding the same quantity on rows (2q, 2q+1) of
// its column, and the arithmetic runs on Blackwell's packed FP32x2 units.  The
// force needs rho within radius 2 of every node whose velocity is needed, and
// the corrections need u, T within radius 1 of the collided node, so four
// stages lag each other by one row pair.  For the leading pair q:
//   A: rho, j (q)              pulled populations                 (W + 6 columns)
//   B: Korteweg stress (q-1)   from rho of pairs q-2..q            (W + 4 columns)
//   C: F, u, T, EOS (q-2)      div Pi of pairs q-3..q-1, Gamma     (W + 2 columns)
//   D: collide (q-3)           Phi, q' from the fields of q-4..q-2 (W columns)
// Fields shared between columns live in 3-deep shared-memory rings of row
// pairs; the pulled f (stage A -> D) and the pulled g (C -> D) of a column live in
// thread-private shared-memory rings, its centre values (C -> D) in a one-pair slot
// that the thread reads before it rewrites it.  Shared memory stays under 97 KiB per
// CTA so that two CTAs leave the L1 60 KB: every global load in flight holds L1
// space, and a 28 KB L1 caps the loads in flight well below HBM bandwidth.  The 6
// halo columns of a strip belong to an extra warp that runs stages A-C only.
// Loads of the next f and g rows are issued one iteration ahead.  Every
// population is read from HBM once per step; re-reads of halo columns are
// served by L2.
#pragma once

#include "bounds.cuh"
#include "dev16.cuh"
#include "dispatch.h"

namespace evlbm {
namespace fused {

// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic.
// ---------------------------------------------------------------------------
typedef float2 v2;
__device__ __forceinline__ v2 V(float a) { return make_float2(a, a); }
__device__ __forceinline__ v2 V(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ v2 operator+(v2 a, v2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ v2 operator*(v2 a, v2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ v2 operator-(v2 a, v2 b) { return __ffma2_rn(b, V(-1.f), a); }
__device__ __forceinline__ v2 operator-(v2 a) { return __fmul2_rn(a, V(-1.f)); }
__device__ __forceinline__ v2 fma2(v2 a, v2 b, v2 c) { return __ffma2_rn(a, b, c); }
// Reciprocal with the hardware approximation (rcp.approx.ftz: at most 1 ulp, relative
// error below 2^-22); the operands (rho, 1 - b rho, EOS polynomials) are normal numbers.
__device__ __forceinline__ float rcpa(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ v2 rcp2(v2 a) { return V(rcpa(a.x), rcpa(a.y)); }
// (lo.y, hi.x): the row pair shifted by one row.
__device__ __forceinline__ v2 shift_up(v2 lo, v2 hi) { return V(lo.y, hi.x); }

constexpr int kFields = 11;      // rho, jx, jy, Pxx, Pxy, Pyy, ux, uy, flux_x, flux_y, wq
constexpr int kDepth = 3;        // ring depth (row pairs) of the shared fields
constexpr int kCentre = 6;       // rho, Fx, Fy, RT, theta0, gamma0 handed from stage C to D

// Strip of W output columns: W + 32 threads (the last warp owns the 6 halo
// columns), MINB resident CTAs per SM requested from the compiler.
template <int W> struct Shape;
template <> struct Shape<64> { static constexpr int MINB = 4; };
template <> struct Shape<96> { static constexpr int MINB = 2; };
template <> struct Shape<128> { static constexpr int MINB = 2; };
template <> struct Shape<192> { static constexpr int MINB = 1; };

template <int W> constexpr int threads_of() { return W + 32; }
template <int W> constexpr int slots_of() { return W + 6; }
template <int W> constexpr size_t smem_of()
{
    return sizeof(v2) * (size_t)(kFields * kDepth * slots_of<W>() + (4 * 9 + 2 * 9 + kCentre) * W);
}

struct FusedArgs {
    const float *f, *g;          // FP32 populations, or the raw 16-bit deviations (16-bit storage)
    float *fo, *go;
    const float *Rin;            // 16-bit storage: reference records read (dev16.cuh) ...
    float *Rout;                 // ... and written
    const float *RT_iso;
    int nx, ny, nz, H;
    unsigned N;                  // nodes of the lattice (Q*N < 2^31)
    int eos;
    float a, b, kappa, lambda, c_eq, c_star;
    int walls;                   // 1: the columns x = 0 and x = nx-1 are wall nodes (KParams::walls)
    float wall_uy[2], wall_RT;   // wall velocities (along y) and R T_w
};

__device__ __forceinline__ int wrap_any(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}
__device__ __forceinline__ int prev_row(int r, int ny) { return r == 0 ? ny - 1 : r - 1; }
__device__ __forceinline__ int next_row(int r, int ny) { return r == ny - 1 ? 0 : r + 1; }

// CG: the populations were written earlier in the same launch (persistent ensemble kernel),
// so the read-only path (ld.global.nc) is not allowed.  A plain L1-cached load (ld.global.ca)
// is: the CTA reads them only after thread 0's gpu-scope acquire of the domain's completion
// counter (which pairs with the producers' fence + atomic release) and a CTA barrier, and an
// acquire at gpu scope makes every later load of the CTA observe the released writes.
template <bool CG> __device__ __forceinline__ float ldpop(const float *p) { return CG ? __ldca(p) : __ldg(p); }

// Pulled populations of rows (r, r+1) of one column: h_i(y) = h~_i(x - c_ix, y - c_iy).
// ro[k] = offset of wrapped row r - 1 + k (k = 0..3), cols[k] = wrapped column x - 1 + k.
template <bool CG>
__device__ __forceinline__ void pull18(const float *__restrict__ base, unsigned N, const unsigned ro[4],
                                       const int cols[3], v2 h[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = i % 3 - 1, cy = i / 3 - 1;
        const float *p = base + i * N + cols[1 - cx];
        const float *p0 = p + ro[1 - cy], *p1 = p + ro[2 - cy];
        h[i] = V(in_bounds(p0 - base, 9ull * N) ? ldpop<CG>(p0) : 0.f, in_bounds(p1 - base, 9ull * N) ? ldpop<CG>(p1) : 0.f);
    }
}

// A wall column's own populations of rows (r, r+1): wall nodes do not stream.
template <bool CG>
__device__ __forceinline__ void pull_own(const float *__restrict__ base, unsigned N, const unsigned ro[4], int col,
                                         v2 h[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float *p = base + i * N + col;
        const float *p0 = p + ro[1], *p1 = p + ro[2];
        h[i] = V(in_bounds(p0 - base, 9ull * N) ? ldpop<CG>(p0) : 0.f, in_bounds(p1 - base, 9ull * N) ? ldpop<CG>(p1) : 0.f);
    }
}

// Store of one encoded 16-bit deviation (streaming: not read again this step).
template <typename S> __device__ __forceinline__ void st16(float *base, unsigned idx, float v)
{
    __stcs(reinterpret_cast<unsigned short *>(base) + idx, Bits16<S>::from_f(v));
}

// 16-bit storage: the pulled populations of rows (r, r+1) of one column, each rebuilt from
// its source node's reference record and its stored deviation (G: energy populations).
template <typename S, bool G>
__device__ __forceinline__ void pull18_dev(const float *base_, const float *R, unsigned N, const unsigned ro[4],
                                           const int cols[3], v2 h[9])
{
    const unsigned short *base = reinterpret_cast<const unsigned short *>(base_);
    auto one = [&](int cx, int cy, unsigned i, unsigned n) {
        if (!(in_bounds(i * N + n, 9ull * N) && in_bounds(n, N))) return 0.f;
        const float d = Bits16<S>::to_f(__ldg(base + i * N + n));
        const Ref16 r = load_rec(R, N, n);
        return G ? decode_g<9>(cx, cy, 0, r, d) : decode_f<9>(cx, cy, 0, r, d);
    };
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = i % 3 - 1, cy = i / 3 - 1;
        h[i] = V(one(cx, cy, i, ro[1 - cy] + cols[1 - cx]), one(cx, cy, i, ro[2 - cy] + cols[1 - cx]));
    }
}

__device__ __forceinline__ v2 sum9(const v2 h[9])
{
    return ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
}

// One tile: rows y0 .. y0 + rows - 1 (y0 even, y0 + rows <= ny) of strip bx of layer
// bz.  smem holds smem_of<kW>() bytes.  CG selects loads that may see populations
// written by other CTAs of the same launch.  A CTA that runs several tiles must pass a
// barrier between them (the rings are reused).  WALLS compiles in the wall columns
// (FusedArgs::walls); without it the kernel has no trace of them.
template <int kW, bool THERMAL, bool CG, bool WALLS = false, typename ST = float>
__device__ __forceinline__ void fused_tile(const FusedArgs &A, int bx, int y0, int rows, int bz, v2 *smem)
{
    // 16-bit deviation storage (ST = __half / __nv_bfloat16): pulls decode, stage D encodes
    // against the node's new reference record (dev16.cuh); no wall columns, no ensemble.
    constexpr bool DEV = Store<ST>::dev;
    static_assert(!(DEV && (WALLS || CG)), "16-bit storage runs the single-lattice kernel without walls");
    constexpr int S = slots_of<kW>();
    enum { RHO, JX, JY, PXX, PXY, PYY, UX, UY, QX, QY, WQ };
    auto fld = [&](int field, int slot3) -> v2 * { return smem + (field * kDepth + slot3) * S; };
    v2 *const f9 = smem + kFields * kDepth * S;          // [4][9][kW]   pulled f, stage A -> D
    v2 *const g9 = f9 + 4 * 9 * kW;                      // [2][9][kW]   pulled g, stage C -> D
    v2 *const cen = g9 + 2 * 9 * kW;                     // [kCentre][kW]: one pair, read before rewritten

    const int nx = A.nx, ny = A.ny;
    const int t = threadIdx.x;
    const int x0 = bx * kW;
    const int Weff = min(kW, nx - x0);
    const int Heff = rows;
    const unsigned layer = (unsigned)bz * (unsigned)nx * (unsigned)ny;

    // Column role.
    int slot = 0, col = 0;
    bool inA = true, inB = true, inC = true, inD = true;
    if (t < kW) {
        slot = t + 3;
        col = x0 + t;
        if (t >= Weff) inA = inB = inC = inD = false;
    } else {
        const int h = t - kW;
        inD = false;
        if (h < 3) {
            slot = h;
            col = x0 - 3 + h;
            inB = h >= 1;
            inC = h == 2;
        } else if (h < 6) {
            slot = Weff + h;
            col = x0 + Weff + (h - 3);
            inB = h <= 4;
            inC = h == 3;
        } else {
            inA = inB = inC = false;
        }
    }
    int cols[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) cols[k] = wrap_any(col - 1 + k, nx);
    // Wall column (x = 0 or nx-1 with walls on): no streaming, no force, no collision.
    const bool wallc = WALLS && A.walls && (cols[1] == 0 || cols[1] == nx - 1);
    // Shared rings: stages B and C read slot +- 1, stage D the thread-private rings at t.
    // A thread that fails the check does no work but still reaches every barrier.
    if (!in_bounds(slot, S) || ((inB || inC) && !(in_bounds(slot - 1, S) && in_bounds(slot + 1, S))) ||
        (inD && !in_bounds(t, kW)))
        inA = inB = inC = inD = false;

    const float a = A.a, b = A.b, kappa = A.kappa, lambda = A.lambda;
    const unsigned N = A.N;
    // gp: energy populations (the decoding of 16-bit storage differs).
    auto pull = [&](const float *base, const unsigned ro[4], v2 h[9], bool gp) {
        if constexpr (DEV) {
            if (gp) pull18_dev<ST, true>(base, A.Rin, N, ro, cols, h);
            else pull18_dev<ST, false>(base, A.Rin, N, ro, cols, h);
        } else if (wallc) {
            pull_own<CG>(base, N, ro, cols[1], h);
        } else {
            pull18<CG>(base, N, ro, cols, h);
        }
    };
    auto rows4 = [&](int r, unsigned ro[4]) {      // rows r-1 .. r+2 of the layer
        const int rp = next_row(r, ny);
        ro[0] = layer + (unsigned)prev_row(r, ny) * nx;
        ro[1] = layer + (unsigned)r * nx;
        ro[2] = layer + (unsigned)rp * nx;
        ro[3] = layer + (unsigned)next_row(rp, ny) * nx;
    };

    // Pair indices: pair q holds rows 2q, 2q+1 (absolute, unwrapped).
    const int q0 = y0 / 2;
    const int qD_end = (y0 + Heff + 1) / 2;              // one past the last collided pair
    const int qbeg = q0 - 3, qend = qD_end + 2;
    int rA = wrap_any(2 * qbeg, ny);                      // wrapped first row of the next A pair
    int rC = wrap_any(2 * (q0 - 1), ny);                  // ... of the next C pair
    int rD = wrap_any(2 * q0, ny);                        // ... of the next D pair
    int s0 = ((qbeg % 3) + 3) % 3;                        // ring slot of pair q

    v2 pf[9], pg[9];
    if (inA) {
        unsigned ro[4];
        rows4(rA, ro);
        pull(A.f, ro, pf, false);
    }
    if (THERMAL && inC) {
        unsigned ro[4];
        rows4(rC, ro);
        pull(A.g, ro, pg, true);
    }

    for (int q = qbeg; q <= qend; ++q) {
        const int sm1 = s0 == 0 ? 2 : s0 - 1;             // slot of q-1 (and of q-4)
        const int sm2 = s0 == 2 ? 0 : s0 + 1;             // slot of q-2 (q-3 shares s0)
        // ---------------- A: rho, j of pair q ----------------
        if (inA) {
            fld(RHO, s0)[slot] = sum9(pf);
            fld(JX, s0)[slot] = ((pf[2] + pf[5]) + pf[8]) - ((pf[0] + pf[3]) + pf[6]);
            fld(JY, s0)[slot] = ((pf[6] + pf[7]) + pf[8]) - ((pf[0] + pf[1]) + pf[2]);
            if (inD) {
                v2 *fr = f9 + (q & 3) * 9 * kW + t;
                if (WALLS && wallc) {
                    // A wall column keeps, for stage D, the mass streaming into it: the three
                    // populations moving toward it, pulled from the fluid column next to it.
                    unsigned ro[4];
                    rows4(rA, ro);
                    const int s = cols[1] == 0 ? -1 : 1;
                    v2 m = V(0.f);
#pragma unroll
                    for (int cy = -1; cy <= 1; ++cy) {
                        const int i = (s + 1) + 3 * (cy + 1);
                        const float *pp = A.f + i * N + cols[1 - s];
                        const float *p0 = pp + ro[1 - cy], *p1 = pp + ro[2 - cy];
                        m = m + V(in_bounds(p0 - A.f, 9ull * N) ? ldpop<CG>(p0) : 0.f,
                                  in_bounds(p1 - A.f, 9ull * N) ? ldpop<CG>(p1) : 0.f);
                    }
                    fr[0] = m;
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) fr[i * kW] = pf[i];
                }
            }
            rA = next_row(next_row(rA, ny), ny);
            if (q < qend) {
                unsigned ro[4];
                rows4(rA, ro);
                pull(A.f, ro, pf, false);
            }
        }
        __syncthreads();

        // ---------------- B: Korteweg stress of pair q-1 ----------------
        if (inB && q - 1 >= q0 - 2) {
            const v2 *r2 = fld(RHO, sm2), *r1 = fld(RHO, sm1), *r0 = fld(RHO, s0);
            const v2 aW = r2[slot - 1], aC = r2[slot], aE = r2[slot + 1];     // pair q-2
            const v2 bW = r1[slot - 1], bC = r1[slot], bE = r1[slot + 1];     // pair q-1 (centre rows)
            const v2 cW = r0[slot - 1], cC = r0[slot], cE = r0[slot + 1];     // pair q
            const v2 SW = shift_up(aW, bW), S_ = shift_up(aC, bC), SE = shift_up(aE, bE);
            const v2 NW = shift_up(bW, cW), N_ = shift_up(bC, cC), NE = shift_up(bE, cE);
            // Isotropic D2Q9 stencils: grad = 3 sum w c phi, lap = 6 sum w (phi - phi_0).
            const v2 dx = fma2(V(1.f / 3.f), bE - bW, V(1.f / 12.f) * ((NE - NW) + (SE - SW)));
            const v2 dy = fma2(V(1.f / 3.f), N_ - S_, V(1.f / 12.f) * ((NE + NW) - (SE + SW)));
            const v2 lap = fma2(V(2.f / 3.f), (bE + bW) + (N_ + S_),
                                fma2(V(1.f / 6.f), (NE + NW) + (SE + SW), V(-10.f / 3.f) * bC));
            const v2 kdx = V(kappa) * dx, kdy = V(kappa) * dy;
            // s = -a rho^2 - kappa rho lap - kappa/2 |grad rho|^2
            const v2 s = -(fma2(V(a) * bC, bC, fma2(V(kappa) * bC, lap, V(0.5f) * fma2(kdx, dx, kdy * dy))));
            fld(PXX, sm1)[slot] = fma2(kdx, dx, s);
            fld(PXY, sm1)[slot] = kdx * dy;
            fld(PYY, sm1)[slot] = fma2(kdy, dy, s);
        }
        __syncthreads();

        // ---------------- C: force, velocity, temperature, EOS of pair q-2 ----------------
        v2 cprev[kCentre];                                 // centre values of pair q-3 (stage D)
        if (inC && q - 2 >= q0 - 1) {
            // Pi of pairs q-3 (slot s0), q-2 (sm2, centre rows), q-1 (sm1).
            const int sw = slot - 1, se = slot + 1;
            const v2 *x3 = fld(PXX, s0), *x2 = fld(PXX, sm2), *x1 = fld(PXX, sm1);
            const v2 *y3 = fld(PXY, s0), *y2 = fld(PXY, sm2), *y1 = fld(PXY, sm1);
            const v2 *z3 = fld(PYY, s0), *z2 = fld(PYY, sm2), *z1 = fld(PYY, sm1);
            auto south = [&](const v2 *lo, const v2 *c, int k) { return shift_up(lo[k], c[k]); };
            auto north = [&](const v2 *c, const v2 *hi, int k) { return shift_up(c[k], hi[k]); };
            const v2 dxPxx = fma2(V(1.f / 3.f), x2[se] - x2[sw],
                                  V(1.f / 12.f) * ((north(x2, x1, se) - north(x2, x1, sw)) +
                                                   (south(x3, x2, se) - south(x3, x2, sw))));
            const v2 yE = y2[se], yW = y2[sw];
            const v2 yNE = north(y2, y1, se), yNW = north(y2, y1, sw), yN = north(y2, y1, slot);
            const v2 ySE = south(y3, y2, se), ySW = south(y3, y2, sw), yS = south(y3, y2, slot);
            const v2 dyPxy = fma2(V(1.f / 3.f), yN - yS, V(1.f / 12.f) * ((yNE + yNW) - (ySE + ySW)));
            const v2 dxPxy = fma2(V(1.f / 3.f), yE - yW, V(1.f / 12.f) * ((yNE - yNW) + (ySE - ySW)));
            const v2 dyPyy = fma2(V(1.f / 3.f), north(z2, z1, slot) - south(z3, z2, slot),
                                  V(1.f / 12.f) * ((north(z2, z1, se) + north(z2, z1, sw)) -
                                                   (south(z3, z2, se) + south(z3, z2, sw))));
            const v2 Fx = wallc ? V(0.f) : -(dxPxx + dyPxy), Fy = wallc ? V(0.f) : -(dxPxy + dyPyy);
            const v2 rho = fld(RHO, sm2)[slot];
            const v2 ir = rcp2(rho);
            const v2 ux = fma2(V(0.5f), Fx, fld(JX, sm2)[slot]) * ir;
            const v2 uy = fma2(V(0.5f), Fy, fld(JY, sm2)[slot]) * ir;
            v2 RT;
            if constexpr (THERMAL) {
                const v2 Gam = sum9(pg);
                const v2 E = fma2(V(0.5f), fma2(ux, Fx, uy * Fy), Gam) * ir;
                RT = V(2.f / 3.f) * fma2(V(-0.5f), fma2(ux, ux, uy * uy), E);
                if (inD) {
                    v2 *gr = g9 + (q & 1) * 9 * kW + t;
#pragma unroll
                    for (int i = 0; i < 9; ++i) gr[i * kW] = pg[i];
                }
                rC = next_row(next_row(rC, ny), ny);
                if (q + 1 <= qend) {           // prefetch the next stage-C pair
                    unsigned ro[4];
                    rows4(rC, ro);
                    pull(A.g, ro, pg, true);
                }
            } else {
                const float *Tp = A.RT_iso + layer + cols[1];
                const float *T0 = Tp + (unsigned)rC * nx, *T1 = Tp + (unsigned)next_row(rC, ny) * nx;
                RT = V(in_bounds(T0 - A.RT_iso, N) ? ldpop<CG>(T0) : 0.f, in_bounds(T1 - A.RT_iso, N) ? ldpop<CG>(T1) : 0.f);
                rC = next_row(next_row(rC, ny), ny);
            }
            // EOS in the Enskog gauge: P0 = P_E = rho RT Z, gamma0 = 1 + rho Z'/Z [+ 2/3 Z].
            v2 Z, dlnZ;
            if (A.eos == 0) {
                const v2 br = V(b) * rho;
                Z = rcp2(V(1.f) - br);
                dlnZ = br * Z;
            } else {
                const v2 eta = V(0.25f * b) * rho;
                const v2 num = fma2(eta, fma2(eta, V(1.f) - eta, V(1.f)), V(1.f));
                const v2 iom = rcp2(V(1.f) - eta);
                Z = num * (iom * iom) * iom;
                dlnZ = eta * fma2(eta, fma2(V(-2.f), eta, V(4.f)), V(4.f)) * iom * rcp2(num);
            }
            const v2 g0 = THERMAL ? fma2(V(2.f / 3.f), Z, V(1.f) + dlnZ) : V(1.f) + dlnZ;
            const v2 th = RT * Z;
            const v2 th3m1 = fma2(V(3.f), th, V(-1.f));
            fld(UX, sm2)[slot] = ux;
            fld(UY, sm2)[slot] = uy;
            fld(QX, sm2)[slot] = rho * ux * fma2(ux, ux, th3m1);
            fld(QY, sm2)[slot] = rho * uy * fma2(uy, uy, th3m1);
            fld(WQ, sm2)[slot] = th - RT;
            if (inD) {
                // The slot still holds pair q-3, which stage D collides later in this
                // iteration: take it into registers before storing pair q-2.
                v2 *cr = cen + t;
#pragma unroll
                for (int k = 0; k < kCentre; ++k) cprev[k] = cr[k * kW];
                cr[0 * kW] = rho; cr[1 * kW] = Fx; cr[2 * kW] = Fy;
                cr[3 * kW] = RT; cr[4 * kW] = th; cr[5 * kW] = g0;
            }
        }
        __syncthreads();

        // ---------------- D: collide pair q-3 ----------------
        if (inD && q - 3 >= q0 && wallc) {
            // Wall nodes (diffuse reflection): the equilibria at the wall velocity (0, U_w) and
            // temperature R T_w (Eqs. feq, geq) with the density rho_w that returns the mass m
            // that streamed in, P_E(rho_w, R T_w) = 2 m.
            const int p = q - 3;
            const v2 P = V(2.f) * f9[(p & 3) * 9 * kW + t];
            const float U = cols[1] == 0 ? A.wall_uy[0] : A.wall_uy[1], RTw = A.wall_RT;
            v2 rho, Z;
            if (A.eos == 0) {
                rho = P * rcp2(fma2(V(b), P, V(RTw)));             // P / (RT + b P)
                Z = rcp2(V(1.f) - V(b) * rho);
            } else {
                // Newton on rho RT Z(eta) = P, dP_E/drho = RT (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4)/(1 - eta)^4
                rho = P * V(1.f / RTw);
                for (int k = 0; k < 16; ++k) {
                    const v2 eta = V(0.25f * b) * rho;
                    const v2 num = fma2(eta, fma2(eta, V(1.f) - eta, V(1.f)), V(1.f));
                    const v2 iom = rcp2(V(1.f) - eta);
                    const v2 z = num * (iom * iom) * iom;
                    const v2 dn = fma2(eta, fma2(eta, fma2(eta, eta - V(4.f), V(4.f)), V(4.f)), V(1.f));
                    rho = rho - (fma2(rho * V(RTw), z, -P)) * rcp2(V(RTw) * dn * ((iom * iom) * (iom * iom)));
                }
                const v2 eta = V(0.25f * b) * rho;
                const v2 num = fma2(eta, fma2(eta, V(1.f) - eta, V(1.f)), V(1.f));
                const v2 iom = rcp2(V(1.f) - eta);
                Z = num * (iom * iom) * iom;
            }
            const v2 th = V(RTw) * Z;
            const v2 hr = V(0.5f) * rho;
            const v2 zey = th + V(U * U);
            const v2 ex[3] = {hr * th, rho - rho * th, hr * th};
            const v2 ey[3] = {V(0.5f) * (zey - V(U)), V(1.f) - zey, V(0.5f) * (zey + V(U))};
            const unsigned out0 = layer + (unsigned)rD * nx + cols[1];
            const unsigned out1 = layer + (unsigned)next_row(rD, ny) * nx + cols[1];
            const bool second = 2 * p + 1 < y0 + Heff;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const v2 o = ex[i % 3] * ey[i / 3];
                if (in_bounds(i * N + out0, 9ull * N)) A.fo[i * N + out0] = o.x;
                if (second && in_bounds(i * N + out1, 9ull * N)) A.fo[i * N + out1] = o.y;
            }
            if constexpr (THERMAL) {
                // g^eq = rho [(e P_x + S_x) P_y + P_x S_y], u_x = 0: S_x = (th^2/2, -th^2, th^2/2).
                const float e = 1.5f * RTw;
                const v2 th2 = th * th;
                const v2 Sx[3] = {V(0.5f) * th2, -th2, V(0.5f) * th2};
                const float S0 = 0.5f * U * U;
                const v2 S1 = V(U) * (th + V(S0)), S2 = fma2(th, th, V(U * U) * fma2(V(2.5f), th, V(S0)));
                const v2 Sy[3] = {V(0.5f) * (S2 - S1), V(S0) - S2, V(0.5f) * (S2 + S1)};
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int ix = i % 3, iy = i / 3;
                    const v2 o = fma2(fma2(V(e), ex[ix], rho * Sx[ix]), ey[iy], ex[ix] * Sy[iy]);
                    if (in_bounds(i * N + out0, 9ull * N)) A.go[i * N + out0] = o.x;
                    if (second && in_bounds(i * N + out1, 9ull * N)) A.go[i * N + out1] = o.y;
                }
            }
            rD = next_row(next_row(rD, ny), ny);
        } else if (inD && q - 3 >= q0) {
            const int p = q - 3;                   // its stage C ran at iteration q-1
            const v2 rho = cprev[0], Fx = cprev[1], Fy = cprev[2], RT = cprev[3], th = cprev[4], g0 = cprev[5];
            const int sw = slot - 1, se = slot + 1;
            // fields of pairs p-1 (slot sm1), p (s0), p+1 (sm2)
            const v2 *uxp = fld(UX, s0), *qxp = fld(QX, s0);
            const v2 *uy4 = fld(UY, sm1), *uy3 = fld(UY, s0), *uy2 = fld(UY, sm2);
            const v2 *qy4 = fld(QY, sm1), *qy3 = fld(QY, s0), *qy2 = fld(QY, sm2);
            const v2 *w4 = fld(WQ, sm1), *w3 = fld(WQ, s0), *w2 = fld(WQ, sm2);
            const v2 ux = uxp[slot], uy = uy3[slot];
            const v2 qyc = qy3[slot], wqc = w3[slot];
            const v2 uyN = shift_up(uy, uy2[slot]), uyS = shift_up(uy4[slot], uy);
            const v2 qyN = shift_up(qyc, qy2[slot]), qyS = shift_up(qy4[slot], qyc);
            const v2 wqN = shift_up(wqc, w2[slot]), wqS = shift_up(w4[slot], wqc);
            const v2 P0 = rho * th;
            const v2 divu = V(0.5f) * ((uxp[se] - uxp[sw]) + (uyN - uyS));
            const v2 Phi1 = P0 * (V(5.f / 3.f) - g0) * divu;
            // Phi_aa = Phi' - d_a[rho u_a (u_a^2 + 3 theta0 - 1)] (sign cancelling the c^3 = c bias).
            const v2 Phx = fma2(V(-0.5f), qxp[se] - qxp[sw], Phi1);
            const v2 Phy = fma2(V(-0.5f), qyN - qyS, Phi1);
            const v2 lP0h = V(0.5f * lambda) * P0, lPhi = V(lambda) * Phi1;
            const v2 qx = fma2(lP0h, w3[se] - w3[sw], ux * lPhi);
            const v2 qy = fma2(lP0h, wqN - wqS, uy * lPhi);

            const v2 lir = V(lambda) * rcp2(rho);
            const v2 usx = fma2(Fx, lir, ux), usy = fma2(Fy, lir, uy);
            const v2 zex = fma2(ux, ux, th), zey = fma2(uy, uy, th);
            const v2 zpx = fma2(usx, usx, th), zpy = fma2(usy, usy, th);
            const v2 zsx = fma2(Phx, lir, zpx), zsy = fma2(Phy, lir, zpy);
            // Psi factors (index 0, 1, 2 <-> c = -1, 0, +1), rho folded into the x factors.
            const v2 hr = V(0.5f) * rho;
            const v2 ex[3] = {hr * (zex - ux), rho - rho * zex, hr * (zex + ux)};
            const v2 ey[3] = {V(0.5f) * (zey - uy), V(1.f) - zey, V(0.5f) * (zey + uy)};
            const v2 sx[3] = {hr * (zsx - usx), rho - rho * zsx, hr * (zsx + usx)};
            const v2 sy[3] = {V(0.5f) * (zsy - usy), V(1.f) - zsy, V(0.5f) * (zsy + usy)};

            // Collision f' = kh f + keq f^eq + kst f*: the weights are folded into the x factors.
            const v2 kh = V(1.f - A.c_eq), keq = V(A.c_eq - A.c_star), kst = V(A.c_star);
            v2 exk[3], sxk[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                exk[k] = keq * ex[k];
                sxk[k] = kst * sx[k];
            }
            const unsigned out0 = layer + (unsigned)rD * nx + cols[1];
            const unsigned out1 = layer + (unsigned)next_row(rD, ny) * nx + cols[1];
            const bool second = 2 * p + 1 < y0 + Heff;
            // 16-bit storage: the node's new reference records (rho, u, theta0, e) for both rows
            // and the equilibria the deviations are taken against (dev16.cuh).
            EncTab tab0, tab1;
            if constexpr (DEV) {
                const Ref16 r0 = make_rec(rho.x, ux.x, uy.x, 0.f, th.x, RT.x);
                const Ref16 r1 = make_rec(rho.y, ux.y, uy.y, 0.f, th.y, RT.y);
                enc_tab<9>(r0, THERMAL, tab0);
                enc_tab<9>(r1, THERMAL, tab1);
                if (in_bounds(out0, N)) store_rec(A.Rout, N, out0, r0);
                if (second && in_bounds(out1, N)) store_rec(A.Rout, N, out1, r1);
            }
            const v2 *fr = f9 + (p & 3) * 9 * kW + t;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int ix = i % 3, iy = i / 3;
                const v2 o = fma2(kh, fr[i * kW], fma2(exk[ix], ey[iy], sxk[ix] * sy[iy]));
                if constexpr (DEV) {
                    if (in_bounds(i * N + out0, 9ull * N)) st16<ST>(A.fo, i * N + out0, encode_f<9>(ix - 1, iy - 1, 0, tab0, o.x));
                    if (second && in_bounds(i * N + out1, 9ull * N))
                        st16<ST>(A.fo, i * N + out1, encode_f<9>(ix - 1, iy - 1, 0, tab1, o.y));
                } else {
                    if (in_bounds(i * N + out0, 9ull * N)) A.fo[i * N + out0] = o.x;
                    if (second && in_bounds(i * N + out1, 9ull * N)) A.fo[i * N + out1] = o.y;
                }
            }
            if constexpr (THERMAL) {
                // g^eq_i = rho [e PsiP_x PsiP_y + PsiS_x PsiP_y + PsiP_x PsiS_y], e = 3/2 RT,
                // PsiP = Psi(u, theta0 + u^2), PsiS = Psi applied to (u^2/2, theta0 u + u^3/2,
                // theta0^2 + 5/2 theta0 u^2 + u^4/2); g* at (u*, RT* = RT - lambda^2 |F|^2/(3 rho^2)).
                const v2 e = V(1.5f) * RT;
                const v2 es = fma2(V(-0.5f), fma2(Fx, Fx, Fy * Fy) * (lir * lir), e);
                auto psiS = [&](v2 v, v2 o3[3]) {
                    const v2 vv = v * v;
                    const v2 S0 = V(0.5f) * vv;
                    const v2 S1 = v * fma2(V(0.5f), vv, th);
                    const v2 S2 = fma2(th, th, vv * fma2(V(2.5f), th, S0));
                    o3[0] = V(0.5f) * (S2 - S1);
                    o3[1] = S0 - S2;
                    o3[2] = V(0.5f) * (S2 + S1);
                };
                v2 Sx[3], Sy[3], SSx[3], SSy[3];
                psiS(ux, Sx); psiS(uy, Sy); psiS(usx, SSx); psiS(usy, SSy);
                // PsiP at the shifted velocity (no Phi: that correction belongs to f* only).
                const v2 px[3] = {hr * (zpx - usx), rho - rho * zpx, hr * (zpx + usx)};
                const v2 py[3] = {V(0.5f) * (zpy - usy), V(1.f) - zpy, V(0.5f) * (zpy + usy)};
                // x factors pre-multiplied by the collision weights keq (g^eq) and kst (g*).
                v2 Ax[3], As[3], pxk[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Ax[k] = keq * fma2(e, ex[k], rho * Sx[k]);      // keq rho (e PsiP_x + PsiS_x)
                    As[k] = kst * fma2(es, px[k], rho * SSx[k]);
                    pxk[k] = kst * px[k];
                }
                const v2 hqx = V(0.5f * A.c_star) * qx, hqy = V(0.5f * A.c_star) * qy;
                const v2 *gr = g9 + (p & 1) * 9 * kW + t;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int ix = i % 3, iy = i / 3;
                    v2 c = fma2(As[ix], py[iy], pxk[ix] * SSy[iy]);          // kst g*
                    if (i == 1) c = c - hqy;   // c = (0,-1)
                    if (i == 3) c = c - hqx;   // c = (-1,0)
                    if (i == 5) c = c + hqx;   // c = (1,0)
                    if (i == 7) c = c + hqy;   // c = (0,1)
                    c = fma2(exk[ix], Sy[iy], fma2(Ax[ix], ey[iy], c));      // + keq g^eq
                    const v2 o = fma2(kh, gr[i * kW], c);
                    if constexpr (DEV) {
                        if (in_bounds(i * N + out0, 9ull * N))
                            st16<ST>(A.go, i * N + out0, encode_g<9>(ix - 1, iy - 1, 0, tab0, o.x));
                        if (second && in_bounds(i * N + out1, 9ull * N))
                            st16<ST>(A.go, i * N + out1, encode_g<9>(ix - 1, iy - 1, 0, tab1, o.y));
                    } else {
                        if (in_bounds(i * N + out0, 9ull * N)) A.go[i * N + out0] = o.x;
                        if (second && in_bounds(i * N + out1, 9ull * N)) A.go[i * N + out1] = o.y;
                    }
                }
            }
            rD = next_row(next_row(rD, ny), ny);
        }
        s0 = sm2;                                          // slot of pair q+1
    }
}

}  // namespace fused
}  // namespace evlbm

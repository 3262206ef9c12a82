// Fused single-pass D2Q9 step of the Enskog-Vlasov lattice Boltzmann model
// (Karlin & Hosseini, arXiv 2508.00577), FP32 arithmetic and storage.
//
// One kernel does the whole step of Eq. (pre_LBM): pull streaming, raw moments,
// the Enskog-gauge force F = grad(a rho^2) + kappa rho grad(lap rho) in
// divergence (Korteweg-stress) form, the shifted velocity and energy
// (Eqs. u_shift, T_shift), the EOS and gamma0 (Eq. gamma), the gradient
// corrections Phi, Phi', q' (Eqs. correction_u/gamma/q), the equilibria
// (Eqs. feq, f_star, geq, gstar, g_corr) and the collision.
//
// Work decomposition.  A CTA owns a strip of W output columns of one 2-D layer
// and marches down a chunk of H rows.  The force needs rho within radius 2 of
// every node whose velocity is needed, and the corrections need u, T within
// radius 1 of the collided node, so the pipeline runs four row stages that lag
// each other by one row.  For the leading row L:
//   A: rho(L), j(L)          pulled populations of row L        (W + 6 columns)
//   B: Pi(L-1)               Korteweg stress from rho(L-2..L)   (W + 4 columns)
//   C: F, u, T, EOS (L-2)    div Pi(L-3..L-1), Gamma(L-2)       (W + 2 columns)
//   D: collide (L-3)         Phi, q' from fields(L-4..L-2)      (W columns)
// Rows of each stage live in 4-deep ring buffers in shared memory; a thread owns
// one column through all stages and keeps that column's centre values of the
// next collision row in registers.  The 6 halo columns of a strip are owned by
// an extra warp that takes part in stages A-C only.  Every population is read
// from HBM once per step; the re-reads of halo columns and of the collided row
// are served by L1/L2.
#include "dispatch.h"

namespace evlbm {

namespace {

constexpr int kW = 256;              // output columns per strip
constexpr int kThreads = kW + 32;    // + one halo warp
constexpr int kSlots = kW + 6;       // columns held per ring row
constexpr int kRing = 4;
constexpr int kFields = 11;          // rho, jx, jy, Pxx, Pxy, Pyy, ux, uy, flux_x, flux_y, wq

struct FusedArgs {
    const float *f, *g;
    float *fo, *go;
    const float *RT_iso;
    int nx, ny, nz, H;
    unsigned N;                      // nodes of the lattice (Q*N < 2^31)
    int eos;
    float a, b, kappa, lambda, c_eq, c_star;
};

__device__ __forceinline__ int wrap_any(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ int prev_row(int r, int ny) { return r == 0 ? ny - 1 : r - 1; }
__device__ __forceinline__ int next_row(int r, int ny) { return r == ny - 1 ? 0 : r + 1; }

// Loads the nine pulled populations of node (col, row): h_i = h~_i(x - c_i).
// rows[k] = wrapped row y + (k - 1), cols[k] = wrapped column x + (k - 1).
__device__ __forceinline__ void pull9(const float *__restrict__ base, unsigned N, const unsigned rowoff[3],
                                      const int cols[3], float h[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = i % 3 - 1, cy = i / 3 - 1;
        h[i] = __ldg(base + i * N + rowoff[1 - cy] + cols[1 - cx]);
    }
}

template <bool THERMAL>
__global__ void __launch_bounds__(kThreads, 2) k_fused2d(FusedArgs A)
{
    extern __shared__ float smem[];
    auto ring = [&](int field, int row) -> float * { return smem + (field * kRing + (row & 3)) * kSlots; };
    enum { RHO, JX, JY, PXX, PXY, PYY, UX, UY, QX, QY, WQ };

    const int nx = A.nx, ny = A.ny;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * kW;
    const int Weff = min(kW, nx - x0);
    const int y0 = blockIdx.y * A.H;
    const int Heff = min(A.H, ny - y0);
    const unsigned layer = (unsigned)blockIdx.z * (unsigned)nx * (unsigned)ny;

    // Column role of this thread.
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

    const float *fl = A.f + layer, *gl = A.g + layer;
    float *fol = A.fo + layer, *gol = A.go + layer;
    const unsigned N = A.N;
    const float a = A.a, b = A.b, kappa = A.kappa, lambda = A.lambda;
    const float c_eq = A.c_eq, c_star = A.c_star;

    // Wrapped centre rows of the stages, advanced by one each iteration.
    const int Lbeg = y0 - 3, Lend = y0 + Heff + 2;
    int rA = wrap_any(Lbeg, ny);
    int rC = wrap_any(Lbeg - 2, ny);
    int rD = wrap_any(Lbeg - 3, ny);

    // Centre values of the row to be collided next (computed in stage C one
    // iteration earlier), and its energy populations.
    float cRho = 1.f, cFx = 0.f, cFy = 0.f, cUx = 0.f, cUy = 0.f, cRT = 0.f, cTh = 0.f, cP0 = 0.f, cG0 = 0.f;
    float pRho = 1.f, pFx = 0.f, pFy = 0.f, pUx = 0.f, pUy = 0.f, pRT = 0.f, pTh = 0.f, pP0 = 0.f, pG0 = 0.f;
    float gC[9], gN[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) gC[i] = gN[i] = 0.f;

    for (int L = Lbeg; L <= Lend; ++L) {
        // ---------------- A: rho, j of row L ----------------
        if (inA) {
            const unsigned ro[3] = {(unsigned)prev_row(rA, ny) * nx, (unsigned)rA * nx, (unsigned)next_row(rA, ny) * nx};
            float h[9];
            pull9(fl, N, ro, cols, h);
            const float rho = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
            ring(RHO, L)[slot] = rho;
            ring(JX, L)[slot] = ((h[2] + h[5]) + h[8]) - ((h[0] + h[3]) + h[6]);
            ring(JY, L)[slot] = ((h[6] + h[7]) + h[8]) - ((h[0] + h[1]) + h[2]);
        }
        rA = next_row(rA, ny);
        __syncthreads();

        // ---------------- B: Korteweg stress of row L-1 ----------------
        if (inB && L - 1 >= y0 - 2) {
            const float *rs = ring(RHO, L - 2), *rc = ring(RHO, L - 1), *rn = ring(RHO, L);
            const float SW = rs[slot - 1], S = rs[slot], SE = rs[slot + 1];
            const float W_ = rc[slot - 1], C = rc[slot], E_ = rc[slot + 1];
            const float NW = rn[slot - 1], Nn = rn[slot], NE = rn[slot + 1];
            // Isotropic D2Q9 stencils: grad = 3 sum w c phi, lap = 6 sum w (phi - phi_0).
            const float dx = (1.f / 3.f) * (E_ - W_) + (1.f / 12.f) * ((NE - NW) + (SE - SW));
            const float dy = (1.f / 3.f) * (Nn - S) + (1.f / 12.f) * ((NE + NW) - (SE + SW));
            const float lap = (2.f / 3.f) * ((E_ + W_) + (Nn + S)) + (1.f / 6.f) * ((NE + NW) + (SE + SW)) -
                              (10.f / 3.f) * C;
            const float s = -a * C * C - kappa * C * lap - 0.5f * kappa * (dx * dx + dy * dy);
            ring(PXX, L - 1)[slot] = s + kappa * dx * dx;
            ring(PXY, L - 1)[slot] = kappa * dx * dy;
            ring(PYY, L - 1)[slot] = s + kappa * dy * dy;
        }
        __syncthreads();

        // ---------------- C: force, velocity, temperature, EOS of row L-2 ----------------
        if (inC && L - 2 >= y0 - 1) {
            const float *xs = ring(PXX, L - 3), *xc = ring(PXX, L - 2), *xn = ring(PXX, L - 1);
            const float *ys = ring(PXY, L - 3), *yc = ring(PXY, L - 2), *yn = ring(PXY, L - 1);
            const float *zs = ring(PYY, L - 3), *zn = ring(PYY, L - 1);
            const int sm = slot - 1, sp = slot + 1;
            const float dxPxx = (1.f / 3.f) * (xc[sp] - xc[sm]) + (1.f / 12.f) * ((xn[sp] - xn[sm]) + (xs[sp] - xs[sm]));
            const float dyPxy = (1.f / 3.f) * (yn[slot] - ys[slot]) + (1.f / 12.f) * ((yn[sp] + yn[sm]) - (ys[sp] + ys[sm]));
            const float dxPxy = (1.f / 3.f) * (yc[sp] - yc[sm]) + (1.f / 12.f) * ((yn[sp] - yn[sm]) + (ys[sp] - ys[sm]));
            const float dyPyy = (1.f / 3.f) * (zn[slot] - zs[slot]) + (1.f / 12.f) * ((zn[sp] + zn[sm]) - (zs[sp] + zs[sm]));
            const float Fx = -(dxPxx + dyPxy), Fy = -(dxPxy + dyPyy);
            const float rho = ring(RHO, L - 2)[slot];
            const float ir = 1.f / rho;
            const float ux = (ring(JX, L - 2)[slot] + 0.5f * Fx) * ir;
            const float uy = (ring(JY, L - 2)[slot] + 0.5f * Fy) * ir;
            float RT;
            if constexpr (THERMAL) {
                const unsigned ro[3] = {(unsigned)prev_row(rC, ny) * nx, (unsigned)rC * nx,
                                        (unsigned)next_row(rC, ny) * nx};
                pull9(gl, N, ro, cols, gN);
                const float Gam = ((gN[0] + gN[1]) + (gN[2] + gN[3])) + ((gN[4] + gN[5]) + (gN[6] + gN[7])) + gN[8];
                const float E = (Gam + 0.5f * (ux * Fx + uy * Fy)) * ir;
                RT = (2.f / 3.f) * (E - 0.5f * (ux * ux + uy * uy));
            } else {
                RT = __ldg(A.RT_iso + layer + (unsigned)rC * nx + cols[1]);
            }
            // EOS in the Enskog gauge: P0 = P_E = rho RT Z, gamma0 = 1 + rho Z'/Z [+ 2/3 Z].
            float Z, dlnZ;
            if (A.eos == 0) {
                Z = 1.f / (1.f - b * rho);
                dlnZ = b * rho * Z;
            } else {
                const float eta = 0.25f * b * rho;
                const float num = 1.f + eta * (1.f + eta * (1.f - eta));
                const float iom = 1.f / (1.f - eta);
                Z = num * iom * iom * iom;
                dlnZ = eta * (4.f + eta * (4.f - 2.f * eta)) * iom / num;
            }
            const float g0 = THERMAL ? 1.f + dlnZ + (2.f / 3.f) * Z : 1.f + dlnZ;
            const float th = RT * Z;
            ring(UX, L - 2)[slot] = ux;
            ring(UY, L - 2)[slot] = uy;
            ring(QX, L - 2)[slot] = rho * ux * (ux * ux + 3.f * th - 1.f);
            ring(QY, L - 2)[slot] = rho * uy * (uy * uy + 3.f * th - 1.f);
            ring(WQ, L - 2)[slot] = th - RT;
            // Centre values for the collision of this row at the next iteration.
            cRho = rho; cFx = Fx; cFy = Fy; cUx = ux; cUy = uy; cRT = RT; cTh = th; cP0 = rho * th; cG0 = g0;
        }
        rC = next_row(rC, ny);
        __syncthreads();

        // ---------------- D: collide row L-3 ----------------
        if (inD && L - 3 >= y0) {
            // Values of row L-3 computed in stage C of the previous iteration.
            const float rho = pRho, Fx = pFx, Fy = pFy, ux = pUx, uy = pUy, RT = pRT, th = pTh, P0 = pP0, g0 = pG0;
            const int sm = slot - 1, sp = slot + 1;
            const float *uxc = ring(UX, L - 3), *qxc = ring(QX, L - 3), *wqc = ring(WQ, L - 3);
            const float *uys = ring(UY, L - 4), *uyn = ring(UY, L - 2);
            const float *qys = ring(QY, L - 4), *qyn = ring(QY, L - 2);
            const float *wqs = ring(WQ, L - 4), *wqn = ring(WQ, L - 2);
            const float divu = 0.5f * (uxc[sp] - uxc[sm]) + 0.5f * (uyn[slot] - uys[slot]);
            const float Phi1 = P0 * (5.f / 3.f - g0) * divu;
            // Phi_aa = Phi' - d_a[rho u_a (u_a^2 + 3 theta0 - 1)] (sign cancelling the c^3 = c bias).
            const float Phx = Phi1 - 0.5f * (qxc[sp] - qxc[sm]);
            const float Phy = Phi1 - 0.5f * (qyn[slot] - qys[slot]);
            const float lP0 = lambda * P0;
            const float qx = lP0 * 0.5f * (wqc[sp] - wqc[sm]) + lambda * ux * Phi1;
            const float qy = lP0 * 0.5f * (wqn[slot] - wqs[slot]) + lambda * uy * Phi1;

            const float ir = 1.f / rho;
            const float usx = ux + lambda * Fx * ir, usy = uy + lambda * Fy * ir;
            const float zex = th + ux * ux, zey = th + uy * uy;
            const float zsx = th + usx * usx + lambda * Phx * ir, zsy = th + usy * usy + lambda * Phy * ir;
            // Psi factors (index 0, 1, 2 <-> c = -1, 0, +1), rho folded into the x factors.
            const float ex[3] = {rho * 0.5f * (zex - ux), rho * (1.f - zex), rho * 0.5f * (zex + ux)};
            const float ey[3] = {0.5f * (zey - uy), 1.f - zey, 0.5f * (zey + uy)};
            const float sx[3] = {rho * 0.5f * (zsx - usx), rho * (1.f - zsx), rho * 0.5f * (zsx + usx)};
            const float sy[3] = {0.5f * (zsy - usy), 1.f - zsy, 0.5f * (zsy + usy)};

            const unsigned ro[3] = {(unsigned)prev_row(rD, ny) * nx, (unsigned)rD * nx, (unsigned)next_row(rD, ny) * nx};
            float h[9];
            pull9(fl, N, ro, cols, h);
            const float k_h = 1.f - c_eq, k_eq = c_eq - c_star;
            const unsigned out = (unsigned)rD * nx + cols[1];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int ix = i % 3, iy = i / 3;
                const float feq = ex[ix] * ey[iy];
                const float fst = sx[ix] * sy[iy];
                fol[i * N + out] = k_h * h[i] + k_eq * feq + c_star * fst;
            }
            if constexpr (THERMAL) {
                // g^eq_i = rho [e PsiP_x PsiP_y + PsiS_x PsiP_y + PsiP_x PsiS_y], e = 3/2 RT,
                // PsiP = Psi(u, theta0 + u^2), PsiS = Psi applied to (u^2/2, theta0 u + u^3/2,
                // theta0^2 + 5/2 theta0 u^2 + u^4/2).
                const float e = 1.5f * RT;
                const float RTs = RT - (lambda * lambda / 3.f) * (Fx * Fx + Fy * Fy) * ir * ir;
                const float es = 1.5f * RTs;
                auto psiS = [&](float v, float out3[3]) {
                    const float v2 = v * v;
                    const float S0 = 0.5f * v2, S1 = v * (th + 0.5f * v2), S2 = th * th + v2 * (2.5f * th + 0.5f * v2);
                    out3[0] = 0.5f * (S2 - S1);
                    out3[1] = S0 - S2;
                    out3[2] = 0.5f * (S2 + S1);
                };
                float Sx[3], Sy[3], SSx[3], SSy[3];
                psiS(ux, Sx); psiS(uy, Sy); psiS(usx, SSx); psiS(usy, SSy);
                // PsiP at the shifted velocity (no Phi: that correction belongs to f* only).
                const float zpx = th + usx * usx, zpy = th + usy * usy;
                const float px[3] = {rho * 0.5f * (zpx - usx), rho * (1.f - zpx), rho * 0.5f * (zpx + usx)};
                const float py[3] = {0.5f * (zpy - usy), 1.f - zpy, 0.5f * (zpy + usy)};
                float Ax[3], As[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Ax[k] = e * ex[k] + rho * Sx[k];      // rho (e PsiP_x + PsiS_x)
                    As[k] = es * px[k] + rho * SSx[k];
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int ix = i % 3, iy = i / 3;
                    const float geq = Ax[ix] * ey[iy] + ex[ix] * Sy[iy];
                    float gst = As[ix] * py[iy] + px[ix] * SSy[iy];
                    if (i == 1) gst -= 0.5f * qy;     // c = (0,-1)
                    if (i == 3) gst -= 0.5f * qx;     // c = (-1,0)
                    if (i == 5) gst += 0.5f * qx;     // c = (1,0)
                    if (i == 7) gst += 0.5f * qy;     // c = (0,1)
                    gol[i * N + out] = k_h * gC[i] + k_eq * geq + c_star * gst;
                }
            }
        }
        rD = next_row(rD, ny);
        // The collision row of the next iteration is the one stage C just produced.
        pRho = cRho; pFx = cFx; pFy = cFy; pUx = cUx; pUy = cUy; pRT = cRT; pTh = cTh; pP0 = cP0; pG0 = cG0;
        if constexpr (THERMAL) {
#pragma unroll
            for (int i = 0; i < 9; ++i) gC[i] = gN[i];
        }
    }
}

}  // namespace

bool fused2d_supported(int prec, int Q, const KParams &p)
{
    return prec == 1 && Q == 9 && p.force_form == 0 && (long long)9 * p.N < (1LL << 31);
}

cudaError_t fused2d_step(int prec, const KParams &p, const void *f, const void *g, void *fo, void *go,
                         const void *RT_iso, cudaStream_t st)
{
    if (!fused2d_supported(prec, 9, p)) return cudaErrorNotSupported;
    FusedArgs A;
    A.f = static_cast<const float *>(f);
    A.g = static_cast<const float *>(g);
    A.fo = static_cast<float *>(fo);
    A.go = static_cast<float *>(go);
    A.RT_iso = static_cast<const float *>(RT_iso);
    A.nx = p.nx;
    A.ny = p.ny;
    A.nz = p.nz;
    A.N = (unsigned)p.N;
    A.eos = p.eos;
    A.a = float(p.a);
    A.b = float(p.b);
    A.kappa = float(p.kappa);
    A.lambda = float(p.lambda);
    A.c_eq = float(p.c_eq);
    A.c_star = float(p.c_star);
    A.H = p.ny <= 128 ? p.ny : 128;
    const size_t smem = sizeof(float) * kFields * kRing * kSlots;
    const dim3 grid((p.nx + kW - 1) / kW, (p.ny + A.H - 1) / A.H, p.nz);
    if (p.thermal) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_fused2d<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_fused2d<true><<<grid, kThreads, smem, st>>>(A);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_fused2d<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr = true;
        }
        k_fused2d<false><<<grid, kThreads, smem, st>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace evlbm

// Fused single-pass D3Q27 step of the Enskog-Vlasov lattice Boltzmann model
// (Karlin & Hosseini, arXiv 2508.00577), FP32 arithmetic with FP32 or 16-bit
// (FP16 / BF16 deviation, dev16.cuh) population storage: one launch per time
// step does pull streaming, raw moments, the Enskog-gauge force
// in divergence (Korteweg-stress) form, the shifted velocity and energy
// (Eqs. u_shift, T_shift), the EOS and gamma0 (Eq. gamma), the corrections
// Phi, Phi', q' (Eqs. correction_u/gamma/q), the equilibria (Eqs. feq, f_star,
// geq, gstar, g_corr) and the collision of Eq. (pre_LBM).
//
// Work decomposition (2.5-D z-marching).  A CTA owns a tile of (x, y) output columns
// (32 x 8 with FP32 storage, 32 x 16 with 16-bit storage, see TileOf) of one z-chunk (the
// last chunks shorter, so that the grid's last wave is short: step_t) and walks its
// planes one per iteration; four stages lag by one plane because the
// collision needs u and T within radius 1,
// hence F within radius 1, hence the Korteweg stress within radius 2, hence rho
// within radius 3:
//   A: rho, j (plane q)            pulled f           on the tile + 3 halo columns
//   B: Korteweg stress (q-1)       rho of q-2..q      on the tile + 2
//   C: F, u, T, EOS (q-2)          stress of q-3..q-1, pulled g   on the tile + 1
//   D: collide (q-3)               u, T fields of q-4..q-2, the tile's pulled f from
//                                  the TMEM stash stage A wrote 3 planes ago, pulled g
//                                  again (L2 hits: stage C read them 1 plane ago; FP32
//                                  loads them at the start of stage C; 16-bit storage
//                                  takes stage C's decoded g from a TMEM stash)
// Shared fields live in 3-deep plane rings sized to the region that reads them;
// centre values pass from C to D through a one-plane per-thread slot (stage C takes
// the tile column a thread collides in D first, and reads the slot before rewriting
// it); at 77 KB per CTA (32 x 8 tiles) two CTAs leave the L1 ~85 KB for loads in flight.
//
// 16-bit storage: every pulled population is rebuilt from its source node's FP32
// reference record (a 16- and an 8-byte load, L1/L2 hits after the first) and the
// stored deviation; stage D writes the node's new record and the deviations of its
// populations from the equilibria it computed for the collision.
#include "bounds.cuh"
#include "dev16.cuh"
#include "dispatch.h"
#include "tmem.cuh"

namespace evlbm {

namespace {

// Geometry of a TX x TY tile, one thread per output column (NT = TX TY threads; 256 run
// two CTAs per SM, 512 one): region widths (x, the row stride) and sizes of the tile + 3 /
// + 2 / + 1 halo regions of stages A / B / C, and the shared-memory layout.
template <int TX_, int TY_> struct Geo {
    static constexpr int TX = TX_, TY = TY_, NT = TX * TY, MINB = 512 / NT;
    static_assert(NT == 256 || NT == 512, "256 or 512 threads per CTA");
    static constexpr int WA = TX + 6, WB = TX + 4, WC = TX + 2;
    static constexpr int SA = WA * (TY + 6), SB = WB * (TY + 4), SC = WC * (TY + 2);
    // Column passes of stages A and B (NT columns per pass); stage C's ring fits in one.
    static constexpr int PA = (SA + NT - 1) / NT, PB = (SB + NT - 1) / NT;
    static_assert(2 * WC + 2 * TY <= NT, "stage C's ring columns exceed one pass");
    // Shared-memory layout (floats).
    static constexpr int O_RHO = 0;               // [3][SA]
    static constexpr int O_J = O_RHO + 3 * SA;    // [3 planes][3 comps][SC]
    static constexpr int O_PI = O_J + 9 * SC;     // [6 comps][SB]  xx xy xz yy yz zz of the newest plane
    static constexpr int O_PF = O_PI + 6 * SB;    // [3 planes][3 comps][SC]  partial forces, per stage-C column
    static constexpr int O_CF = O_PF + 9 * SC;    // [3 planes][7][SC]  ux uy uz qx qy qz wq
    static constexpr int O_CEN = O_CF + 21 * SC;  // [7][NT]  rho Fx Fy Fz RT theta0 gamma0 (one plane)
    static constexpr int NR = 2 * WC + 2 * TY;    // stage C's ring columns (the tile + 1 outside the tile)
    static constexpr size_t SMEM_BYTES = sizeof(float) * (O_CEN + 7 * NT);
};
// Tile shape per storage type.  FP32: 32 x 8, so that a warp's load of one population is
// one row of 32 consecutive nodes (16 x 16 tiles load two half rows per warp; 32 x 8 ran
// 7 % faster despite 10 % more halo columns).  16-bit storage, bound by its decoding:
// 32 x 16 (512 threads, one CTA per SM), whose halo is the smallest (stage A decodes 1.63
// columns per tile column against 1.89 for 16 x 16 and 2.08 for 32 x 8; 16 x 16 ran 2.5 %
// slower, 32 x 8 6 %).
template <typename S> struct TileOf { using G = Geo<32, 16>; };
template <> struct TileOf<float> { using G = Geo<32, 8>; };

constexpr int kMaxTail = 8, kMinTail = 8;

template <typename S> struct Args {
    const S *f, *g;
    S *fo, *go;
    const float *Rin;                             // reference records read (16-bit storage)
    float *Rout;                                  // reference records written
    const float *RT_iso;
    int nx, ny, nz, HZ;
    // z-chunks: nfull chunks of HZ planes, then ntail shorter ones at offsets tail[] from
    // nfull * HZ (tail[ntail] = the planes left), so that the last CTAs to run are short.
    int nfull, ntail;
    int tail[kMaxTail + 1];
    unsigned N;
    int eos;
    float a, b, kappa, lambda, c_eq, c_star;
};

// Reciprocal with the hardware approximation (rcp.approx.ftz: at most 1 ulp); the
// operands (rho, 1 - b rho, EOS polynomials) are normal numbers.
__device__ __forceinline__ float rcpa(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// Tensor memory as a per-thread stash (no tensor-core work here).  Stage A pulls the 27 f
// of the thread's own tile column three planes before stage D collides that node; the
// values wait in TMEM instead of being pulled from L2/DRAM a second time.  4 plane slots
// of 32 columns per thread; the warps of a lane quarter (w, w + 4, ...) use consecutive
// 128-column blocks of the CTA's NT columns (256 threads: two CTAs per SM fill the 512;
// 512 threads: one).  In a slot,
// population i = 9 kz + j sits at column 8 kz + j for j < 8 and at 24 + kz for j = 8, so
// that every access starts at a multiple of its width.
constexpr int TM_WARP_COLS = 128, TM_SLOT = 32, TM_SLOTS = 4;
static_assert(TM_SLOTS * TM_SLOT <= TM_WARP_COLS, "stash slots exceed a warp's columns");

__device__ __forceinline__ uint32_t tm_addr(uint32_t base, int t)
{
    const int w = t >> 5;
    return tmem::lane_base(base, w) + (uint32_t)((w >> 2) * TM_WARP_COLS);
}
// Warp-collective (.sync.aligned): every thread of the warp executes these (they
// reconverge the warp first).
__device__ __forceinline__ void tm_st27(uint32_t ta, const float v[27])
{
    __syncwarp();
#define R_(k) "r"(__float_as_uint(v[k]))
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(ta), R_(0), R_(1), R_(2), R_(3), R_(4), R_(5), R_(6), R_(7), R_(9), R_(10), R_(11), R_(12),
                 R_(13), R_(14), R_(15), R_(16) : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(ta + 16), R_(18), R_(19), R_(20), R_(21), R_(22), R_(23), R_(24), R_(25) : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};"
                 ::"r"(ta + 24), R_(8), R_(17), R_(26), "r"(0u) : "memory");
#undef R_
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// The nine populations of layer kz, waited for before they are used.
__device__ __forceinline__ void tm_ld9(uint32_t ta, int kz, float v[9])
{
    __syncwarp();
    uint32_t r[9];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%9];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%8}, [%10];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8])
                 : "r"(ta + 8u * (uint32_t)kz), "r"(ta + 24u + (uint32_t)kz) : "memory");
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = __uint_as_float(r[k]);
}

// Thermal kernel with 16-bit storage: stage D would otherwise decode the tile's 27 g a
// second time (stage C decoded them one iteration earlier for the energy), and a g costs
// about three times an f to decode.  The thread's 128 columns then hold two plane slots of
// stage C's decoded g (plane mod 2, columns 32 s + [0, 27) in the layout above) and four
// plane slots of stage A's decoded f of the layers c_z = -1, 0 only (kz = 0, 1): population
// 9 kz + j at 64 + 16 s + 8 kz + j for j < 8 and at gs_f8(s) + kz for j = 8 (columns 28-31
// and 60-63, free in the g slots).  Stage D decodes the f of the third layer again.
constexpr uint32_t GS_F = 64;
__device__ __forceinline__ uint32_t gs_f8(int s) { return (uint32_t)((s < 2 ? 28 : 56) + 2 * s); }

// Layer kz of nine values into a slot of the 27-value layout (completed by tm_wait_st).
__device__ __forceinline__ void tm_st9(uint32_t ta, int kz, const float v[9])
{
    __syncwarp();
#define R_(k) "r"(__float_as_uint(v[k]))
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(ta + 8u * (uint32_t)kz), R_(0), R_(1), R_(2), R_(3), R_(4), R_(5), R_(6), R_(7) : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(ta + 24u + (uint32_t)kz), R_(8) : "memory");
#undef R_
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// The f of layers kz = 0, 1 of v[27] into f slot s.
__device__ __forceinline__ void tm_st18(uint32_t tb, int s, const float v[27])
{
    __syncwarp();
#define R_(k) "r"(__float_as_uint(v[k]))
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(tb + GS_F + 16u * (uint32_t)s), R_(0), R_(1), R_(2), R_(3), R_(4), R_(5), R_(6), R_(7), R_(9),
                 R_(10), R_(11), R_(12), R_(13), R_(14), R_(15), R_(16) : "memory");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(tb + gs_f8(s)), R_(8), R_(17) : "memory");
#undef R_
    tm_wait_st();
}
// Layer kz (0 or 1) of f slot s, waited for before it is used.
__device__ __forceinline__ void tm_ld9f(uint32_t tb, int s, int kz, float v[9])
{
    __syncwarp();
    uint32_t r[9];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%9];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%8}, [%10];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8])
                 : "r"(tb + GS_F + 16u * (uint32_t)s + 8u * (uint32_t)kz), "r"(tb + gs_f8(s) + (uint32_t)kz)
                 : "memory");
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = __uint_as_float(r[k]);
}

// Global loads and stores with the bounds check of checked builds (no-op otherwise).
// 16-bit storage loads and stores the raw deviation.
__device__ __forceinline__ float ldc(const float *base, unsigned off, unsigned long long n)
{
    return in_bounds(off, n) ? __ldg(base + off) : 0.f;
}
template <typename S>
__device__ __forceinline__ float ldc(const S *base, unsigned off, unsigned long long n)
{
    return in_bounds(off, n) ? Bits16<S>::to_f(__ldg(reinterpret_cast<const unsigned short *>(base) + off)) : 0.f;
}
__device__ __forceinline__ void stc(float *base, unsigned off, unsigned long long n, float v)
{
    if (in_bounds(off, n)) __stcs(base + off, v);
}
template <typename S>
__device__ __forceinline__ void stc(S *base, unsigned off, unsigned long long n, float v)
{
    if (in_bounds(off, n)) __stcs(reinterpret_cast<unsigned short *>(base) + off, Bits16<S>::from_f(v));
}
// Reference record of node n (16-bit storage).
__device__ __forceinline__ Ref16 ldrec(const float *R, unsigned n, unsigned long long N)
{
    if (!in_bounds(n, N)) return Ref16{1.f, {0.f, 0.f, 0.f}, 0.f, 0.f};
    return load_rec(R, (long long)N, n);
}
__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

constexpr __host__ __device__ int cxi(int i) { return i % 3 - 1; }
constexpr __host__ __device__ int cyi(int i) { return (i / 3) % 3 - 1; }
constexpr __host__ __device__ int czi(int i) { return i / 9 - 1; }
// 1-D weights 2/3 (c = 0), 1/6 (c = +-1); w_i is their product.
constexpr __host__ __device__ float w1(int c) { return c == 0 ? 2.f / 3.f : 1.f / 6.f; }
constexpr __host__ __device__ float wi(int i) { return w1(cxi(i)) * w1(cyi(i)) * w1(czi(i)); }

// Offsets of the 27 pulled populations of node (x, y, z): source x - c_i.
// xo[k] = wrapped x - 1 + k, yo[k] = (wrapped y - 1 + k) * nx, zo[k] = (wrapped z - 1 + k) * nx*ny.
struct Cell {
    unsigned xo[3], yo[3];
};

__device__ __forceinline__ Cell cell_of(int x, int y, int nx, int ny)
{
    Cell c;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c.xo[k] = (unsigned)wrapi(x - 1 + k, nx);
        c.yo[k] = (unsigned)wrapi(y - 1 + k, ny) * (unsigned)nx;
    }
    return c;
}

__device__ __forceinline__ void plane_offsets(int z, int nx, int ny, int nz, unsigned zo[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) zo[k] = (unsigned)wrapi(z - 1 + k, nz) * (unsigned)nx * (unsigned)ny;
}

// h_i = h~_i(x - c_i): index of the source of population i.
__device__ __forceinline__ unsigned src_of(int i, const Cell &c, const unsigned zo[3], unsigned N)
{
    return (unsigned)i * N + zo[1 - czi(i)] + c.yo[1 - cyi(i)] + c.xo[1 - cxi(i)];
}

// Psi(c; xi, zeta): 1 - zeta (c = 0), (zeta +- xi)/2 (c = +-1), Eq. (phi).
__device__ __forceinline__ void psi3(float xi, float zeta, float out[3])
{
    out[0] = 0.5f * (zeta - xi);
    out[1] = 1.f - zeta;
    out[2] = 0.5f * (zeta + xi);
}

// The same linear combination applied to (A0, A1, A2).
__device__ __forceinline__ void psi3_poly(float A0, float A1, float A2, float out[3])
{
    out[0] = 0.5f * (A2 - A1);
    out[1] = A0 - A2;
    out[2] = 0.5f * (A2 + A1);
}

// 16 warps per SM at 128 registers per thread: two CTAs of 256 threads (FP32) or one of
// 512 (16-bit storage).  The thermal kernel with 16-bit storage spills ~30 B per thread at
// that budget; 8 warps per SM with 245 registers and no spill was measured slower (2.11
// against 2.49 GLUPS at 256^3, an earlier form).
template <bool THERMAL, typename S>
__global__ void __launch_bounds__(TileOf<S>::G::NT, TileOf<S>::G::MINB) k_fused3d(const Args<S> A)
{
    constexpr bool DEV = Store<S>::dev;
    constexpr bool GST = DEV && THERMAL;                  // the g-stash layout of the TMEM columns
    using G = typename TileOf<S>::G;
    constexpr int TX = G::TX, TY = G::TY, NT = G::NT, WA = G::WA, WB = G::WB, WC = G::WC;
    constexpr uint32_t TM_COLS = NT;                      // 128 columns per warp of a lane quarter
    constexpr int SA = G::SA, SB = G::SB, SC = G::SC, PA = G::PA, PB = G::PB;
    extern __shared__ float sm[];
    const int t = threadIdx.x;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int ch = (int)blockIdx.z, zt = ch - A.nfull, zb = A.nfull * A.HZ;
    const int z0 = zt < 0 ? ch * A.HZ : zb + A.tail[zt];
    const int zend = zt < 0 ? z0 + A.HZ : zb + A.tail[zt + 1];
    const unsigned N = A.N;
    const float a = A.a, b = A.b, kappa = A.kappa, lambda = A.lambda;

    // Columns this thread handles in stages A, B, C (up to two each).
    // Stage A: first the thread's own tile column (whose pulled f it stashes for stage D),
    // then the halo columns, NT per further pass: three rows above and below the tile
    // (WA columns each), then three columns left and right of each tile row.
    auto colA = [&](int k, int &cx, int &cy) {
        if (k == 0) { cx = t % TX; cy = t / TX; return true; }
        const int r = t + (k - 1) * NT;
        if (r < 3 * WA) { cx = r % WA - 3; cy = r / WA - 3; }
        else if (r < 6 * WA) { cx = (r - 3 * WA) % WA - 3; cy = TY + (r - 3 * WA) / WA; }
        else { const int m = (r - 6 * WA) % 6; cy = (r - 6 * WA) / 6; cx = m < 3 ? m - 3 : TX + m - 3; }
        return r < SA - NT;
    };
    auto colB = [&](int k, int &cx, int &cy) { const int c = t + k * NT; cx = c % WB - 2; cy = c / WB - 2; return c < SB; };
    // Stage C: first the tile's own column of this thread (the one it collides in stage D,
    // so the centre values stay thread-private), then the NR ring columns on threads 0..NR-1.
    auto ringC = [&](int r, int &cx, int &cy) {
        if (r < WC) { cx = r - 1; cy = -1; }
        else if (r < 2 * WC) { cx = r - WC - 1; cy = TY; }
        else if (r < 2 * WC + TY) { cx = -1; cy = r - 2 * WC; }
        else { cx = TX; cy = r - 2 * WC - TY; }
    };
    auto colC = [&](int k, int &cx, int &cy) {
        if (k == 0) { cx = t % TX; cy = t / TX; return true; }
        ringC(t, cx, cy);
        return t < G::NR;
    };
    auto sa = [](int cx, int cy) { return (cy + 3) * WA + (cx + 3); };
    auto sb = [](int cx, int cy) { return (cy + 2) * WB + (cx + 2); };
    auto sc = [](int cx, int cy) { return (cy + 1) * WC + (cx + 1); };
    float *RHO = sm + G::O_RHO, *J = sm + G::O_J, *PI = sm + G::O_PI, *PF = sm + G::O_PF, *CF = sm + G::O_CF,
          *CEN = sm + G::O_CEN;

    const int dcx = t % TX, dcy = t / TX;                 // this thread's output column
    const bool inD = x0 + dcx < nx && y0 + dcy < ny;
    const Cell cD = cell_of(x0 + dcx, y0 + dcy, nx, ny);

    // TMEM stash of the tile's pulled f (allocated by warp 0, freed after the last plane).
    __shared__ uint32_t tm_base_sh;
    if (t < 32) tmem::alloc(&tm_base_sh, TM_COLS);
    tmem::fence_sync();
    const uint32_t tmt = tm_addr(tm_base_sh, t);

    const int qbeg = z0 - 3, qend = zend + 2;
    for (int q = qbeg; q <= qend; ++q) {
        const int s0 = ((q % 3) + 3) % 3;                 // ring slot of plane q (and of q-3)
        const int sm1 = s0 == 0 ? 2 : s0 - 1;             // plane q-1 (and q-4)
        const int sm2 = s0 == 2 ? 0 : s0 + 1;             // plane q-2
        // ---------------- A: rho, j of plane q ----------------
        if (q <= zend + 2) {
            unsigned zo[3];
            plane_offsets(q, nx, ny, nz, zo);
#pragma unroll 1
            for (int k = 0; k < PA; ++k) {
                int cx, cy;
                if (!colA(k, cx, cy)) continue;
                const Cell c = cell_of(x0 + cx, y0 + cy, nx, ny);
                float rho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
                float hv[27];
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    const unsigned si = src_of(i, c, zo, N);
                    float h = ldc(A.f, si, 27ull * N);
                    if constexpr (DEV) h = decode_f<27>(cxi(i), cyi(i), czi(i), ldrec(A.Rin, si - i * N, N), h);
                    hv[i] = h;
                    rho += h;
                    if (cxi(i) == 1) jx += h; else if (cxi(i) == -1) jx -= h;
                    if (cyi(i) == 1) jy += h; else if (cyi(i) == -1) jy -= h;
                    if (czi(i) == 1) jz += h; else if (czi(i) == -1) jz -= h;
                }
                if (k == 0) {                                 // all threads: slot of plane q
                    if constexpr (GST) tm_st18(tmt, (q + 4) & 3, hv);
                    else tm_st27(tmt + (uint32_t)(((q + 4) & 3) * TM_SLOT), hv);
                }
                if (in_bounds(sa(cx, cy), SA)) RHO[s0 * SA + sa(cx, cy)] = rho;
                if (cx >= -1 && cx <= TX && cy >= -1 && cy <= TY && in_bounds(sc(cx, cy), SC)) {
                    float *jr = J + s0 * 3 * SC + sc(cx, cy);
                    jr[0] = jx;
                    jr[SC] = jy;
                    jr[2 * SC] = jz;
                }
            }
        }
        __syncthreads();

        const bool haveP = q - 1 >= z0 - 2 && q - 1 <= zend + 1;   // stage B writes Pi(q-1)
        const bool runC = q - 2 >= z0 - 1 && q - 2 <= zend;        // stage C's plane is needed

        // ---------------- B: Korteweg stress of plane q-1 ----------------
        if (haveP) {
#pragma unroll
            for (int k = 0; k < PB; ++k) {
                int cx, cy;
                if (!colB(k, cx, cy)) continue;
                const float *r[3] = {RHO + sm2 * SA, RHO + sm1 * SA, RHO + s0 * SA};   // planes q-2, q-1, q
                const int c0 = sa(cx, cy);
                if (!(in_bounds(c0 - WA - 1, SA) && in_bounds(c0 + WA + 1, SA) && in_bounds(sb(cx, cy), SB))) continue;
                const float rc = r[1][c0];
                float gx = 0.f, gy = 0.f, gz = 0.f, lap = 0.f;
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    if (i == 13) continue;
                    const float v = r[1 + czi(i)][c0 + cyi(i) * WA + cxi(i)];
                    const float w = wi(i);
                    if (cxi(i)) gx += (cxi(i) * w) * v;
                    if (cyi(i)) gy += (cyi(i) * w) * v;
                    if (czi(i)) gz += (czi(i) * w) * v;
                    lap += w * (v - rc);
                }
                gx *= 3.f; gy *= 3.f; gz *= 3.f; lap *= 6.f;
                const float s = -a * rc * rc - kappa * rc * lap - 0.5f * kappa * (gx * gx + gy * gy + gz * gz);
                float *pr = PI + sb(cx, cy);
                pr[0] = s + kappa * gx * gx;
                pr[SB] = kappa * gx * gy;
                pr[2 * SB] = kappa * gx * gz;
                pr[3 * SB] = s + kappa * gy * gy;
                pr[4 * SB] = kappa * gy * gz;
                pr[5 * SB] = s + kappa * gz * gz;
            }
        }
        __syncthreads();

        // ---------------- C: F, u, T, EOS of plane q-2 ----------------
        // The force F_a = -d_b Pi_ab = -3 sum_i w_i c_ib Pi_ab(x + c_i) splits by plane: the
        // stress plane P adds w1(cz) (T_a + cz S_a) to the force of plane P - cz, with the
        // in-plane sums T_a = sum w1(cx) w1(cy) (cx Pi_ax + cy Pi_ay) and
        // S_a = sum w1(cx) w1(cy) Pi_az over the 3 x 3 neighbours (w_i = w1(cx) w1(cy) w1(cz),
        // w1(0) = 2/3, w1(+-1) = 1/6).  Each new stress plane (q-1, from stage B) is folded
        // into the partial forces of planes q (first term), q-1 and q-2 (complete), kept
        // per stage-C column (thread-private).
        float cprev[7];                                   // centre values of plane q-3 (stage D)
        // Software pipelining (FP32 thermal): stage D's pulled g (plane q-3) are loaded at the
        // start of stage C, so that their latency overlaps stage C and its barrier instead
        // of following it.  (Loading stage C's g before stage B the same way made the kernel
        // 11 % slower.)
        constexpr bool PRE = THERMAL && !DEV;
        float gD[27];
        if constexpr (PRE) {
            if (q - 3 >= z0 && q - 3 < zend) {
                unsigned zo[3];
                plane_offsets(q - 3, nx, ny, nz, zo);
#pragma unroll
                for (int i = 0; i < 27; ++i) gD[i] = ldc(A.g, src_of(i, cD, zo, N), 27ull * N);
            }
        }
        if (haveP) {
            unsigned zo[3];
            if (THERMAL) plane_offsets(q - 2, nx, ny, nz, zo);
            const int zc = wrapi(q - 2, nz);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                int cx, cy;
                if (!colC(k, cx, cy)) continue;
                float Gam = 0.f;                          // sum of the pulled g (thermal)
                if constexpr (GST) {
                    // The tile column's g of plane q-2, summed and stashed for stage D of the
                    // next iteration (warp-collective stores: before any per-thread branch).
                    if (k == 0 && runC) {
                        const Cell c = cell_of(x0 + cx, y0 + cy, nx, ny);
                        const uint32_t tg = tmt + (uint32_t)(((q + 2) & 1) * TM_SLOT);
#pragma unroll
                        for (int kz = 0; kz < 3; ++kz) {
                            float v9[9];
#pragma unroll
                            for (int j = 0; j < 9; ++j) {
                                const int i = 9 * kz + j;
                                const unsigned si = src_of(i, c, zo, N);
                                v9[j] = decode_g<27>(cxi(i), cyi(i), czi(i), ldrec(A.Rin, si - i * N, N),
                                                     ldc(A.g, si, 27ull * N));
                                Gam += v9[j];             // in index order, as the ring columns sum
                            }
                            tm_st9(tg, kz, v9);
                        }
                        tm_wait_st();
                    }
                }
                const int b0 = sb(cx, cy);
                const int pc = k == 0 ? t : NT + t;       // this column's partial-force slot
                if (!(in_bounds(b0 - WB - 1, SB) && in_bounds(b0 + WB + 1, SB) && in_bounds(sc(cx, cy), SC) &&
                      in_bounds(sa(cx, cy), SA) && in_bounds(pc, SC)))
                    continue;
                float T[3] = {0.f, 0.f, 0.f}, Sz[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
                    for (int ox = -1; ox <= 1; ++ox) {
                        const float w = (ox ? 1.f / 6.f : 2.f / 3.f) * (oy ? 1.f / 6.f : 2.f / 3.f);
                        const float *pp = PI + b0 + oy * WB + ox;
                        if (ox) {
                            const float cw = ox * w;
                            T[0] += cw * pp[0];
                            T[1] += cw * pp[SB];
                            T[2] += cw * pp[2 * SB];
                        }
                        if (oy) {
                            const float cw = oy * w;
                            T[0] += cw * pp[SB];
                            T[1] += cw * pp[3 * SB];
                            T[2] += cw * pp[4 * SB];
                        }
                        Sz[0] += w * pp[2 * SB];
                        Sz[1] += w * pp[4 * SB];
                        Sz[2] += w * pp[5 * SB];
                    }
                float *fq = PF + s0 * 3 * SC + pc, *fq1 = PF + sm1 * 3 * SC + pc, *fq2 = PF + sm2 * 3 * SC + pc;
                float F[3];
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    fq[m * SC] = (1.f / 6.f) * (T[m] - Sz[m]);           // plane q,   cz = -1 (first term)
                    fq1[m * SC] += (2.f / 3.f) * T[m];                  // plane q-1, cz = 0
                    F[m] = -3.f * (fq2[m * SC] + (1.f / 6.f) * (T[m] + Sz[m]));   // plane q-2, complete
                }
                if (!runC) continue;
                const float Fx = F[0], Fy = F[1], Fz = F[2];
                const float rho = RHO[sm2 * SA + sa(cx, cy)];
                const float *jr = J + sm2 * 3 * SC + sc(cx, cy);
                const float ir = rcpa(rho);
                const float ux = (jr[0] + 0.5f * Fx) * ir, uy = (jr[SC] + 0.5f * Fy) * ir, uz = (jr[2 * SC] + 0.5f * Fz) * ir;
                float RT;
                if (THERMAL) {
                    if (!(GST && k == 0)) {
                        const Cell c = cell_of(x0 + cx, y0 + cy, nx, ny);
#pragma unroll
                        for (int i = 0; i < 27; ++i) {
                            const unsigned si = src_of(i, c, zo, N);
                            float h = ldc(A.g, si, 27ull * N);
                            if constexpr (DEV) h = decode_g<27>(cxi(i), cyi(i), czi(i), ldrec(A.Rin, si - i * N, N), h);
                            Gam += h;
                        }
                    }
                    const float E = (Gam + 0.5f * (ux * Fx + uy * Fy + uz * Fz)) * ir;
                    RT = (2.f / 3.f) * (E - 0.5f * (ux * ux + uy * uy + uz * uz));
                } else {
                    const unsigned n = (unsigned)zc * (unsigned)nx * (unsigned)ny +
                                       (unsigned)wrapi(y0 + cy, ny) * (unsigned)nx + (unsigned)wrapi(x0 + cx, nx);
                    RT = ldc(A.RT_iso, n, N);
                }
                // EOS in the Enskog gauge: P0 = P_E = rho RT Z, gamma0 = 1 + rho Z'/Z [+ 2/3 Z].
                float Z, dlnZ;
                if (A.eos == 0) {
                    Z = rcpa(1.f - b * rho);
                    dlnZ = b * rho * Z;
                } else {
                    const float eta = 0.25f * b * rho;
                    const float num = 1.f + eta + eta * eta - eta * eta * eta;
                    const float iom = rcpa(1.f - eta);
                    Z = num * iom * iom * iom;
                    dlnZ = eta * (4.f + 4.f * eta - 2.f * eta * eta) * iom * rcpa(num);
                }
                const float g0 = THERMAL ? 1.f + dlnZ + (2.f / 3.f) * Z : 1.f + dlnZ;
                const float th = RT * Z;
                const float th3m1 = 3.f * th - 1.f;
                float *cf = CF + sm2 * 7 * SC + sc(cx, cy);
                cf[0] = ux;
                cf[SC] = uy;
                cf[2 * SC] = uz;
                cf[3 * SC] = rho * ux * (ux * ux + th3m1);
                cf[4 * SC] = rho * uy * (uy * uy + th3m1);
                cf[5 * SC] = rho * uz * (uz * uz + th3m1);
                cf[6 * SC] = th - RT;
                if (k == 0) {
                    // The slot still holds plane q-3, collided by this thread in stage D of
                    // this iteration: take it into registers before storing plane q-2.
                    float *ce = CEN + t;
#pragma unroll
                    for (int m = 0; m < 7; ++m) cprev[m] = ce[m * NT];
                    ce[0] = rho; ce[NT] = Fx; ce[2 * NT] = Fy; ce[3 * NT] = Fz;
                    ce[4 * NT] = RT; ce[5 * NT] = th; ce[6 * NT] = g0;
                }
            }
        }
        __syncthreads();

        // ---------------- D: collide plane q-3 ----------------
        const int p = q - 3;
        if (p >= z0 && p < zend) {
            // Every thread runs stage D (the TMEM loads are warp-collective); threads whose
            // column lies outside the lattice compute on wrapped values and store nothing.
            const bool act = inD && in_bounds(sc(dcx, dcy) - WC, SC) && in_bounds(sc(dcx, dcy) + WC, SC);
            const uint32_t tmp = tmt + (uint32_t)(((p + 4) & 3) * TM_SLOT);       // stash slot of plane p
            // Centre values of plane p (stage C ran at iteration q-1), read in stage C.
            const float rho = cprev[0], Fx = cprev[1], Fy = cprev[2], Fz = cprev[3];
            const float RT = cprev[4], th = cprev[5], g0 = cprev[6];
            // C fields of planes p-1 (slot sm1), p (s0), p+1 (sm2).
            const float *Fm = CF + sm1 * 7 * SC, *F0 = CF + s0 * 7 * SC, *Fp = CF + sm2 * 7 * SC;
            const int c0 = sc(dcx, dcy);
            const int xp = c0 + 1, xm = c0 - 1, yp = c0 + WC, ym = c0 - WC;
            const float ux = F0[c0], uy = F0[SC + c0], uz = F0[2 * SC + c0];
            const float P0 = rho * th;
            const float divu = 0.5f * ((F0[xp] - F0[xm]) + (F0[SC + yp] - F0[SC + ym]) + (Fp[2 * SC + c0] - Fm[2 * SC + c0]));
            const float Phi1 = P0 * (5.f / 3.f - g0) * divu;
            // Phi_aa = Phi' - d_a[rho u_a (u_a^2 + 3 theta0 - 1)] (sign cancelling the c^3 = c bias).
            const float Phx = Phi1 - 0.5f * (F0[3 * SC + xp] - F0[3 * SC + xm]);
            const float Phy = Phi1 - 0.5f * (F0[4 * SC + yp] - F0[4 * SC + ym]);
            const float Phz = Phi1 - 0.5f * (Fp[5 * SC + c0] - Fm[5 * SC + c0]);
            const float lP0h = 0.5f * lambda * P0, lPhi = lambda * Phi1;
            const float qx = lP0h * (F0[6 * SC + xp] - F0[6 * SC + xm]) + ux * lPhi;
            const float qy = lP0h * (F0[6 * SC + yp] - F0[6 * SC + ym]) + uy * lPhi;
            const float qz = lP0h * (Fp[6 * SC + c0] - Fm[6 * SC + c0]) + uz * lPhi;

            const float lir = lambda * rcpa(rho);
            const float usx = ux + Fx * lir, usy = uy + Fy * lir, usz = uz + Fz * lir;
            // Separable equilibria: h_i = X[c_ix] * YZ[c_iy][c_iz] (+ X'[c_ix] * YZ'[..]),
            // the per-axis Psi factors combined once per node (Eqs. feq, f_star, geq, gstar).
            // f^eq and g^eq are evaluated with the rounding-exact functions of the 16-bit
            // storage references (dev16.cuh): there they are the references themselves.
            float ex[3], ey[3], ez[3], sx[3], sy[3], sz[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ex[k] = refP(k - 1, ux, th);
                ey[k] = refP(k - 1, uy, th);
                ez[k] = refP(k - 1, uz, th);
            }
            psi3(usx, th + usx * usx + Phx * lir, sx);
            psi3(usy, th + usy * usy + Phy * lir, sy);
            psi3(usz, th + usz * usz + Phz * lir, sz);
            float rex[3], rsx[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                rex[k] = __fmul_rn(rho, ex[k]);
                rsx[k] = rho * sx[k];
            }

            unsigned zo[3];
            plane_offsets(p, nx, ny, nz, zo);
            const unsigned out = (unsigned)wrapi(p, nz) * (unsigned)nx * (unsigned)ny +
                                 (unsigned)(y0 + dcy) * (unsigned)nx + (unsigned)(x0 + dcx);
            const float kh = 1.f - A.c_eq, keq = A.c_eq - A.c_star, kst = A.c_star;
            const float e = __fmul_rn(1.5f, RT);
            // 16-bit storage: this node's new reference record (rho, u, theta0, e); the
            // deviations written are taken against the equilibria computed here from it.
            float inv_f = 0.f, inv_g = 0.f;
            if constexpr (DEV) {
                if (act && in_bounds(out, N)) {
                    __stcs(reinterpret_cast<float4 *>(A.Rout) + out, make_float4(rho, ux, uy, uz));
                    __stcs(reinterpret_cast<float2 *>(A.Rout + 4ull * N) + out, make_float2(th, e));
                }
                inv_f = rcpa(rho);
                inv_g = THERMAL ? rcpa(rho * e) : 0.f;
            }
            // g^eq_i = rho [e PP_x PP_y PP_z + PS_x PP_y PP_z + PP_x PS_y PP_z + PP_x PP_y PS_z]
            //        = rho (e PP_x + PS_x) [PP_y PP_z] + rho PP_x [PS_y PP_z + PP_y PS_z],
            // e = 3/2 RT, PP = Psi(u, theta0 + u^2), PS = Psi applied to (u^2/2,
            // theta0 u + u^3/2, theta0^2 + 5/2 theta0 u^2 + u^4/2); g* the same at
            // (u*, RT*) without Phi, plus g' = 1/2 c_i . q' on the |c| = 1 populations.
            float Ag[3], As[3], rpx[3], Sy[3], Sz[3], Ty[3], Tz[3], py[3], pz[3];
            float hq[3] = {0.f, 0.f, 0.f};
            if (THERMAL) {
                const float es = e - 0.5f * (Fx * Fx + Fy * Fy + Fz * Fz) * (lir * lir);
                auto psiS = [&](float v, float o3[3]) {
                    const float vv = v * v;
                    psi3_poly(0.5f * vv, v * (th + 0.5f * vv), th * th + vv * (2.5f * th + 0.5f * vv), o3);
                };
                float T[3], px[3];
                psi3(usx, th + usx * usx, px);
                psiS(usx, T);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Ag[k] = ref_A(rho, e, ex[k], refS(k - 1, ux, th));
                    rpx[k] = rho * px[k];
                    As[k] = rho * (es * px[k] + T[k]);
                    Sy[k] = refS(k - 1, uy, th);
                    Sz[k] = refS(k - 1, uz, th);
                }
                psiS(usy, Ty);
                psiS(usz, Tz);
                psi3(usy, th + usy * usy, py);
                psi3(usz, th + usz * usz, pz);
                hq[0] = 0.5f * qx;
                hq[1] = 0.5f * qy;
                hq[2] = 0.5f * qz;
            }
            auto sel3 = [](const float v[3], int k) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); };
            auto sel3u = [](const unsigned v[3], int k) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); };
            // One c_z layer of nine populations per pass; with 16-bit storage the passes are
            // not unrolled, which bounds how many source records the compiler keeps in flight.
#pragma unroll(DEV ? 1 : 3)
            for (int kz = 0; kz < 3; ++kz) {
                const int cz = kz - 1;
                const float ezk = sel3(ez, kz), szk = sel3(sz, kz);
                const unsigned zs = cz == 1 ? zo[0] : (cz == 0 ? zo[1] : zo[2]);     // plane of z - c_z
                float E[3], Sl[3];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    E[j] = __fmul_rn(ey[j], ezk);
                    Sl[j] = sy[j] * szk;
                }
                const float iwz = cz ? 6.f : 1.5f;
                float hf9[9];                                 // pulled f of this layer (stage A's stash)
                if constexpr (GST) {
                    // 16-bit thermal: the pulled g of this layer from stage C's stash, the f of
                    // layers c_z = -1, 0 from stage A's, those of c_z = +1 decoded again from
                    // their source records (Eq. feq at the record).
                    // f first (its output written before the g are loaded: fewer live registers)
                    auto emit_f = [&](int cx, float Ey, float Sly, float iwxy, unsigned i, float hf) {
                        const float feq = ref_f_of(rex[cx + 1], Ey);
                        const float vf = kh * hf + keq * feq + kst * (rsx[cx + 1] * Sly);
                        if (act) stc(A.fo, i * N + out, 27ull * N, (vf - feq) * (inv_f * (iwxy * iwz)));
                    };
                    if (kz < 2) {
                        tm_ld9f(tmt, (p + 4) & 3, kz, hf9);
#pragma unroll
                        for (int j = 0; j < 9; ++j) {
                            const int cx = j % 3 - 1, cy = j / 3 - 1;
                            emit_f(cx, E[cy + 1], Sl[cy + 1], (cx ? 6.f : 1.5f) * (cy ? 6.f : 1.5f),
                                   (unsigned)j + 9u * (unsigned)kz, hf9[j]);
                        }
                    } else {
                        // c_z = +1 (sources in plane p - 1): decoded as decode_f does, one row of
                        // three sources at a time (bounds the records in flight)
#pragma unroll 1
                        for (int cy = -1; cy <= 1; ++cy) {
                            const float Ey = sel3(E, cy + 1), Sly = sel3(Sl, cy + 1);
                            const unsigned yo = sel3u(cD.yo, 1 - cy);
#pragma unroll
                            for (int cx = -1; cx <= 1; ++cx) {
                                const unsigned sn = zo[0] + yo + cD.xo[1 - cx];
                                const unsigned i = 18u + 3u * (unsigned)(cy + 1) + (unsigned)(cx + 1);
                                const Ref16 r = ldrec(A.Rin, sn, N);
                                const float rPx = __fmul_rn(r.rho, refP(cx, r.u[0], r.th));
                                const float PyPz = __fmul_rn(refP(cy, r.u[1], r.th), refP(1, r.u[2], r.th));
                                const float w = cy ? wgt16<27>(cx, 1, 1) : wgt16<27>(cx, 0, 1);
                                const float hf = __fmaf_rn(__fmul_rn(w, r.rho), ldc(A.f, i * N + sn, 27ull * N),
                                                           ref_f_of(rPx, PyPz));
                                emit_f(cx, Ey, Sly, (cx ? 6.f : 1.5f) * (cy ? 6.f : 1.5f), i, hf);
                            }
                        }
                    }
                    // then the g of this layer, from stage C's stash
                    float hg9[9];
                    tm_ld9(tmt + (uint32_t)(((p + 4) & 1) * TM_SLOT), kz, hg9);
                    const float Szk = sel3(Sz, kz), pzk = sel3(pz, kz), Tzk = sel3(Tz, kz);
                    float C[3], P[3], Dd[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        C[j] = ref_D(ey[j], Sy[j], ezk, Szk);
                        P[j] = py[j] * pzk;
                        Dd[j] = Ty[j] * pzk + py[j] * Tzk;
                    }
#pragma unroll
                    for (int j = 0; j < 9; ++j) {
                        const int cx = j % 3 - 1, cy = j / 3 - 1;
                        const unsigned i = (unsigned)j + 9u * (unsigned)kz;
                        const float iw = (cx ? 6.f : 1.5f) * (cy ? 6.f : 1.5f) * iwz;
                        const float geq = ref_g_of(Ag[cx + 1], rex[cx + 1], E[cy + 1], C[cy + 1]);
                        float gst = As[cx + 1] * P[cy + 1] + rpx[cx + 1] * Dd[cy + 1];
                        if (cx != 0 && cy == 0) gst += cz == 0 ? cx * hq[0] : 0.f;
                        if (cx == 0 && cy != 0) gst += cz == 0 ? cy * hq[1] : 0.f;
                        if (cx == 0 && cy == 0) gst += float(cz) * hq[2];
                        const float vg = kh * hg9[j] + keq * geq + kst * gst;
                        if (act) stc(A.go, i * N + out, 27ull * N, (vg - geq) * (inv_g * iw));
                    }
                } else {
                    tm_ld9(tmp, kz, hf9);
#pragma unroll
                    for (int j = 0; j < 9; ++j) {
                        const int cx = j % 3 - 1, cy = j / 3 - 1;
                        const unsigned i = (unsigned)j + 9u * (unsigned)kz;
                        const float h = hf9[j];
                        const float feq = ref_f_of(rex[cx + 1], E[cy + 1]);
                        float v = kh * h + keq * feq + kst * (rsx[cx + 1] * Sl[cy + 1]);
                        if constexpr (DEV)
                            v = (v - feq) * (inv_f * ((cx ? 6.f : 1.5f) * (cy ? 6.f : 1.5f) * iwz));
                        // The output is not read again this step: a streaming store keeps L2 for
                        // the populations the stages still share.
                        if (act) stc(A.fo, i * N + out, 27ull * N, v);
                    }
                    if (THERMAL) {
                        const float Szk = sel3(Sz, kz), pzk = sel3(pz, kz), Tzk = sel3(Tz, kz);
                        float C[3], P[3], Dd[3];
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            C[j] = ref_D(ey[j], Sy[j], ezk, Szk);
                            P[j] = py[j] * pzk;
                            Dd[j] = Ty[j] * pzk + py[j] * Tzk;
                        }
#pragma unroll
                        for (int j = 0; j < 9; ++j) {
                            const int cx = j % 3 - 1, cy = j / 3 - 1;
                            const unsigned sn = zs + cD.yo[1 - cy] + cD.xo[1 - cx];
                            const unsigned i = (unsigned)j + 9u * (unsigned)kz;
                            const float h = PRE ? gD[i] : ldc(A.g, i * N + sn, 27ull * N);   // FP32 storage here
                            const float geq = ref_g_of(Ag[cx + 1], rex[cx + 1], E[cy + 1], C[cy + 1]);
                            float gst = As[cx + 1] * P[cy + 1] + rpx[cx + 1] * Dd[cy + 1];
                            // g' on the |c| = 1 populations
                            if (cx != 0 && cy == 0) gst += cz == 0 ? cx * hq[0] : 0.f;
                            if (cx == 0 && cy != 0) gst += cz == 0 ? cy * hq[1] : 0.f;
                            if (cx == 0 && cy == 0) gst += float(cz) * hq[2];
                            if (act) stc(A.go, i * N + out, 27ull * N, kh * h + keq * geq + kst * gst);
                        }
                    }
                }
            }
        }
    }
    tmem::fence_sync();
    if (t < 32) tmem::dealloc(tm_base_sh, TM_COLS);
}

template <bool THERMAL, typename S>
cudaError_t launch(const Args<S> &A, cudaStream_t st)
{
    using G = typename TileOf<S>::G;
    static int attr_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_dev != dev) {
        e = cudaFuncSetAttribute(k_fused3d<THERMAL, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const dim3 grid((A.nx + G::TX - 1) / G::TX, (A.ny + G::TY - 1) / G::TY, A.nfull + A.ntail);
    k_fused3d<THERMAL, S><<<grid, G::NT, G::SMEM_BYTES, st>>>(A);
    return cudaGetLastError();
}

template <typename S>
cudaError_t step_t(const KParams &p, const void *f, const void *g, void *fo, void *go, const void *RT_iso,
                   const void *Rin, void *Rout, cudaStream_t st)
{
    Args<S> A;
    A.f = static_cast<const S *>(f);
    A.g = static_cast<const S *>(g);
    A.fo = static_cast<S *>(fo);
    A.go = static_cast<S *>(go);
    A.Rin = static_cast<const float *>(Rin);
    A.Rout = static_cast<float *>(Rout);
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
    A.HZ = p.tile_h > 0 ? p.tile_h : (p.nz < 64 ? p.nz : 64);
    // Chunks of HZ planes while more than 2 HZ remain, then the rest halved down to
    // kMinTail planes: CTAs start in chunk order, so the short chunks fill the last wave.
    // Chunks of at most 2 kMinTail planes are all HZ (the last one what is left).
    const int H = A.HZ < p.nz ? A.HZ : p.nz;
    A.HZ = H;
    A.tail[0] = 0;
    if (H > 2 * kMinTail) {
        A.nfull = p.nz > 2 * H ? (p.nz - 2 * H + H - 1) / H : 0;
        const int R = p.nz - A.nfull * H;
        int off = 0, k = 0;
        while (off < R) {
            const int rem = R - off;
            off += (rem > 2 * kMinTail && k < kMaxTail - 1) ? (rem + 1) / 2 : rem;
            A.tail[++k] = off;
        }
        A.ntail = k;
    } else {
        A.nfull = (p.nz - 1) / H;
        A.tail[1] = p.nz - A.nfull * H;
        A.ntail = 1;
    }
    return p.thermal ? launch<true, S>(A, st) : launch<false, S>(A, st);
}

}  // namespace

EVLBM_DEFINE_OOB_READER(fused3d_oob)

int fused3d_tile_w(int prec)
{
    return prec == 1 ? TileOf<float>::G::TX : TileOf<__half>::G::TX;
}

bool fused3d_supported(int prec, int Q, const KParams &p)
{
    return prec >= 1 && prec <= 3 && Q == 27 && p.force_form == 0 && !p.walls && (long long)27 * p.N < (1LL << 31);
}

cudaError_t fused3d_step(int prec, const KParams &p, const void *f, const void *g, void *fo, void *go,
                         const void *RT_iso, const void *Rin, void *Rout, cudaStream_t st)
{
    if (prec == 2) return step_t<__half>(p, f, g, fo, go, RT_iso, Rin, Rout, st);
    if (prec == 3) return step_t<__nv_bfloat16>(p, f, g, fo, go, RT_iso, Rin, Rout, st);
    return step_t<float>(p, f, g, fo, go, RT_iso, Rin, Rout, st);
}

}  // namespace evlbm

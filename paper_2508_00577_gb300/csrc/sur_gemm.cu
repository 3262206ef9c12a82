// Tensor-core GEMM of the learned surrogate.
//
// C[m][n] = sum_k A(m, k) B(n, k) with BF16 operands in shared memory,
// tcgen05.mma issued by one thread into an FP32 accumulator in tensor memory,
// and an epilogue (tcgen05.ld) that fuses bias, SiLU, the transposed-
// convolution pixel shuffle, the periodic halo copies, or the split-K sum.
//
// Activations are NHWC matrices stored halo-padded: [B][H+2][W+2][C], the
// border rows and columns holding periodic copies, so a 3x3 tap is a plain
// shifted window of the stored tensor.  Two mainloops feed the tensor core:
//   * TMA: the forward convolutions.  Each 64-deep K block of A is one (or,
//     for 32- and 8-channel inputs, 2 or 8) cp.async.bulk.tensor boxes of 128
//     pixels of the shifted window, swizzled 128/64 B (none for 8 channels); B
//     (the weights) is one swizzled box.  One thread issues the copies, one the
//     MMAs, four warps run the epilogue.
//   * cp.async: every other operand form (the adjoint gathers and the MN-major
//     weight-gradient operands); four producer warps, one MMA warp.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "surrogate.cuh"

namespace evsur {

namespace {

constexpr int BM = 128, BK = 64;
constexpr long kWaitLimit = 1L << 24;   // mbarrier polls before a CTA gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, lbo = byte stride between core
// matrices along K, sbo = byte stride between 8-row groups, layout = swizzle
// mode (0 none, 2 128-byte, 4 64-byte).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout = 0)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46) | ((uint64_t)layout << 61);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int *abort_flag = nullptr)
{
    uint32_t done = 0;
    for (long it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity));
        if (!done && abort_flag && (it & 63) == 63 && *abort_flag) return false;
    }
    return done != 0;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// 16-byte cp.async; an invalid chunk is zero-filled without reading memory.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0));
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }

// ---------------------------------------------------------------------------
// Epilogue (shared by both mainloops)
// ---------------------------------------------------------------------------
struct Epi {
    long long M;
    int N, epi;
    const float *bias;
    void *out;
    int ldo, co0;
    bf16 *y;
    int ldy, cy0;
    int shuf_cout;
    int pix, lh, lw;   // rows are interior pixels of a padded 2^lh x 2^lw grid
    int *status;
};

template <int BN>
__device__ __forceinline__ void epilogue(const Epi &g, uint32_t tmem, long long m0, int n0, int warp, int lane)
{
    const long long row = m0 + warp * 32 + lane;
    const bool rv = row < g.M;
    long long tg[4];
    int nt = 0;
    long long orow = row;
    if (rv && g.pix) {
        if (g.epi == SUR_EPI_SHUF) nt = 0;
        else nt = halo_targets(row, g.lh, g.lw, tg);
        orow = pad_pix(row, g.lh, g.lw);
    }
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (!rv) continue;
        const int col = n0 + c0;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
        if (g.epi == SUR_EPI_F32_ATOMIC) {
            float *o = static_cast<float *>(g.out) + row * g.ldo + g.co0 + col;
#pragma unroll
            for (int j = 0; j < 32; ++j) atomicAdd(o + j, v[j]);
        } else if (g.epi == SUR_EPI_SHUF) {
            const int sidx = col / g.shuf_cout, c = col - sidx * g.shuf_cout;
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] += g.bias[c + j];
            // Child s of coarse pixel `row` on the fine grid, with its halo copies.
            const int Hc = 1 << g.lh, Wc = 1 << g.lw;
            const long long b = row >> (g.lh + g.lw);
            const int y = (int)((row >> g.lw) & (Hc - 1)), x = (int)(row & (Wc - 1));
            const long long qf = ((b * 2 * Hc + 2 * y + (sidx >> 1)) << (g.lw + 1)) | (2 * x + (sidx & 1));
            long long ft[4];
            const int nf = halo_targets(qf, g.lh + 1, g.lw + 1, ft);
            for (int i = 0; i < nf; ++i) store32_bf16(g.y + ft[i] * g.ldy + g.cy0 + c, v);
        } else {
            if (g.bias) {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] += g.bias[col + j];
            }
            if (g.epi == SUR_EPI_F32) {
                float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(g.out) + orow * g.ldo + g.co0 + col);
#pragma unroll
                for (int j = 0; j < 8; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            } else {
                if (g.out) store32_bf16(static_cast<bf16 *>(g.out) + orow * g.ldo + g.co0 + col, v);
                if (g.epi == SUR_EPI_CONV) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = silu(v[j]);
                    if (g.pix) {
                        for (int i = 0; i < nt; ++i) store32_bf16(g.y + tg[i] * g.ldy + g.cy0 + col, v);
                    } else {
                        store32_bf16(g.y + row * g.ldy + g.cy0 + col, v);
                    }
                }
            }
        }
    }
}

template <int BN> struct Tmem {
    static constexpr int COLS = BN < 32 ? 32 : BN;
};

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, int cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, int cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// Instruction descriptor: FP32 accumulator, BF16 A and B, transpose flags for
// MN-major operands, N >> 3, M >> 4.
__device__ __forceinline__ uint32_t make_idesc(int bn, bool a_mn, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// ---------------------------------------------------------------------------
// cp.async mainloop
// ---------------------------------------------------------------------------

// Device-side operand description.
struct Op {
    const bf16 *p;
    int kind, ld, c0, rows;
    int lc, lh, lw;   // log2 C, log2 H, log2 W of the gather grid
};

// Per-thread loader state.  Producer thread t (0..127) owns ROWS/16 chunks of
// 16 bytes per stage:
//   K-major (DENSE, PIX, CONV3, UPADJ): rows (t >> 3) + 16 i, K group t & 7;
//     the rows' stored positions are computed once, a stage only adds the tap.
//   MN-major (TPIX, TCONV3, TUP): row group t % (ROWS/8) (one tap, 8 channels),
//     K indices (pixels) t / (ROWS/8) + (1024/ROWS) j.
template <int ROWS> struct Loader {
    static constexpr int NCH = ROWS / 16;
    long long base[NCH];   // K-major: element offset of the row (tap 0 / child 0 / channel c0)
    bool rv[NCH];
    int g, c;              // MN-major: row group and channel
    long long toff;        // MN-major: element offset of the tap / child
    bool gv;
};

template <int ROWS>
__device__ __forceinline__ void loader_init(const Op &o, Loader<ROWS> &L, long long row0, int t)
{
    if (o.kind <= SUR_OP_UPADJ) {
#pragma unroll
        for (int i = 0; i < Loader<ROWS>::NCH; ++i) {
            const long long q = row0 + (t >> 3) + 16 * i;
            L.rv[i] = q < o.rows;
            long long pos = q;
            if (o.kind == SUR_OP_PIX || o.kind == SUR_OP_CONV3) pos = pad_pix(q, o.lh, o.lw);
            else if (o.kind == SUR_OP_UPADJ) pos = child0(q, o.lh, o.lw);
            L.base[i] = pos * o.ld + o.c0;
        }
    } else {
        constexpr int G = ROWS / 8;
        L.g = t % G;
        const long long r0 = row0 + 8 * L.g;
        L.gv = r0 < o.rows;
        L.c = (int)r0;
        L.toff = 0;
        if (o.kind != SUR_OP_TPIX) {
            const int tap = (int)(r0 >> o.lc);
            L.c = (int)(r0 & ((1 << o.lc) - 1));
            L.gv = L.gv && tap < (o.kind == SUR_OP_TCONV3 ? 9 : 4);
            if (o.kind == SUR_OP_TCONV3) {
                const int dy = ((tap * 11) >> 5) - 1, dx = tap - 3 * (dy + 1) - 1;
                L.toff = (long long)(dy * ((1 << o.lw) + 2) + dx) * o.ld;
            } else {
                L.toff = (long long)((tap >> 1) * (2 * (1 << o.lw) + 2) + (tap & 1)) * o.ld;
            }
        }
    }
}

// Fill one ROWS x 64 operand tile (no swizzle) for the K block at kbase
// (K indices >= kend read zero).
//   K-major: core matrix (row group r/8, k group k/8) at ((r/8)*8 + k/8)*128 B,
//            row r%8 at +16 B (LBO = 128, SBO = 1024).
//   MN-major: core matrix (k group k/8, row group g) at ((k/8)*(ROWS/8) + g)*128 B,
//            k%8 at +16 B (SBO = 128, LBO = ROWS*16).
template <int ROWS>
__device__ __forceinline__ void load_tile(const Op &o, const Loader<ROWS> &L, uint32_t s, long long kbase,
                                          long long kend, int t)
{
    constexpr int NCH = Loader<ROWS>::NCH;
    if (o.kind <= SUR_OP_UPADJ) {
        const int k8 = t & 7;
        const long long k = kbase + k8 * 8;
        bool kval = k < kend;
        long long off = k;
        if (o.kind == SUR_OP_PIX) {
            kval = kval && k < (1LL << o.lc);
        } else if (o.kind != SUR_OP_DENSE) {
            const int q = (int)(k >> 3);
            const int tap = q >> (o.lc - 3);
            const int cc = (q & ((1 << (o.lc - 3)) - 1)) << 3;
            if (o.kind == SUR_OP_CONV3) {
                kval = kval && tap < 9;
                const int dy = ((tap * 11) >> 5) - 1, dx = tap - 3 * (dy + 1) - 1;
                off = (long long)(dy * ((1 << o.lw) + 2) + dx) * o.ld + cc;
            } else {
                kval = kval && tap < 4;
                off = (long long)((tap >> 1) * (2 * (1 << o.lw) + 2) + (tap & 1)) * o.ld + cc;
            }
        }
        const uint32_t sk = s + (uint32_t)(k8 * 128 + ((t >> 3) & 7) * 16 + ((t >> 6) << 10));
#pragma unroll
        for (int i = 0; i < NCH; ++i) {
            const bool v = kval && L.rv[i];
            cp_async16(sk + (uint32_t)(i * 2048), v ? o.p + L.base[i] + off : o.p, v);
        }
    } else {
        constexpr int G = ROWS / 8;
        constexpr int KSTEP = 128 / G;
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            const int k = t / G + KSTEP * j;
            const long long q = kbase + k;
            const bool v = L.gv && q < kend;
            const bf16 *src = o.p;
            if (v) {
                const long long pos = o.kind == SUR_OP_TUP ? child0(q, o.lh, o.lw) : pad_pix(q, o.lh, o.lw);
                src = o.p + pos * o.ld + L.toff + o.c0 + L.c;
            }
            cp_async16(s + (uint32_t)(((k >> 3) * G + L.g) * 128 + (k & 7) * 16), src, v);
        }
    }
}

struct KArgs {
    Op a, b;
    long long K, kps;   // K per split, multiple of BK
    Epi e;
};

template <int BN> struct CfgA {
    static constexpr int NS = BN <= 64 ? 4 : 3;
    static constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = NS * STAGE;
};

// Warps 0-3: producers, then epilogue; warp 4: MMA issuer.
//   full[s]  (128 arrivals, cp.async.mbarrier.arrive.noinc): stage s landed;
//   empty[s] (tcgen05.commit): the MMAs that read stage s completed;
//   done     (tcgen05.commit): every MMA of the tile completed.
template <int BN>
__global__ void __launch_bounds__(160, 1) k_gemm_cpasync(const KArgs g)
{
    using C = CfgA<BN>;
    constexpr int NS = C::NS;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS], done_bar;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const long long kbeg = (long long)blockIdx.z * g.kps;
    long long kend = kbeg + g.kps;
    if (kend > g.K) kend = g.K;
    const int nkb = kend > kbeg ? (int)((kend - kbeg + BK - 1) / BK) : 0;
    const bool a_mn = g.a.kind >= SUR_OP_TPIX, b_mn = g.b.kind >= SUR_OP_TPIX;
    volatile int *abort_v = &abort_flag;

    if (warp == 0) tmem_alloc(&tmem_sh, Tmem<BN>::COLS);
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), 128);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_sh;
    const uint32_t sbase = smem_u32(dsm);

    if (warp < 4) {
        Loader<BM> La;
        Loader<BN> Lb;
        loader_init<BM>(g.a, La, m0, t);
        loader_init<BN>(g.b, Lb, n0, t);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % NS;
            if (kb >= NS && !mbar_wait(smem_u32(&empty[s]), ((kb / NS) - 1) & 1, abort_v)) {
                *abort_v = 1;
                break;
            }
            const uint32_t sa = sbase + (uint32_t)(s * C::STAGE);
            const long long kbase = kbeg + (long long)kb * BK;
            load_tile<BM>(g.a, La, sa, kbase, kend, t);
            load_tile<BN>(g.b, Lb, sa + C::A_BYTES, kbase, kend, t);
            // Arrives on full[s] once this thread's copies above have landed.
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s])));
        }
        asm volatile("cp.async.wait_all;");
        const bool fin = mbar_wait(smem_u32(&done_bar), 0);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!fin) *abort_v = 1;
        __syncwarp();
        // Warp-uniform: tcgen05.ld is a .sync.aligned warp instruction.
        if (__all_sync(0xffffffffu, fin && !*abort_v && nkb > 0)) epilogue<BN>(g.e, tmem, m0, n0, warp, lane);
    } else if (lane == 0) {
        const uint32_t idesc = make_idesc(BN, a_mn, b_mn);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % NS;
            if (!mbar_wait(smem_u32(&full[s]), (kb / NS) & 1, abort_v)) {
                *abort_v = 1;
                break;
            }
            // Written through the generic proxy (cp.async), read through the async proxy.
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = sbase + (uint32_t)(s * C::STAGE), sb = sa + C::A_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
                const uint64_t da =
                    a_mn ? smem_desc(sa + k * (BM * 32), BM * 16, 128) : smem_desc(sa + k * 256, 128, 1024);
                const uint64_t db =
                    b_mn ? smem_desc(sb + k * (BN * 32), BN * 16, 128) : smem_desc(sb + k * 256, 128, 1024);
                mma_bf16(tmem, da, db, idesc, (kb > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&empty[s]));
        }
        mma_commit(smem_u32(&done_bar));   // arrives once every MMA above completed
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (t == 0 && *abort_v) atomicExch(g.e.status, 1);
    if (warp == 0) tmem_free(tmem, Tmem<BN>::COLS);
}

// ---------------------------------------------------------------------------
// TMA mainloop (forward convolutions)
// ---------------------------------------------------------------------------
struct TArgs {
    int nkb;
    int mtiles, ntiles;   // tile grid (the launch grid is smaller: CTAs loop over tiles)
    int kind;          // SUR_OP_CONV3 or SUR_OP_PIX
    int lc, c0;        // log2 channels of the gathered tensor, first channel
    int lh, lw;        // interior grid of A
    int boxw, boxh;    // pixels of one box row, box rows (a tile is boxw * boxh * boxs pixels)
    int b_c0;          // first K column of B
    // MN-major mode (weight gradients: pixels along K, split over K):
    int a_cb, b_cb;    // channels per box (MN atom): 64 (128-byte swizzle), 32 (64-byte), 8 (none)
    int a_lbo, a_sbo, a_kstep, a_sw;   // smem descriptor of A: byte offsets, K-step advance, layout
    int b_lbo, b_sbo, b_kstep, b_sw;
    int splits;        // K splits (tiles = mtiles x ntiles x splits)
    long long K, kps;  // reduction length and K per split (multiples of 64)
    Epi e;
};

template <int BN> struct CfgT {
    // Two CTAs per SM: 97-101 KB of stages each.
    static constexpr int NS = BN == 128 ? 3 : (BN == 64 ? 4 : 5);
    static constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;   // multiple of 1024
    static constexpr int SMEM = NS * STAGE + 1024;    // + alignment slack
};

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Persistent TMA GEMM.  ASW: inner width of one A box in bytes (128: 64
// channels, swizzle 128 B; 64: 32 channels, swizzle 64 B; 16: 8 channels, no
// swizzle).  Each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... with
// two TMEM accumulators, so the epilogue of one tile overlaps the mainloop of
// the next.
//   warp 4 (one thread): TMA producer        full[s]   <- expect_tx + TMA bytes
//   warp 5 (one thread): MMA issuer          empty[s]  <- tcgen05.commit
//   warps 0-3: epilogue                      tfull[b]  <- tcgen05.commit (accumulator b ready)
//                                            tempty[b] <- 128 epilogue arrivals (b drained)
// Tile of the persistent loop: output block (m0, n0) and its K range.  MN-major mode
// orders tiles (split, m, n), n fastest, so that tiles over the same pixels run together.
struct TileCoord {
    long long m0, kbeg;
    int n0, nkb;
};

template <bool MN>
__device__ __forceinline__ TileCoord tile_coord(const TArgs &g, int tile)
{
    TileCoord c;
    if (MN) {
        const int per = g.mtiles * g.ntiles, sp = tile / per, rem = tile - sp * per;
        c.m0 = (long long)(rem / g.ntiles) * BM;
        c.n0 = rem % g.ntiles;
        c.kbeg = (long long)sp * g.kps;
        const long long kend = c.kbeg + g.kps < g.K ? c.kbeg + g.kps : g.K;
        c.nkb = (int)((kend - c.kbeg) / BK);
    } else {
        c.m0 = (long long)(tile / g.ntiles) * BM;
        c.n0 = tile % g.ntiles;
        c.kbeg = 0;
        c.nkb = g.nkb;
    }
    return c;
}

// MN = true: weight-gradient form, A = TCONV3 or TPIX and B = TPIX (pixels along K),
// both MN-major.  A K block is 64 consecutive pixels (boxw x boxh of one image); each
// box loads one MN atom of cb channels for those 64 pixels, 64 rows of cb x 2 bytes:
// with cb = 64 a 128-byte-swizzled atom column (8-row groups 1 KB apart), cb = 32 a
// 64-byte-swizzled one (512 B), cb = 8 unswizzled core matrices (128 B).  Descriptors:
// swizzled MN-major layouts take LBO = stride between MN atoms and SBO = stride between
// 8-row K groups; the unswizzled one LBO = K-group stride and SBO = MN stride.
template <int BN, int ASW, bool MN>
__global__ void __launch_bounds__(192, 1)
    k_gemm_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TArgs g)
{
    using Cf = CfgT<BN>;
    constexpr int NS = Cf::NS;
    constexpr int CB = ASW / 2;               // channels per box
    constexpr int NBOX = 64 / CB;             // A boxes per K block
    constexpr int BOXB = BM * ASW;            // bytes per A box
    constexpr int TCOLS = 2 * BN < 32 ? 32 : 2 * BN;
    extern __shared__ unsigned char dsm_raw[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull[2], tempty[2], done_bar;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    volatile int *abort_v = &abort_flag;
    const int ntiles = g.mtiles * g.ntiles * (MN ? g.splits : 1);

    if (warp == 0) tmem_alloc(&tmem_sh, TCOLS);
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), 128);
        }
        mbar_init(smem_u32(&done_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_sh;
    const uint32_t sbase = (smem_u32(dsm_raw) + 1023u) & ~1023u;   // swizzle atoms need 1024-byte alignment

    if (warp == 4) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            const int H = 1 << g.lh, W = 1 << g.lw;
            long long it = 0;
            bool ok = true;
            if constexpr (MN) {
                const int nsa = BM / g.a_cb, nsb = BN / g.b_cb;
                const int boxw = W < 64 ? W : 64;
                for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                    const TileCoord tc = tile_coord<true>(g, tile);
                    for (int kb = 0; kb < tc.nkb; ++kb, ++it) {
                        const int s = (int)(it % NS);
                        if (it >= NS && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((it / NS) - 1) & 1), abort_v)) {
                            *abort_v = 1;
                            ok = false;
                            break;
                        }
                        const uint32_t sa = sbase + (uint32_t)(s * Cf::STAGE), sb = sa + Cf::A_BYTES;
                        const uint32_t bar = smem_u32(&full[s]);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                                     "r"((uint32_t)Cf::STAGE));
                        const long long q = tc.kbeg + (long long)kb * BK;      // first pixel of the block
                        const int b = (int)(q >> (g.lh + g.lw));
                        const int y = (int)((q >> g.lw) & (H - 1)), x = (int)(q & (W - 1));
                        (void)boxw;
                        for (int sg = 0; sg < nsa; ++sg) {
                            const long long r = tc.m0 + (long long)sg * g.a_cb;
                            int tap = 4, c = (int)r;
                            if (g.kind == SUR_OP_TCONV3) {
                                tap = (int)(r >> g.lc);
                                c = (int)(r & ((1 << g.lc) - 1));
                            }
                            const int dy = ((tap * 11) >> 5) - 1, dx = tap - 3 * (dy + 1) - 1;
                            // Rows of taps 9.. (M padding) load a box wholly below the tensor: zeros.
                            const bool tv = tap < 9;
                            tma_load_4d(sa + (uint32_t)(sg * g.a_cb * 128), &tmA, g.c0 + c, tv ? x + 1 + dx : 0,
                                        tv ? y + 1 + dy : H + 2, b, bar);
                        }
                        for (int sg = 0; sg < nsb; ++sg)
                            tma_load_4d(sb + (uint32_t)(sg * g.b_cb * 128), &tmB, g.b_c0 + tc.n0 * BN + sg * g.b_cb,
                                        x + 1, y + 1, b, bar);
                    }
                }
            } else
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const long long m0 = (long long)(tile / g.ntiles) * BM;
                const int n0 = (tile % g.ntiles) * BN;
                const int b0 = (int)(m0 >> (g.lh + g.lw));
                const int y0 = (int)((m0 >> g.lw) & (H - 1)), x0 = (int)(m0 & (W - 1));
                for (int kb = 0; kb < g.nkb; ++kb, ++it) {
                    const int s = (int)(it % NS);
                    if (it >= NS && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((it / NS) - 1) & 1), abort_v)) {
                        *abort_v = 1;
                        ok = false;
                        break;
                    }
                    const uint32_t sa = sbase + (uint32_t)(s * Cf::STAGE);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[s])),
                                 "r"((uint32_t)Cf::STAGE));
#pragma unroll
                    for (int j = 0; j < NBOX; ++j) {
                        const int k = kb * 64 + j * CB;          // first K index of the box
                        int tap = 4, cc = k;                     // PIX: centre tap, channels k..
                        if (g.kind == SUR_OP_CONV3) {
                            tap = k >> g.lc;
                            cc = k & ((1 << g.lc) - 1);
                        }
                        const int dy = ((tap * 11) >> 5) - 1, dx = tap - 3 * (dy + 1) - 1;
                        // Taps 9.. (K padding) load a box wholly below the tensor: zeros.
                        const int yc = tap < 9 ? y0 + 1 + dy : H + 2;
                        tma_load_4d(sa + j * BOXB, &tmA, g.c0 + cc, x0 + 1 + dx, yc, b0, smem_u32(&full[s]));
                    }
                    tma_load_2d(sa + Cf::A_BYTES, &tmB, g.b_c0 + kb * 64, n0, smem_u32(&full[s]));
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = make_idesc(BN, MN, MN);
            long long it = 0;
            int lt = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
                const int nkb = tile_coord<MN>(g, tile).nkb;
                const int buf = lt & 1;
                if (lt >= 2 && !mbar_wait(smem_u32(&tempty[buf]), (uint32_t)(((lt >> 1) - 1) & 1), abort_v)) {
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t acc_t = tmem + (uint32_t)(buf * BN);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % NS);
                    if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((it / NS) & 1), abort_v)) {
                        *abort_v = 1;
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t sa = sbase + (uint32_t)(s * Cf::STAGE), sb = sa + Cf::A_BYTES;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {
                        if constexpr (MN) {
                            const uint64_t da = smem_desc(sa + k * g.a_kstep, g.a_lbo, g.a_sbo, g.a_sw);
                            const uint64_t db = smem_desc(sb + k * g.b_kstep, g.b_lbo, g.b_sbo, g.b_sw);
                            mma_bf16(acc_t, da, db, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                            continue;
                        }
                        uint64_t da;
                        if (ASW == 128) da = smem_desc(sa + k * 32, 16, 1024, 2);
                        else if (ASW == 64) da = smem_desc(sa + (k >> 1) * BOXB + (k & 1) * 32, 16, 512, 4);
                        else da = smem_desc(sa + k * 2 * BOXB, BOXB, 128, 0);
                        const uint64_t db = smem_desc(sb + k * 32, 16, 1024, 2);
                        mma_bf16(acc_t, da, db, idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&empty[s]));
                }
                if (ok) mma_commit(smem_u32(&tfull[buf]));
            }
            mma_commit(smem_u32(&done_bar));   // arrives once every MMA above completed
        }
    } else {
        // ---------------- epilogue (warps 0-3) ----------------
        int lt = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
            const int buf = lt & 1;
            const bool ready = mbar_wait(smem_u32(&tfull[buf]), (uint32_t)((lt >> 1) & 1), abort_v);
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!__all_sync(0xffffffffu, ready && !*abort_v)) {
                *abort_v = 1;
                break;
            }
            const TileCoord tc = tile_coord<MN>(g, tile);
            epilogue<BN>(g.e, tmem + (uint32_t)(buf * BN), tc.m0, tc.n0 * BN, warp, lane);
            asm volatile("tcgen05.fence::before_thread_sync;");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])));
        }
        // Tensor memory must be idle before it is freed.
        if (!mbar_wait(smem_u32(&done_bar), 0)) *abort_v = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (t == 0 && *abort_v) atomicExch(g.e.status, 1);
    if (warp == 0) tmem_free(tmem, TCOLS);
}

}  // namespace

}  // namespace evsur

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace evsur {

namespace {

bool g_tma_enabled = true;

int ilog2(long long v)
{
    int l = 0;
    while (l < 62 && (1LL << l) < v) ++l;
    return (1LL << l) == v ? l : -1;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Validate a public operand and convert it; false if it is malformed.
bool make_op(const sur_operand &s, Op &o)
{
    if (!s.p || !aligned16(s.p) || s.kind < SUR_OP_DENSE || s.kind > SUR_OP_TUP) return false;
    if (s.ld <= 0 || s.ld % 8 || s.c0 < 0 || s.c0 % 8 || s.rows < 0) return false;
    o.p = static_cast<const bf16 *>(s.p);
    o.kind = s.kind;
    o.ld = s.ld;
    o.c0 = s.c0;
    o.rows = s.rows;
    o.lc = o.lh = o.lw = 0;
    if (s.kind == SUR_OP_DENSE) return true;
    o.lh = ilog2(s.H);
    o.lw = ilog2(s.W);
    if (o.lh < 0 || o.lw < 0) return false;
    if (s.kind == SUR_OP_TPIX) return true;
    o.lc = ilog2(s.C);
    return o.lc >= 3 && s.c0 + s.C <= s.ld;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

template <class K>
cudaError_t set_smem(K kernel, int bytes, int &attr_dev)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_dev != dev) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    return cudaSuccess;
}

template <int BN>
cudaError_t launch_cpasync(const KArgs &g, long long mtiles, int splits, cudaStream_t st)
{
    static int attr_dev = -1;
    cudaError_t e = set_smem(k_gemm_cpasync<BN>, CfgA<BN>::SMEM, attr_dev);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)mtiles, (unsigned)(g.e.N / BN), (unsigned)splits);
    k_gemm_cpasync<BN><<<grid, 160, CfgA<BN>::SMEM, st>>>(g);
    return cudaGetLastError();
}

template <int BN, int ASW, bool MN = false>
cudaError_t launch_tma(const CUtensorMap &ma, const CUtensorMap &mb, const TArgs &g, long long mtiles,
                       cudaStream_t st)
{
    static int attr_dev = -1, sms = 0;
    cudaError_t e = set_smem(k_gemm_tma<BN, ASW, MN>, CfgT<BN>::SMEM, attr_dev);
    if (e != cudaSuccess) return e;
    if (!sms) {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    }
    TArgs gg = g;
    gg.mtiles = (int)mtiles;
    gg.ntiles = g.e.N / BN;
    const long long tiles = (long long)gg.mtiles * gg.ntiles * (MN ? gg.splits : 1);
    const long long ctas = tiles < 2LL * sms ? tiles : 2LL * sms;   // two resident CTAs per SM
    k_gemm_tma<BN, ASW, MN><<<(unsigned)ctas, 192, CfgT<BN>::SMEM, st>>>(ma, mb, gg);
    return cudaGetLastError();
}

template <int ASW>
cudaError_t dispatch_tma(int N, const CUtensorMap &ma, const CUtensorMap &mb, const TArgs &g, long long mtiles,
                         cudaStream_t st)
{
    if (N % 128 == 0) return launch_tma<128, ASW>(ma, mb, g, mtiles, st);
    if (N % 64 == 0) return launch_tma<64, ASW>(ma, mb, g, mtiles, st);
    return launch_tma<32, ASW>(ma, mb, g, mtiles, st);
}

// Tensor maps of a TMA-eligible GEMM; false if the encoder rejects them.
bool make_maps(const sur_gemm_args &a, int bn, CUtensorMap &ma, CUtensorMap &mb, TArgs &tg)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    const int C = a.a.C, H = a.a.H, W = a.a.W;
    const int cb = C >= 64 ? 64 : C;
    const int boxw = W < 128 ? W : 128;
    const int boxh = H < 128 / boxw ? H : 128 / boxw;
    const int boxs = 128 / (boxw * boxh);
    const long long samples = (long long)a.a.rows / ((long long)H * W);
    const size_t e2 = 2;
    cuuint64_t dims[4] = {(cuuint64_t)a.a.ld, (cuuint64_t)(W + 2), (cuuint64_t)(H + 2), (cuuint64_t)samples};
    cuuint64_t strides[3] = {a.a.ld * e2, (cuuint64_t)(W + 2) * a.a.ld * e2,
                             (cuuint64_t)(H + 2) * (W + 2) * a.a.ld * e2};
    cuuint32_t box[4] = {(cuuint32_t)cb, (cuuint32_t)boxw, (cuuint32_t)boxh, (cuuint32_t)boxs};
    cuuint32_t es[4] = {1, 1, 1, 1};
    const CUtensorMapSwizzle sw = cb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                           : (cb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE);
    if (enc(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(a.a.p), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    cuuint64_t bdims[2] = {(cuuint64_t)a.b.ld, (cuuint64_t)a.b.rows};
    cuuint64_t bstr[1] = {a.b.ld * e2};
    cuuint32_t bbox[2] = {64, (cuuint32_t)bn};
    cuuint32_t bes[2] = {1, 1};
    if (enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(a.b.p), bdims, bstr, bbox, bes,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    tg.nkb = a.K / 64;
    tg.kind = a.a.kind;
    tg.lc = ilog2(C);
    tg.c0 = a.a.c0;
    tg.lh = ilog2(H);
    tg.lw = ilog2(W);
    tg.boxw = boxw;
    tg.boxh = boxh;
    tg.b_c0 = a.b.c0;
    return true;
}

// Weight-gradient GEMMs: A = TCONV3 or TPIX, B = TPIX on the same pixel grid, dense FP32
// output.  Rows of A at or beyond `rows` must read zero: TCONV3 rows of taps >= 9 load
// boxes wholly outside the tensor (zeros), so M may exceed `rows` when rows >= 9 C (the
// K padding of the weights); any other row range must lie inside `rows`.
bool tma_mn_eligible(const sur_gemm_args &a)
{
    if (!g_tma_enabled || a.b.kind != SUR_OP_TPIX) return false;
    if (a.a.kind != SUR_OP_TCONV3 && a.a.kind != SUR_OP_TPIX) return false;
    if (a.epi != SUR_EPI_F32_ATOMIC && a.epi != SUR_EPI_F32) return false;
    if (a.K % 64 || a.a.H != a.b.H || a.a.W != a.b.W || a.a.W < 8 || a.a.H < 1) return false;
    const long long hw = (long long)a.a.H * a.a.W;
    if (a.K % hw || a.N > a.b.rows) return false;
    if (a.M > a.a.rows && !(a.a.kind == SUR_OP_TCONV3 && a.a.rows >= 9 * a.a.C)) return false;
    if (hw % 64) return false;
    if (a.a.kind == SUR_OP_TCONV3 && !(a.a.C == 8 || a.a.C == 32 || a.a.C % 64 == 0)) return false;
    return true;
}

// Tensor maps of the MN-major form: (channels, x, y, image) over the halo-padded NHWC
// tensor, boxes {cb channels, boxw, boxh, 1} of 64 pixels; descriptor fields per cb.
bool make_maps_mn(const sur_gemm_args &a, int bn, CUtensorMap &ma, CUtensorMap &mb, TArgs &tg)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    const int H = a.a.H, W = a.a.W;
    const long long images = a.K / ((long long)H * W);
    const int boxw = W < 64 ? W : 64, boxh = 64 / boxw;
    const int acb = a.a.kind == SUR_OP_TCONV3 ? (a.a.C < 64 ? a.a.C : 64) : 64;
    const int bcb = bn < 64 ? bn : 64;
    if (!(acb == 64 || acb == 32 || acb == 8) || !(bcb == 64 || bcb == 32)) return false;
    auto encode = [&](CUtensorMap &m, const sur_operand &o, int cb) {
        const size_t e2 = 2;
        cuuint64_t dims[4] = {(cuuint64_t)o.ld, (cuuint64_t)(W + 2), (cuuint64_t)(H + 2), (cuuint64_t)images};
        cuuint64_t strides[3] = {o.ld * e2, (cuuint64_t)(W + 2) * o.ld * e2, (cuuint64_t)(H + 2) * (W + 2) * o.ld * e2};
        cuuint32_t box[4] = {(cuuint32_t)cb, (cuuint32_t)boxw, (cuuint32_t)boxh, 1};
        cuuint32_t es[4] = {1, 1, 1, 1};
        const CUtensorMapSwizzle sw = cb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                               : (cb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE);
        return enc(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(o.p), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!encode(ma, a.a, acb) || !encode(mb, a.b, bcb)) return false;
    // Descriptor fields: (lbo, sbo, k-step, layout) per channels of the MN atom.
    auto fields = [](int cb, int &lbo, int &sbo, int &kstep, int &sw) {
        if (cb == 64) { lbo = 8192; sbo = 1024; kstep = 2048; sw = 2; }
        else if (cb == 32) { lbo = 4096; sbo = 512; kstep = 1024; sw = 4; }
        else { lbo = 128; sbo = 1024; kstep = 256; sw = 0; }
    };
    fields(acb, tg.a_lbo, tg.a_sbo, tg.a_kstep, tg.a_sw);
    fields(bcb, tg.b_lbo, tg.b_sbo, tg.b_kstep, tg.b_sw);
    // A B tile of one MN atom (BN <= 64) never steps between atoms: LBO = SBO makes every
    // byte the tensor core can address lie inside the tile whichever field it reads.
    if (bn == bcb) tg.b_lbo = tg.b_sbo;
    const long long kb = a.K / 64;
    const long long kbps = (kb + a.splits - 1) / a.splits;
    tg.kind = a.a.kind;
    tg.lc = a.a.kind == SUR_OP_TCONV3 ? ilog2(a.a.C) : 0;
    tg.lh = ilog2(H);
    tg.lw = ilog2(W);
    tg.c0 = a.a.c0;
    tg.b_c0 = a.b.c0;
    tg.a_cb = acb;
    tg.b_cb = bcb;
    tg.K = a.K;
    tg.kps = kbps * 64;
    tg.splits = (int)((kb + kbps - 1) / kbps);   // every split non-empty
    tg.nkb = 0;
    return true;
}

bool tma_eligible(const sur_gemm_args &a)
{
    if (!g_tma_enabled || a.splits != 1 || a.epi == SUR_EPI_F32_ATOMIC) return false;
    if (a.b.kind != SUR_OP_DENSE || a.K % 64) return false;
    const int C = a.a.C;
    if (a.a.kind == SUR_OP_CONV3) {
        if (!(C == 8 || C == 32 || C % 64 == 0)) return false;
        if (a.K > (9 * C + 63) / 64 * 64) return false;
    } else if (a.a.kind == SUR_OP_PIX) {
        if (C % 64 || a.K > C) return false;
    } else {
        return false;
    }
    const long long hw = (long long)a.a.H * a.a.W;
    return hw > 0 && a.a.rows % hw == 0;
}

}  // namespace

void set_tma(bool on) { g_tma_enabled = on; }

int gemm(const sur_gemm_args &a, int *status, cudaStream_t st)
{
    if (!status || a.M < 1 || a.N < 32 || a.N % 32 || a.K < 1 || a.splits < 1) return SUR_EINVAL;
    if (a.splits > 1 && a.epi != SUR_EPI_F32_ATOMIC) return SUR_EINVAL;
    if (a.epi < SUR_EPI_BF16 || a.epi > SUR_EPI_SHUF) return SUR_EINVAL;
    KArgs g;
    if (!make_op(a.a, g.a) || !make_op(a.b, g.b)) return SUR_EINVAL;
    if (a.b.rows < a.N) return SUR_EINVAL;
    // Chunks are 8 elements wide: a dense operand's K tail and a TPIX operand's
    // last row group must stay inside the row of ld elements.
    const long long k8 = (a.K + 7) / 8 * 8;
    for (const sur_operand *o : {&a.a, &a.b}) {
        if (o->kind == SUR_OP_DENSE && o->c0 + k8 > o->ld) return SUR_EINVAL;
        if (o->kind == SUR_OP_TPIX && o->c0 + (o->rows + 7) / 8 * 8 > o->ld) return SUR_EINVAL;
    }
    Epi &e = g.e;
    e.M = a.M;
    e.N = a.N;
    e.epi = a.epi;
    e.bias = a.bias;
    e.out = a.out;
    e.ldo = a.ldo;
    e.co0 = a.co0;
    e.y = static_cast<bf16 *>(a.y);
    e.ldy = a.ldy;
    e.cy0 = a.cy0;
    e.shuf_cout = a.shuf_cout;
    // Output rows are pixels (stored padded) when A's rows are pixels.
    e.pix = (a.a.kind == SUR_OP_PIX || a.a.kind == SUR_OP_CONV3 || a.a.kind == SUR_OP_UPADJ) &&
            a.epi != SUR_EPI_F32_ATOMIC;
    e.lh = g.a.lh;
    e.lw = g.a.lw;
    e.status = status;
    const bool f32 = a.epi == SUR_EPI_F32 || a.epi == SUR_EPI_F32_ATOMIC;
    if (a.epi == SUR_EPI_CONV || a.epi == SUR_EPI_SHUF) {
        if (!a.y || !aligned16(a.y) || !a.bias || a.ldy % 8 || a.cy0 % 8 || a.cy0 < 0) return SUR_EINVAL;
    }
    if (a.epi == SUR_EPI_SHUF) {
        if (!e.pix || a.shuf_cout < 32 || a.shuf_cout % 32 || a.N != 4 * a.shuf_cout || a.cy0 + a.shuf_cout > a.ldy)
            return SUR_EINVAL;
    } else if (a.epi == SUR_EPI_CONV) {
        if (a.cy0 + a.N > a.ldy) return SUR_EINVAL;
        if (a.out && (!aligned16(a.out) || a.ldo % 8 || a.co0 % 8 || a.co0 < 0 || a.co0 + a.N > a.ldo))
            return SUR_EINVAL;
    } else {
        if (!a.out || !aligned16(a.out) || a.co0 + a.N > a.ldo || a.co0 < 0) return SUR_EINVAL;
        if (!f32 && (a.ldo % 8 || a.co0 % 8)) return SUR_EINVAL;
        if (a.epi == SUR_EPI_F32 && (a.ldo % 4 || a.co0 % 4)) return SUR_EINVAL;
    }
    const long long mtiles = (a.M + BM - 1) / BM;
    if (mtiles > 0x7FFFFFFF) return SUR_EINVAL;
    const int bn = a.N % 128 == 0 ? 128 : (a.N % 64 == 0 ? 64 : 32);
    cudaError_t err;
    if (tma_mn_eligible(a)) {
        CUtensorMap ma, mb;
        TArgs tg;
        if (make_maps_mn(a, bn, ma, mb, tg)) {
            tg.e = e;
            if (bn == 128) err = launch_tma<128, 16, true>(ma, mb, tg, mtiles, st);
            else if (bn == 64) err = launch_tma<64, 16, true>(ma, mb, tg, mtiles, st);
            else err = launch_tma<32, 16, true>(ma, mb, tg, mtiles, st);
            return err == cudaSuccess ? SUR_OK : SUR_ECUDA;
        }
    }
    if (tma_eligible(a)) {
        CUtensorMap ma, mb;
        TArgs tg;
        if (make_maps(a, bn, ma, mb, tg)) {
            tg.e = e;
            const int cb = a.a.C >= 64 ? 64 : a.a.C;
            if (cb == 64) err = dispatch_tma<128>(a.N, ma, mb, tg, mtiles, st);
            else if (cb == 32) err = dispatch_tma<64>(a.N, ma, mb, tg, mtiles, st);
            else err = dispatch_tma<16>(a.N, ma, mb, tg, mtiles, st);
            return err == cudaSuccess ? SUR_OK : SUR_ECUDA;
        }
    }
    g.K = a.K;
    const long long kb = (a.K + BK - 1) / BK;
    const long long kbps = (kb + a.splits - 1) / a.splits;
    g.kps = kbps * BK;
    const int splits = (int)((kb + kbps - 1) / kbps);
    if (bn == 128) err = launch_cpasync<128>(g, mtiles, splits, st);
    else if (bn == 64) err = launch_cpasync<64>(g, mtiles, splits, st);
    else err = launch_cpasync<32>(g, mtiles, splits, st);
    return err == cudaSuccess ? SUR_OK : SUR_ECUDA;
}

}  // namespace evsur

extern "C" int sur_gemm(const sur_gemm_args *g, int *d_status, void *stream)
{
    if (!g) return SUR_EINVAL;
    return evsur::gemm(*g, d_status, static_cast<cudaStream_t>(stream));
}

extern "C" int sur_set_tma(int enable)
{
    evsur::set_tma(enable != 0);
    return SUR_OK;
}
